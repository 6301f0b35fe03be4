// msm_impl.cuh -- templated MSM kernels and driver, instantiated once per
// group by msm_g1.cu and msm_g2.cu (see msm.cuh for the method).
#pragma once
#include "curve_quad.cuh"
#include "msm.cuh"

namespace ace {

// ---------------------------------------------------------------------------
// vectorised loads / stores of points (16-byte aligned arrays)
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T ld_vec(const T* p) {
    static_assert(sizeof(T) % 16 == 0, "16-byte multiple");
    T r;
    const uint4* s = reinterpret_cast<const uint4*>(p);
    uint4* d = reinterpret_cast<uint4*>(&r);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 16); i++) d[i] = __ldg(s + i);
    return r;
}
// A random gather of one 64-byte point (G1) or 128-byte point (G2) from a
// read-only table: the L2 prefetch-size hint asks for that many bytes from
// DRAM.  Without it the L2 filled a whole 128-byte line for every 64-byte
// point, almost twice the bytes the additions need.
template <class T>
__device__ __forceinline__ T ld_gather(const T* p) {
    static_assert(sizeof(T) == 64 || sizeof(T) == 128, "a 64- or 128-byte point");
    T r;
    const uint4* s = reinterpret_cast<const uint4*>(p);
    uint4* d = reinterpret_cast<uint4*>(&r);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 16); i++) {
        if constexpr (sizeof(T) == 64)
            asm("ld.global.nc.L2::64B.v4.u32 {%0, %1, %2, %3}, [%4];"
                : "=r"(d[i].x), "=r"(d[i].y), "=r"(d[i].z), "=r"(d[i].w)
                : "l"(s + i));
        else
            asm("ld.global.nc.L2::128B.v4.u32 {%0, %1, %2, %3}, [%4];"
                : "=r"(d[i].x), "=r"(d[i].y), "=r"(d[i].z), "=r"(d[i].w)
                : "l"(s + i));
    }
    return r;
}
template <class T>
__device__ __forceinline__ void st_vec(T* p, const T& v) {
    const uint4* s = reinterpret_cast<const uint4*>(&v);
    uint4* d = reinterpret_cast<uint4*>(p);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 16); i++) d[i] = s[i];
}
template <class T>
__device__ __forceinline__ T ld_plain(const T* p) {
    T r;
    const uint4* s = reinterpret_cast<const uint4*>(p);
    uint4* d = reinterpret_cast<uint4*>(&r);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 16); i++) d[i] = s[i];
    return r;
}

template <class F>
uint32_t bucket_split(const MsmPlan& p);

template <class F, class A>
template <class Alloc>
bool MsmBufs<F, A>::carve(Alloc& a, const MsmPlan& p, bool need_conv) {
    size_t keys = p.keys();
    offsets = (uint32_t*)a.take((keys + 1) * 4);
    cursor = (uint32_t*)a.take(keys * 4);
    scan_tmp = (uint32_t*)a.take(scan_tmp_words(keys + 1) * 4);
    entries = (uint32_t*)a.take(p.scalars() * (size_t)p.K * 4 + 4);
    order = (uint32_t*)a.take(keys * 4);
    size_bins = (uint32_t*)a.take((SIZE_BINS + 1) * 4);
    buckets = (Xyzz<F>*)a.take(keys * sizeof(Xyzz<F>));
    const uint32_t split = bucket_split<F>(p);
    partial = split > 1 ? (Xyzz<F>*)a.take(keys * split * sizeof(Xyzz<F>)) : buckets;
    segW = (Xyzz<F>*)a.take((size_t)p.all_windows() * p.M * sizeof(Xyzz<F>));
    segS = (Xyzz<F>*)a.take((size_t)p.all_windows() * p.M * sizeof(Xyzz<F>));
    need_conv = need_conv || p.glv || p.gls;
    conv = need_conv ? (Affine<F>*)a.take(p.n * sizeof(Affine<F>)) : nullptr;
    gsc = p.glv || p.gls ? (uint32_t*)a.take(p.n * 32) : nullptr;
    return offsets && cursor && scan_tmp && entries && order && size_bins && buckets && partial && segW && segS &&
           (!need_conv || conv) && (!(p.glv || p.gls) || gsc);
}

template <class F>
size_t msm_scratch_bytes(const MsmPlan& plan, bool base_mont) {
    Sizer s;
    MsmBufs<F, Sizer> b;
    b.carve(s, plan, !base_mont);
    return s.off + 256;
}

// ---------------------------------------------------------------------------
// bucket accumulation: one thread per bucket, one mixed addition per entry
// (ACE_BUCKET_MIN_BLOCKS: resident blocks of 128 threads per SM the compiler
// must allow, which caps the registers per thread)
// ---------------------------------------------------------------------------
#ifndef ACE_BUCKET_MIN_BLOCKS
#define ACE_BUCKET_MIN_BLOCKS 1
#endif
#ifndef ACE_BUCKET_MIN_BLOCKS_G2
#define ACE_BUCKET_MIN_BLOCKS_G2 1
#endif
template <class F>
__global__ void __launch_bounds__(128, sizeof(F) == sizeof(fp_t) ? ACE_BUCKET_MIN_BLOCKS : ACE_BUCKET_MIN_BLOCKS_G2)
    k_bucket_acc(const Affine<F>* __restrict__ bases,
                                                    const uint32_t* __restrict__ entries,
                                                    const uint32_t* __restrict__ offsets,
                                                    const uint32_t* __restrict__ order, uint32_t nkeys,
                                                    uint32_t split, Xyzz<F>* out) {
    // thread t adds part t % split of bucket order[t / split]; with split > 1
    // the partial sums go to out[key split + part] (combined below)
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nkeys * split) return;
    const uint32_t rank = t / split, part = t - rank * split;
    uint32_t key = __ldg(order + rank);
    uint32_t b0 = offsets[key], e0 = offsets[key + 1];
    uint32_t len = e0 - b0;
    uint32_t b = b0 + (uint32_t)(((uint64_t)len * part) / split);
    uint32_t e = b0 + (uint32_t)(((uint64_t)len * (part + 1)) / split);
    Xyzz<F> acc = xyzz_inf<F>();
    for (uint32_t i = b; i < e; i++) {
        uint32_t v = __ldg(entries + i);
        Affine<F> p = ld_gather(bases + (v & 0x7fffffffu));
        if (v >> 31) p.y = fe_neg(p.y);
        acc = xyzz_add_aff(acc, p);
    }
    st_vec(out + (size_t)key * split + part, acc);
}

// bucket = sum of its split partial sums (one thread per bucket)
template <class F>
__global__ void __launch_bounds__(128) k_bucket_combine(const Xyzz<F>* __restrict__ partial, uint32_t nkeys,
                                                        uint32_t split, Xyzz<F>* buckets) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nkeys) return;
    Xyzz<F> acc = ld_plain(partial + (size_t)k * split);
    for (uint32_t p = 1; p < split; p++) acc = xyzz_add(acc, ld_plain(partial + (size_t)k * split + p));
    st_vec(buckets + k, acc);
}

// Parts per bucket: when the keys are too few to fill the GPU (fewer than 4
// resident waves of the accumulation kernel) and the buckets are long, each
// bucket's entries are split among 2..16 threads (at least ~8 entries each)
// whose partial sums are then combined.  Entries per digit bucket are taken
// as n K / 2^(c-1) (tabled) or n / 2^(c-1) (one set per window).
template <class F>
uint32_t bucket_split(const MsmPlan& p) {
    // resident threads of the accumulation kernel, per device ordinal
    // (written once per device, always with that device's value)
    static double res_of[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    double res = dev >= 0 && dev < 64 ? res_of[dev] : 0.0;
    if (res <= 0.0) {
        int sms = 0, nb = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bucket_acc<F>, 128, 0);
        res = (double)(sms > 0 ? sms : 1) * (nb > 0 ? nb : 1) * 128.0;
        if (dev >= 0 && dev < 64) res_of[dev] = res;
    }
    const double keys = (double)p.keys();
    const double load = (double)p.n * (p.tabled ? p.K : 1) / (double)p.B;
    uint32_t S = 1;
    while (S < 16 && 2 * S <= p.max_split && keys * S < 4.0 * res && load / (2.0 * S) >= 8.0) S *= 2;
    return S;
}

// ---------------------------------------------------------------------------
// bucket reduction: segments of L buckets, then a weighted binary tree
// ---------------------------------------------------------------------------
template <class F>
__global__ void __launch_bounds__(128) k_seg_reduce(const Xyzz<F>* __restrict__ buckets, uint32_t nseg,
                                                    uint32_t B, uint32_t L, uint32_t M, uint32_t windows,
                                                    uint32_t ones, Xyzz<F>* segW, Xyzz<F>* segS) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nseg) return;
    uint32_t w = t / M, j = t % M;
    const Xyzz<F>* bk = buckets + (size_t)w * B + (size_t)j * L;
    Xyzz<F> run = xyzz_inf<F>(), acc = xyzz_inf<F>();
    if (w % windows == ones) {  // the ones window needs only its plain sum
        for (int b = (int)L - 1; b >= 0; b--) run = xyzz_add(run, ld_plain(bk + b));
    } else {
        for (int b = (int)L - 1; b >= 0; b--) {
            run = xyzz_add(run, ld_plain(bk + b));
            acc = xyzz_add(acc, run);
        }
    }
    st_vec(segW + t, acc);
    st_vec(segS + t, run);
}

// weighted segment values: bucket b of a window carries weight b + 1, so
// segment j (buckets jL .. jL + L - 1) contributes W_j + j L S_j; the ones
// window contributes its plain sum S_j.  P_j overwrites W_j.  One thread per
// segment: j L S_j by double-and-add (at most c - 1 doublings).
template <class F>
__global__ void __launch_bounds__(128) k_seg_weight(Xyzz<F>* W, const Xyzz<F>* __restrict__ S, uint32_t nseg,
                                                    uint32_t M, int lambda, uint32_t windows, uint32_t ones) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nseg) return;
    const uint32_t w = t / M, j = t % M;
    Xyzz<F> s = ld_plain(S + t);
    if (w % windows == ones) {
        st_vec(W + t, s);
        return;
    }
    Xyzz<F> acc = ld_plain(W + t);
    if (j != 0) {
        Xyzz<F> m = xyzz_inf<F>();
        for (int b = 31 - __clz(j); b >= 0; b--) {
            m = xyzz_dbl(m);
            if ((j >> b) & 1u) m = xyzz_add(m, s);
        }
        for (int k = 0; k < lambda; k++) m = xyzz_dbl(m);
        acc = xyzz_add(acc, m);
    }
    st_vec(W + t, acc);
}

// The same two steps on four lanes per segment (curve_quad.cuh).  A
// reduction with few segments leaves most of the GPU idle, and each
// thread's time is its chain of additions (about 16 products in sequence
// each, against 4 levels of products on four lanes).  With more segments
// than about one wave of the four-lane kernel holds, or beside other proofs'
// kernels, the one-lane form is faster: it does the same products without
// the shuffles and the repeated additions of the four lanes.
template <class F>
__global__ void __launch_bounds__(128) k_seg_reduce_quad(const Xyzz<F>* __restrict__ buckets, uint32_t nseg,
                                                         uint32_t B, uint32_t L, uint32_t M, uint32_t windows,
                                                         uint32_t ones, Xyzz<F>* segW, Xyzz<F>* segS) {
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t t = gt >> 2;
    const int sub = (int)(gt & 3u);
    if (t >= nseg) return;  // whole groups of four leave together
    const unsigned mask = 0xfu << (threadIdx.x & 28u);
    const uint32_t w = t / M, j = t % M;
    const Xyzz<F>* bk = buckets + (size_t)w * B + (size_t)j * L;
    Xyzz<F> run = xyzz_inf<F>(), acc = xyzz_inf<F>();
    if (w % windows == ones) {
        for (int b = (int)L - 1; b >= 0; b--) run = quad_add(run, ld_plain(bk + b), sub, mask);
    } else {
        for (int b = (int)L - 1; b >= 0; b--) {
            run = quad_add(run, ld_plain(bk + b), sub, mask);
            acc = quad_add(acc, run, sub, mask);
        }
    }
    if (sub != 0) return;
    st_vec(segW + t, acc);
    st_vec(segS + t, run);
}

template <class F>
__global__ void __launch_bounds__(128) k_seg_weight_quad(Xyzz<F>* W, const Xyzz<F>* __restrict__ S, uint32_t nseg,
                                                         uint32_t M, int lambda, uint32_t windows, uint32_t ones) {
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t t = gt >> 2;
    const int sub = (int)(gt & 3u);
    if (t >= nseg) return;
    const unsigned mask = 0xfu << (threadIdx.x & 28u);
    const uint32_t w = t / M, j = t % M;
    const Xyzz<F> s = ld_plain(S + t);
    if (w % windows == ones) {
        if (sub == 0) st_vec(W + t, s);
        return;
    }
    Xyzz<F> acc = ld_plain(W + t);
    if (j != 0) {
        Xyzz<F> m = xyzz_inf<F>();
        for (int b = 31 - __clz(j); b >= 0; b--) {
            m = quad_dbl(m, sub, mask);
            if ((j >> b) & 1u) m = quad_add(m, s, sub, mask);
        }
        for (int k = 0; k < lambda; k++) m = quad_dbl(m, sub, mask);
        acc = quad_add(acc, m, sub, mask);
    }
    // every lane has read W[t] before the shuffles above; with j = 0 the
    // value written is the one read
    if (sub == 0) st_vec(W + t, acc);
}

// Resident threads of a 128-thread-block kernel on the current device
// (cached per device ordinal in res_of, always with that device's value).
static inline double resident_threads(const void* kernel, double* res_of) {
    int dev = 0;
    cudaGetDevice(&dev);
    double res = dev >= 0 && dev < 64 ? res_of[dev] : 0.0;
    if (res <= 0.0) {
        int sms = 0, nb = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, 128, 0);
        res = (double)(sms > 0 ? sms : 1) * (nb > 0 ? nb : 1) * 128.0;
        if (dev >= 0 && dev < 64) res_of[dev] = res;
    }
    return res;
}
// Four lanes for a plan that runs alone, while 4 nseg threads fit in 1.25
// waves of the four-lane segment kernel.
template <class F>
bool reduce_on_quads(const MsmPlan& p, uint32_t nseg) {
    static double res_of[64] = {};
    return p.alone && 4.0 * nseg <= 1.25 * resident_threads((const void*)k_seg_reduce_quad<F>, res_of);
}

// out[g nb + b] = sum of in[g n + 256 b .. g n + 256 b + 255] (within n),
// nb = ceil(n / 256): block (b, g), 128 threads, a tree in shared memory
template <class F>
__global__ void __launch_bounds__(128) k_group_sum(const Xyzz<F>* __restrict__ in, uint32_t n, Xyzz<F>* out) {
    __shared__ Xyzz<F> sh[128];
    const uint32_t g = blockIdx.y, b = blockIdx.x, nb = gridDim.x;
    const uint32_t i0 = 256 * b + threadIdx.x, i1 = i0 + 128;
    Xyzz<F> v = i0 < n ? ld_plain(in + (size_t)g * n + i0) : xyzz_inf<F>();
    if (i1 < n) v = xyzz_add(v, ld_plain(in + (size_t)g * n + i1));
    sh[threadIdx.x] = v;
    __syncthreads();
    for (uint32_t h = 64; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] = xyzz_add(sh[threadIdx.x], sh[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) st_vec(out + (size_t)g * nb + b, sh[0]);
}

// The same sum on four lanes per value (a call that runs alone, see
// reduce_on_quads): out[g nb + b] = sum of in[g n + 64 b .. g n + 64 b + 63]
// (within n), nb = ceil(n / 64); block (b, g) is 32 groups of four lanes,
// each adding two inputs, then a five-level tree in shared memory.
template <class F>
__global__ void __launch_bounds__(128) k_group_sum_quad(const Xyzz<F>* __restrict__ in, uint32_t n, Xyzz<F>* out) {
    __shared__ Xyzz<F> sh[32];
    const uint32_t g = blockIdx.y, b = blockIdx.x, nb = gridDim.x;
    const uint32_t q = threadIdx.x >> 2;
    const int sub = (int)(threadIdx.x & 3u);
    const unsigned mask = 0xfu << (threadIdx.x & 28u);
    const uint32_t i0 = 64 * b + q, i1 = i0 + 32;
    Xyzz<F> v = i0 < n ? ld_plain(in + (size_t)g * n + i0) : xyzz_inf<F>();
    if (i1 < n) v = quad_add(v, ld_plain(in + (size_t)g * n + i1), sub, mask);
    if (sub == 0) sh[q] = v;
    __syncthreads();
    for (uint32_t h = 16; h > 0; h >>= 1) {
        if (q < h) v = quad_add(sh[q], sh[q + h], sub, mask);
        __syncthreads();  // every read of this level before its writes
        if (q < h && sub == 0) sh[q] = v;
        __syncthreads();
    }
    if (threadIdx.x == 0) st_vec(out + (size_t)g * nb + b, sh[0]);
}

// The group sum on four lanes runs about 2 nseg threads in its first pass,
// half as many as the segment kernels: a plan that runs alone takes it while
// those fit 1.25 waves, even when its segments stay on one lane.
template <class F>
bool group_sum_on_quads(const MsmPlan& p, uint32_t nseg) {
    static double res_of[64] = {};
    return p.alone && 2.0 * nseg <= 1.25 * resident_threads((const void*)k_group_sum_quad<F>, res_of);
}

// Horner over the K digit windows' totals, plus the ones-window total; four
// lanes per MSM of a batch (T holds K + 1 totals per MSM): the c (K - 1)
// sequential doublings are the longest chain of an MSM without window tables
template <class F>
__global__ void __launch_bounds__(128) k_msm_final(const Xyzz<F>* T, uint32_t K, int c, uint32_t batch,
                                                   Xyzz<F>* res, Affine<F>* out) {
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t q = gt >> 2;
    const int sub = (int)(gt & 3u);
    if (q >= batch) return;  // whole groups of four leave together
    const unsigned mask = 0xfu << (threadIdx.x & 28u);
    T += (size_t)q * (K + 1);
    Xyzz<F> acc = ld_plain(T + (K - 1));
    for (int w = (int)K - 2; w >= 0; w--) {
        for (int k = 0; k < c; k++) acc = quad_dbl(acc, sub, mask);
        acc = quad_add(acc, ld_plain(T + w), sub, mask);
    }
    acc = quad_add(acc, ld_plain(T + K), sub, mask);
    if (sub != 0) return;
    if (res) st_vec(res + q, acc);
    if (out) {
        Affine<F> a = aff_from_mont(xyzz_to_aff(acc));
        st_vec(out + q, a);
    }
}

template <class F>
__global__ void k_msm_empty(uint32_t batch, Xyzz<F>* res, Affine<F>* out) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= batch) return;
    if (res) res[q] = xyzz_inf<F>();
    if (out) {
        out[q].x = field_zero<F>();
        out[q].y = field_zero<F>();
    }
}

template <class F>
__global__ void k_bases_to_mont(const Affine<F>* in, size_t n, Affine<F>* out) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Affine<F> p = ld_vec(in + i);
    st_vec(out + i, aff_to_mont(p));
}

// tab[w n + i] = 2^(c w) P_i: c doublings per window, one inversion per
// stored point (setup time only)
template <class F>
__global__ void __launch_bounds__(128) k_window_table(const Affine<F>* pts, size_t n, int c, int K, Affine<F>* tab) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Affine<F> p = ld_plain(pts + i);
    st_vec(tab + i, p);
    Xyzz<F> x = xyzz_from_aff(p);
    for (int w = 1; w < K; w++) {
        for (int k = 0; k < c; k++) x = xyzz_dbl(x);
        st_vec(tab + (size_t)w * n + i, xyzz_to_aff(x));
    }
}

template <class F>
int msm_build_table(const MsmPlan& plan, const Affine<F>* pts, Affine<F>* tab, cudaStream_t st) {
    if (plan.n == 0) return ACE_OK;
    k_window_table<F><<<(unsigned)((plan.n + 127) / 128), 128, 0, st>>>(pts, plan.n, plan.c, plan.K, tab); ::ace::note_launch();
    ACE_TRY_CUDA(cudaGetLastError());
    return ACE_OK;
}

template <class F>
int msm_run(const MsmPlan& plan, const Affine<F>* d_bases, bool base_mont, const uint32_t* d_scalars,
            Arena& ar, Xyzz<F>* d_res, Affine<F>* d_out, cudaStream_t st, const MsmSorted* pre,
            MsmSorted* sorted, cudaEvent_t sorted_ev) {
    if (plan.n == 0) {
        k_msm_empty<F><<<(plan.batch + 31) / 32, 32, 0, st>>>(plan.batch, d_res, d_out); ::ace::note_launch();
        ACE_TRY_CUDA(cudaGetLastError());
        return ACE_OK;
    }
    MsmBufs<F, Arena> b;
    if (!b.carve(ar, plan, !base_mont)) {
        set_error("msm: scratch arena too small");
        return ACE_E_OOM;
    }
    const size_t n = plan.scalars();
    const uint32_t keys = plan.keys();
    const Affine<F>* bases = d_bases;
    if (plan.glv) {
        if constexpr (sizeof(F) == sizeof(fp_t)) {
            ACE_TRY(glv_prepare((const Affine<fp_t>*)d_bases, base_mont, d_scalars, plan.n / 2,
                                (Affine<fp_t>*)b.conv, b.gsc, st));
            bases = b.conv;
            d_scalars = b.gsc;
        } else {
            set_error("msm: the GLV plan is for G1 only");
            return ACE_E_ARG;
        }
    } else if (plan.gls) {
        if constexpr (sizeof(F) == sizeof(fp2_t)) {
            ACE_TRY(gls_prepare((const Affine<fp2_t>*)d_bases, base_mont, d_scalars, plan.n / 4,
                                (Affine<fp2_t>*)b.conv, b.gsc, st));
            bases = b.conv;
            d_scalars = b.gsc;
        } else {
            set_error("msm: the psi split is for G2 only");
            return ACE_E_ARG;
        }
    } else if (!base_mont) {
        k_bases_to_mont<F><<<(unsigned)((plan.n + 127) / 128), 128, 0, st>>>(d_bases, plan.n, b.conv); ::ace::note_launch();
        bases = b.conv;
    }
    const uint32_t *offsets = b.offsets, *entries = b.entries, *order = b.order;
    if (pre) {
        offsets = pre->offsets;
        entries = pre->entries;
        order = pre->order;
    } else {
        int prof_sort = prof_begin(PROF_SORT, st);
        ACE_TRY_CUDA(cudaMemsetAsync(b.offsets, 0, (keys + 1) * sizeof(uint32_t), st));
        launch_digits<false>(plan, d_scalars, b.offsets, nullptr, st);
        ACE_TRY(scan_exclusive_u32(b.offsets, keys + 1, b.scan_tmp, st));
        ACE_TRY_CUDA(cudaMemcpyAsync(b.cursor, b.offsets, keys * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        launch_digits<true>(plan, d_scalars, b.cursor, b.entries, st);
        ACE_TRY(bucket_order(b.offsets, keys, b.size_bins, b.scan_tmp, b.order, st));
        prof_end(prof_sort, st, nullptr, n);
    }
    if (sorted) {
        sorted->offsets = offsets;
        sorted->entries = entries;
        sorted->order = order;
    }
    if (sorted_ev) ACE_TRY_CUDA(cudaEventRecord(sorted_ev, st));
    int prof = prof_begin(sizeof(F) == sizeof(fp_t) ? PROF_G1_BUCKET : PROF_G2_BUCKET, st);
    const uint32_t split = bucket_split<F>(plan);
    k_bucket_acc<F><<<(unsigned)(((uint64_t)keys * split + 127) / 128), 128, 0, st>>>(bases, entries, offsets, order,
                                                                              keys, split, b.partial); ::ace::note_launch();
    prof_end(prof, st, offsets + keys, 0);
    if (split > 1) {
        k_bucket_combine<F><<<(keys + 127) / 128, 128, 0, st>>>(b.partial, keys, split, b.buckets); ::ace::note_launch();
    }
    uint32_t nseg = plan.all_windows() * plan.M;
    int prof_red = prof_begin(PROF_REDUCE, st);
    const bool quads = reduce_on_quads<F>(plan, nseg);
    if (quads) {
        const unsigned blocks = (unsigned)((4ull * nseg + 127) / 128);
        k_seg_reduce_quad<F><<<blocks, 128, 0, st>>>(b.buckets, nseg, plan.B, plan.L, plan.M, plan.windows(),
                                                     plan.bucket_windows(), b.segW, b.segS); ::ace::note_launch();
        k_seg_weight_quad<F><<<blocks, 128, 0, st>>>(b.segW, b.segS, nseg, plan.M, plan.lambda, plan.windows(),
                                                     plan.bucket_windows()); ::ace::note_launch();
    } else {
        k_seg_reduce<F><<<(nseg + 127) / 128, 128, 0, st>>>(b.buckets, nseg, plan.B, plan.L, plan.M, plan.windows(),
                                                            plan.bucket_windows(), b.segW, b.segS); ::ace::note_launch();
        k_seg_weight<F><<<(nseg + 127) / 128, 128, 0, st>>>(b.segW, b.segS, nseg, plan.M, plan.lambda,
                                                            plan.windows(), plan.bucket_windows()); ::ace::note_launch();
    }
    // sum each window's M weighted segments: 256 (four lanes: 64) to 1 per
    // pass, ping-pong between the two segment arrays
    const bool quad_sum = quads || group_sum_on_quads<F>(plan, nseg);
    Xyzz<F>*src = b.segW, *dst = b.segS;
    for (uint32_t n = plan.M; n > 1;) {
        const uint32_t per = quad_sum ? 64 : 256;
        uint32_t nb = (n + per - 1) / per;
        if (quad_sum) {
            k_group_sum_quad<F><<<dim3(nb, plan.all_windows()), 128, 0, st>>>(src, n, dst); ::ace::note_launch();
        } else {
            k_group_sum<F><<<dim3(nb, plan.all_windows()), 128, 0, st>>>(src, n, dst); ::ace::note_launch();
        }
        Xyzz<F>* t = src;
        src = dst;
        dst = t;
        n = nb;
    }
    k_msm_final<F><<<(unsigned)((4ull * plan.batch + 127) / 128), 128, 0, st>>>(src, plan.bucket_windows(), plan.c, plan.batch, d_res, d_out); ::ace::note_launch();
    prof_end(prof_red, st, nullptr, (uint64_t)plan.keys());
    ACE_TRY_CUDA(cudaGetLastError());
    return ACE_OK;
}

}  // namespace ace
