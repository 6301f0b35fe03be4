// msm_common.cu -- MSM plan, exclusive scan and the digit / histogram / scatter
// kernels shared by the G1 and G2 instantiations (see msm.cuh).
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

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
// Window size c: the throughput cost n K mixed additions plus the bucket
// reduction (2 full additions per bucket of 1.4 mixed-addition costs each, per
// bucket set, counted twice for the single bucket set of a tabled MSM), over
// the sizes whose top window is not a long pole.  The top window holds only
// 254 - c (K - 1) scalar bits (c = 18: 2, c = 19: 7), so its digits fall into
// few buckets, and one thread adds each bucket's entries in sequence; one
// sequential addition costs about MSM_SEQ_MADD additions of the whole GPU.
// Without window tables the top window has buckets of its own, and the time
// is the longer of the throughput work and that sequence.  With window tables
// the top window's digits share the low buckets with every other window,
// whose long buckets are split among threads; there c is skipped when a
// top-window bucket gets more than MSM_TOP_LOAD entries and that sequence
// would take more than half the throughput time.
static const double MSM_TOP_LOAD = 512.0;
static const double MSM_SEQ_MADD = 2.0e4;
// bits: 255 for full Fr scalars (254 bits and the top digit's carry), 128
// for GLV halves (below 2^127), 67 for the G2 split's parts (below 2^66).
static double msm_cost(size_t n, int c, bool tabled, int bits = 255) {
    const int K = (bits + c - 1) / c;
    const double B = (double)(1u << (c - 1));
    const double work = (double)n * K + (tabled ? 5.6 * B : 2.8 * K * B);
    int top_bits = (bits - 1) - c * (K - 1);
    if (top_bits < 1) top_bits = 1;
    if (top_bits > c - 1) top_bits = c - 1;
    const double top_load = (double)n / (double)(1u << top_bits);
    if (!tabled) return work > top_load * MSM_SEQ_MADD ? work : top_load * MSM_SEQ_MADD;
    if (top_load > MSM_TOP_LOAD && top_load * MSM_SEQ_MADD > 0.5 * work) return 1e300;
    return work;
}

// largest window size whose single-MSM plans reduce in segments of 4 buckets
#ifndef ACE_SHORT_SEGMENT_MAX_C
#define ACE_SHORT_SEGMENT_MAX_C 14
#endif
static MsmPlan plan_for(size_t n, int c, bool tabled, bool glv = false, bool gls = false) {
    MsmPlan p;
    p.n = n;
    if (c < 6) c = 6;
    if (c > 20) c = 20;
    p.c = c;
    p.glv = glv;
    p.gls = gls;
    p.K = (p.bits() + p.c - 1) / p.c;
    p.B = 1u << (p.c - 1);
    // segments of 16 buckets; of 4 when a window holds at most 2^13 buckets:
    // there a segment's sequential running sum (2 additions per bucket, one
    // thread) is the longest chain of the reduction, and four times as many
    // threads still leave the GPU mostly idle
    p.lambda = p.c - 1 < 4 ? p.c - 1 : 4;
    if (p.c <= ACE_SHORT_SEGMENT_MAX_C) p.lambda = 2;
    p.L = 1u << p.lambda;
    p.M = p.B / p.L;
    p.tabled = tabled;
    p.B1 = 1;
    while (p.B1 < p.B && (size_t)p.B1 * 64 < n) p.B1 *= 2;
    return p;
}

void msm_plan_set_batch(MsmPlan& p, uint32_t batch) {
    p.batch = batch;
    // many MSMs at once give the reduction threads enough: back to segments
    // of 16 buckets (fewer segments to weight)
    if (batch > 1) {
        p.lambda = p.c - 1 < 4 ? p.c - 1 : 4;
        p.L = 1u << p.lambda;
        p.M = p.B / p.L;
    }
}

static int best_window(size_t n, bool tabled, int bits = 255) {
    int best_c = 20;  // top window of 14 bits: the fallback for any n
    double best = 1e300;
    for (int c = tabled ? 8 : 6; c <= 20; c++) {
        double cost = msm_cost(n, c, tabled, bits);
        if (cost < best) {
            best = cost;
            best_c = c;
        }
    }
    return best_c;
}

MsmPlan msm_plan_tabled(size_t n, int force_c) { return plan_for(n, force_c > 0 ? force_c : best_window(n, true), true); }

MsmPlan msm_plan(size_t n, int force_c) { return plan_for(n, force_c > 0 ? force_c : best_window(n, false), false); }

MsmPlan msm_plan_glv(size_t n, int force_c) {
    return plan_for(2 * n, force_c > 0 ? force_c : best_window(2 * n, false, 128), false, true);
}

// Window of the G2 split, measured: the parts lie below 2^65 in practice
// (2^66 is the proven bound the 67-bit digit windows cover), so the window
// holding bit 64 decides the balance.  c = 11 leaves it 10 value bits and no
// carry into the (empty) window above; c = 13 fills it and carries into the
// next one for half the points, c = 12, 15, 16 leave it 1-5 bits: buckets of
// thousands of entries.  Measured per G2 MSM over 2^12 / 2^14 / 2^16 points:
// c = 11 1.5 / 1.7 / 2.6 ms, c = 17 (what the G1 cost model picks) 3.2 /
// 3.0 / 3.9 ms, the full-width MSM 3.9 / 3.8 / 4.0 ms.
static const int MSM_GLS_C = 11;
MsmPlan msm_plan_gls(size_t n, int force_c) {
    return plan_for(4 * n, force_c > 0 ? force_c : MSM_GLS_C, false, false, true);
}

// ---------------------------------------------------------------------------
// scan
// ---------------------------------------------------------------------------
size_t scan_tmp_words(size_t n) { return (n + 1023) / 1024 + 1; }

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) >= (unsigned)o) v += t;
    }
    return v;
}

// block of 256 threads scans a tile of 1024 values (4 per thread), exclusive
__global__ void k_scan_tiles(uint32_t* d, size_t n, uint32_t* sums) {
    __shared__ uint32_t wsum[8];
    size_t base = (size_t)blockIdx.x * 1024 + threadIdx.x * 4;
    uint32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; k++) v[k] = (base + k < n) ? d[base + k] : 0u;
    uint32_t tsum = v[0] + v[1] + v[2] + v[3];
    uint32_t incl = warp_incl_scan(tsum);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < 8 ? wsum[lane] : 0u;
        uint32_t wi = warp_incl_scan(w);
        if (lane < 8) wsum[lane] = wi - w;  // exclusive warp offsets
    }
    __syncthreads();
    uint32_t run = wsum[warp] + incl - tsum;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (base + k < n) d[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 255) sums[blockIdx.x] = run;
}

// one block scans the tile sums (any count), exclusive, in place
__global__ void k_scan_sums(uint32_t* sums, uint32_t nb) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t start = 0; start < nb; start += 1024) {
        uint32_t i = start + threadIdx.x;
        uint32_t v = i < nb ? sums[i] : 0u;
        uint32_t incl = warp_incl_scan(v);
        int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = wsum[lane];
            uint32_t wi = warp_incl_scan(w);
            wsum[lane] = wi - w;
        }
        __syncthreads();
        uint32_t ex = carry + wsum[warp] + incl - v;
        if (i < nb) sums[i] = ex;
        __syncthreads();
        if (threadIdx.x == 1023) carry = ex + v;
        __syncthreads();
    }
}

__global__ void k_scan_add(uint32_t* d, size_t n, const uint32_t* sums) {
    size_t base = (size_t)blockIdx.x * 1024 + threadIdx.x * 4;
    uint32_t add = sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < 4; k++)
        if (base + k < n) d[base + k] += add;
}

int scan_exclusive_u32(uint32_t* d, size_t n, uint32_t* tmp, cudaStream_t st) {
    if (n == 0) return ACE_OK;
    uint32_t nb = (uint32_t)((n + 1023) / 1024);
    k_scan_tiles<<<nb, 256, 0, st>>>(d, n, tmp); ::ace::note_launch();
    k_scan_sums<<<1, 1024, 0, st>>>(tmp, nb); ::ace::note_launch();
    k_scan_add<<<nb, 256, 0, st>>>(d, n, tmp); ::ace::note_launch();
    ACE_TRY_CUDA(cudaGetLastError());
    return ACE_OK;
}

// ---------------------------------------------------------------------------
// digits, histogram and scatter
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ld_scalar(const uint32_t* sc, size_t i, uint32_t s[8]) {
    const uint4* p = reinterpret_cast<const uint4*>(sc + 8 * i);
    uint4 a = __ldg(p), b = __ldg(p + 1);
    s[0] = a.x; s[1] = a.y; s[2] = a.z; s[3] = a.w;
    s[4] = b.x; s[5] = b.y; s[6] = b.z; s[7] = b.w;
}

template <int C>
__device__ __forceinline__ uint32_t window_bits(const uint32_t s[8], int w) {
    const int bit = w * C;
    const int limb = bit >> 5, sh = bit & 31;
    uint32_t lo = s[limb] >> sh;
    uint32_t hi = (sh != 0 && limb + 1 < 8) ? (s[limb + 1] << (32 - sh)) : 0u;
    return (lo | hi) & ((1u << C) - 1u);
}

// kind: 0 zero, 1 one, 2 general
__device__ __forceinline__ int scalar_kind(const uint32_t s[8]) {
    uint32_t hi = s[1] | s[2] | s[3] | s[4] | s[5] | s[6] | s[7];
    if (hi == 0 && s[0] == 0) return 0;
    if (hi == 0 && s[0] == 1) return 1;
    return 2;
}

// SCATTER = false: histogram into cnt; true: place entries using cnt as cursor.
// TAB: digits of all windows go to bucket window 0 with entry w n + i
// (precomputed window tables); otherwise window w's buckets hold entry i.
// A batch of MSMs over the same n points: scalar t belongs to MSM t / n and
// multiplies point t mod n; each MSM has its own keys_per keys.
// BITS: 255 for Fr scalars, 128 for GLV halves (magnitudes below 2^127), 67
// for the parts of the G2 split (below 2^66).
template <int C, bool SCATTER, bool TAB, int BITS = 255>
__global__ void k_msm_digits(const uint32_t* __restrict__ sc, size_t total, size_t n, uint32_t keys_per,
                             uint32_t ones_mask, uint32_t* cnt, uint32_t* entries) {
    constexpr int K = (BITS + C - 1) / C;
    constexpr uint32_t B = 1u << (C - 1);
    constexpr uint32_t BW = TAB ? 1u : (uint32_t)K;
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    uint32_t s[8];
    ld_scalar(sc, t, s);
    int kind = scalar_kind(s);
    if (kind == 0) return;
    const size_t q = total == n ? 0 : t / n;  // which MSM of the batch
    const size_t i = t - q * n;               // which point
    cnt += q * keys_per;
    if (kind == 1) {
        uint32_t key = BW * B + ((uint32_t)i & ones_mask);
        if (SCATTER) {
            uint32_t pos = atomicAdd(&cnt[key], 1u);
            entries[pos] = (uint32_t)i;
        } else {
            atomicAdd(&cnt[key], 1u);
        }
        return;
    }
    uint32_t carry = 0;
#pragma unroll
    for (int w = 0; w < K; w++) {
        uint32_t raw = window_bits<C>(s, w) + carry;
        uint32_t mag, neg;
        if (raw > B) {
            mag = (1u << C) - raw;  // digit raw - 2^C < 0
            neg = 1u;
            carry = 1u;
        } else {
            mag = raw;
            neg = 0u;
            carry = 0u;
        }
        if (mag != 0) {
            uint32_t key = (TAB ? 0u : (uint32_t)w * B) + (mag - 1u);
            if (SCATTER) {
                uint32_t pos = atomicAdd(&cnt[key], 1u);
                uint32_t e = TAB ? (uint32_t)((size_t)w * n + i) : (uint32_t)i;
                entries[pos] = e | (neg << 31);
            } else {
                atomicAdd(&cnt[key], 1u);
            }
        }
    }
}

template <bool SCATTER>
void launch_digits(const MsmPlan& plan, const uint32_t* sc, uint32_t* cnt, uint32_t* entries, cudaStream_t st) {
    const size_t total = plan.scalars(), n = plan.n;
    const uint32_t kp = plan.keys_per(), om = plan.ones_mask();
    unsigned grid = (unsigned)((total + 255) / 256);
    if (plan.gls) {
        switch (plan.c) {
#define ACE_DIGITS_GLS(CC) \
    case CC: k_msm_digits<CC, SCATTER, false, 67><<<grid, 256, 0, st>>>(sc, total, n, kp, om, cnt, entries); break;
            ACE_DIGITS_GLS(6) ACE_DIGITS_GLS(7) ACE_DIGITS_GLS(8) ACE_DIGITS_GLS(9) ACE_DIGITS_GLS(10)
            ACE_DIGITS_GLS(11) ACE_DIGITS_GLS(12) ACE_DIGITS_GLS(13) ACE_DIGITS_GLS(14) ACE_DIGITS_GLS(15)
            ACE_DIGITS_GLS(16) ACE_DIGITS_GLS(17) ACE_DIGITS_GLS(18) ACE_DIGITS_GLS(19) ACE_DIGITS_GLS(20)
#undef ACE_DIGITS_GLS
            default: break;
        }
        ::ace::note_launch();
        return;
    }
    if (plan.glv) {
        switch (plan.c) {
#define ACE_DIGITS_GLV(CC) \
    case CC: k_msm_digits<CC, SCATTER, false, 128><<<grid, 256, 0, st>>>(sc, total, n, kp, om, cnt, entries); break;
            ACE_DIGITS_GLV(6) ACE_DIGITS_GLV(7) ACE_DIGITS_GLV(8) ACE_DIGITS_GLV(9) ACE_DIGITS_GLV(10)
            ACE_DIGITS_GLV(11) ACE_DIGITS_GLV(12) ACE_DIGITS_GLV(13) ACE_DIGITS_GLV(14) ACE_DIGITS_GLV(15)
            ACE_DIGITS_GLV(16) ACE_DIGITS_GLV(17) ACE_DIGITS_GLV(18) ACE_DIGITS_GLV(19) ACE_DIGITS_GLV(20)
#undef ACE_DIGITS_GLV
            default: break;
        }
        ::ace::note_launch();
        return;
    }
    switch (plan.c * 2 + (plan.tabled ? 1 : 0)) {
#define ACE_DIGITS_CASE(CC)                                                                                        \
    case 2 * CC: k_msm_digits<CC, SCATTER, false><<<grid, 256, 0, st>>>(sc, total, n, kp, om, cnt, entries); break; \
    case 2 * CC + 1: k_msm_digits<CC, SCATTER, true><<<grid, 256, 0, st>>>(sc, total, n, kp, om, cnt, entries); break;
        ACE_DIGITS_CASE(6) ACE_DIGITS_CASE(7) ACE_DIGITS_CASE(8) ACE_DIGITS_CASE(9) ACE_DIGITS_CASE(10)
        ACE_DIGITS_CASE(11) ACE_DIGITS_CASE(12) ACE_DIGITS_CASE(13) ACE_DIGITS_CASE(14) ACE_DIGITS_CASE(15)
        ACE_DIGITS_CASE(16) ACE_DIGITS_CASE(17) ACE_DIGITS_CASE(18) ACE_DIGITS_CASE(19) ACE_DIGITS_CASE(20)
#undef ACE_DIGITS_CASE
        default: break;
    }
    ::ace::note_launch();
}

template void launch_digits<false>(const MsmPlan&, const uint32_t*, uint32_t*, uint32_t*, cudaStream_t);
template void launch_digits<true>(const MsmPlan&, const uint32_t*, uint32_t*, uint32_t*, cudaStream_t);

// ---------------------------------------------------------------------------
// bucket order: counting sort of keys by decreasing size
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t size_bin(const uint32_t* off, uint32_t key) {
    uint32_t s = off[key + 1] - off[key];
    if (s > SIZE_BINS - 1) s = SIZE_BINS - 1;
    return SIZE_BINS - 1 - s;  // bin 0 holds the largest buckets
}

// Bucket sizes cluster around the mean, so a few bins take most keys: both
// passes count in shared memory first and touch each global bin once per
// block (blocks of 256 threads).
__global__ void __launch_bounds__(256) k_size_hist(const uint32_t* __restrict__ off, uint32_t keys, uint32_t* bins) {
    __shared__ uint32_t cnt[SIZE_BINS];
    for (uint32_t j = threadIdx.x; j < SIZE_BINS; j += blockDim.x) cnt[j] = 0;
    __syncthreads();
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < keys) atomicAdd(&cnt[size_bin(off, k)], 1u);
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < SIZE_BINS; j += blockDim.x)
        if (cnt[j]) atomicAdd(&bins[j], cnt[j]);
}

// bins holds each bin's first position (exclusive scan of the histogram)
__global__ void __launch_bounds__(256) k_size_scatter(const uint32_t* __restrict__ off, uint32_t keys, uint32_t* bins,
                                                      uint32_t* order) {
    __shared__ uint32_t cnt[SIZE_BINS], base[SIZE_BINS];
    for (uint32_t j = threadIdx.x; j < SIZE_BINS; j += blockDim.x) cnt[j] = 0;
    __syncthreads();
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t bin = 0, rank = 0;
    if (k < keys) {
        bin = size_bin(off, k);
        rank = atomicAdd(&cnt[bin], 1u);
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < SIZE_BINS; j += blockDim.x)
        if (cnt[j]) base[j] = atomicAdd(&bins[j], cnt[j]);
    __syncthreads();
    if (k < keys) order[base[bin] + rank] = k;
}

int bucket_order(const uint32_t* offsets, uint32_t keys, uint32_t* bins, uint32_t* scan_tmp, uint32_t* order,
                 cudaStream_t st) {
    ACE_TRY_CUDA(cudaMemsetAsync(bins, 0, (SIZE_BINS + 1) * sizeof(uint32_t), st));
    unsigned grid = (keys + 255) / 256;
    k_size_hist<<<grid, 256, 0, st>>>(offsets, keys, bins); ::ace::note_launch();
    ACE_TRY(scan_exclusive_u32(bins, SIZE_BINS + 1, scan_tmp, st));
    k_size_scatter<<<grid, 256, 0, st>>>(offsets, keys, bins, order); ::ace::note_launch();
    ACE_TRY_CUDA(cudaGetLastError());
    return ACE_OK;
}

}  // namespace ace
