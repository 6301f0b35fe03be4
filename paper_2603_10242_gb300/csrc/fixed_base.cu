// fixed_base.cu -- batch k_i * G for the G1 / G2 generators: the scalar
// multiplications of the toy trusted setup (Section 9, "Trusted setup": the
// circuit-specific setup of Groth16) and of synthetic MSM inputs.
//
// Table T[w][d-1] = d 2^(8w) G (w < 32, d = 1..255, affine Montgomery), built
// once per context; then k G = sum_w T[w][byte_w(k)]: at most 32 mixed
// additions, followed by one inversion for the affine result.
#include "fixed_base.cuh"

namespace ace {

// EIP-197 generator of G2, canonical decimal:
//  x = 10857046999023057135944570762232829481370756359578518086990519993285655852781
//    + 11559732032986387107991004021392285783925812861821192530917403151452391805634 u
//  y = 8495653923123431417604973247489272438418190587263600148770280649306958101930
//    + 4082367875863433681332203403145435568316851327593401208105741076214120093531 u
// as little-endian 32-bit limbs:
static const uint32_t G2X0[8] = {0xd992f6edu, 0x46debd5cu, 0xf75edaddu, 0x674322d4u, 0x5e5c4479u, 0x426a0066u, 0x121f1e76u, 0x1800deefu};
static const uint32_t G2X1[8] = {0xaef312c2u, 0x97e485b7u, 0x35a9e712u, 0xf1aa4933u, 0x31fb5d25u, 0x7260bfb7u, 0x920d483au, 0x198e9393u};
static const uint32_t G2Y0[8] = {0x66fa7daau, 0x4ce6cc01u, 0x0c43d37bu, 0xe3d1e769u, 0x8dcb408fu, 0x4aab7180u, 0xdb8c6debu, 0x12c85ea5u};
static const uint32_t G2Y1[8] = {0xd122975bu, 0x55acdadcu, 0x70b38ef3u, 0xbc4b3133u, 0x690c3395u, 0xec9e99adu, 0x585ff075u, 0x090689d0u};

template <class F>
struct GenConst;
template <>
struct GenConst<fp_t> {
    static Affine<fp_t> get() {
        Affine<fp_t> g;
        g.x = fe_zero<FpCfg>();
        g.y = fe_zero<FpCfg>();
        g.x.v[0] = 1;
        g.y.v[0] = 2;
        return aff_to_mont(g);
    }
};
template <>
struct GenConst<fp2_t> {
    static Affine<fp2_t> get() {
        Affine<fp2_t> g;
        for (int i = 0; i < 8; i++) {
            g.x.c0.v[i] = G2X0[i];
            g.x.c1.v[i] = G2X1[i];
            g.y.c0.v[i] = G2Y0[i];
            g.y.c1.v[i] = G2Y1[i];
        }
        return aff_to_mont(g);
    }
};

template <class F>
Affine<F> generator_mont() {
    return GenConst<F>::get();
}
template Affine<fp_t> generator_mont<fp_t>();
template Affine<fp2_t> generator_mont<fp2_t>();

// Q_w = 2^(8w) G, sequential doublings in one thread
template <class F>
__global__ void k_fb_powers(Affine<F> g, Xyzz<F>* q) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Xyzz<F> acc = xyzz_from_aff(g);
    for (int w = 0; w < 32; w++) {
        q[w] = acc;
        for (int k = 0; k < 8; k++) acc = xyzz_dbl(acc);
    }
}

// T[w][d-1] = d Q_w
template <class F>
__global__ void k_fb_table(const Xyzz<F>* q, Affine<F>* tab) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 32 * 255) return;
    int w = t / 255, d = t % 255 + 1;
    Affine<F> qw = xyzz_to_aff(q[w]);
    Xyzz<F> acc = xyzz_inf<F>();
    for (int b = 7; b >= 0; b--) {
        acc = xyzz_dbl(acc);
        if ((d >> b) & 1) acc = xyzz_add_aff(acc, qw);
    }
    tab[t] = xyzz_to_aff(acc);
}

template <class F>
__global__ void __launch_bounds__(128) k_fb_mul(const Affine<F>* __restrict__ tab, const uint32_t* __restrict__ sc,
                                                size_t n, Affine<F>* out, int out_mont) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Xyzz<F> acc = xyzz_inf<F>();
#pragma unroll 1
    for (int limb = 0; limb < 8; limb++) {
        uint32_t cur = sc[8 * i + limb];
#pragma unroll 1
        for (int b = 0; b < 4; b++) {
            uint32_t d = (cur >> (8 * b)) & 255u;
            if (d) acc = xyzz_add_aff(acc, tab[(limb * 4 + b) * 255 + d - 1]);
        }
    }
    Affine<F> a = xyzz_to_aff(acc);
    out[i] = out_mont ? a : aff_from_mont(a);
}

template <class F>
int fixed_base_table(ace_ctx* ctx, Affine<F>** tab_out) {
    void*& slot = sizeof(F) == sizeof(fp_t) ? ctx->g1_fixed_tab : ctx->g2_fixed_tab;
    if (slot) {
        *tab_out = (Affine<F>*)slot;
        return ACE_OK;
    }
    void* q = nullptr;
    void* tab = nullptr;
    ACE_TRY(dev_alloc(ctx, &q, 32 * sizeof(Xyzz<F>)));
    int rc = dev_alloc(ctx, &tab, 32 * 255 * sizeof(Affine<F>));
    if (rc != ACE_OK) {
        dev_free(ctx, q, 32 * sizeof(Xyzz<F>));
        return rc;
    }
    k_fb_powers<F><<<1, 1, 0, ctx->stream>>>(generator_mont<F>(), (Xyzz<F>*)q); ::ace::note_launch();
    k_fb_table<F><<<(32 * 255 + 127) / 128, 128, 0, ctx->stream>>>((Xyzz<F>*)q, (Affine<F>*)tab); ::ace::note_launch();
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, q, 32 * sizeof(Xyzz<F>));
    if (e != cudaSuccess) {
        set_error("fixed-base table: %s", cudaGetErrorString(e));
        dev_free(ctx, tab, 32 * 255 * sizeof(Affine<F>));
        return ACE_E_CUDA;
    }
    slot = tab;
    *tab_out = (Affine<F>*)tab;
    return ACE_OK;
}

template <class F>
int fixed_base_mul(ace_ctx* ctx, const uint32_t* d_scalars, size_t n, Affine<F>* d_out, bool out_mont,
                   cudaStream_t st) {
    if (n == 0) return ACE_OK;
    Affine<F>* tab = nullptr;
    ACE_TRY(fixed_base_table<F>(ctx, &tab));
    k_fb_mul<F><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(tab, d_scalars, n, d_out, out_mont ? 1 : 0); ::ace::note_launch();
    ACE_TRY_CUDA(cudaGetLastError());
    return ACE_OK;
}

template <class F>
int fixed_table_build(ace_ctx* ctx, const Affine<F>& base_mont, Affine<F>* d_tab, cudaStream_t st) {
    void* q = nullptr;
    ACE_TRY(dev_alloc(ctx, &q, 32 * sizeof(Xyzz<F>)));
    k_fb_powers<F><<<1, 1, 0, st>>>(base_mont, (Xyzz<F>*)q); ::ace::note_launch();
    k_fb_table<F><<<(32 * 255 + 127) / 128, 128, 0, st>>>((Xyzz<F>*)q, d_tab); ::ace::note_launch();
    cudaError_t e = cudaStreamSynchronize(st);
    dev_free(ctx, q, 32 * sizeof(Xyzz<F>));
    if (e != cudaSuccess) {
        set_error("fixed-base table: %s", cudaGetErrorString(e));
        return ACE_E_CUDA;
    }
    return ACE_OK;
}
template int fixed_table_build<fp_t>(ace_ctx*, const Affine<fp_t>&, Affine<fp_t>*, cudaStream_t);
template int fixed_table_build<fp2_t>(ace_ctx*, const Affine<fp2_t>&, Affine<fp2_t>*, cudaStream_t);

template int fixed_base_mul<fp_t>(ace_ctx*, const uint32_t*, size_t, Affine<fp_t>*, bool, cudaStream_t);
template int fixed_base_mul<fp2_t>(ace_ctx*, const uint32_t*, size_t, Affine<fp2_t>*, bool, cudaStream_t);

}  // namespace ace
