// msm_g2.cu -- G2 instantiation of the Pippenger MSM, and the inputs of G2
// MSMs without window tables split by the endomorphism psi (glv.cuh).
#define ACE_FIELD_MUL_CALL 1
#include "glv.cuh"
#include "msm_impl.cuh"

namespace ace {
template int msm_run<fp2_t>(const MsmPlan&, const Affine<fp2_t>*, bool, const uint32_t*, Arena&, Xyzz<fp2_t>*,
                           Affine<fp2_t>*, cudaStream_t, const MsmSorted*, MsmSorted*, cudaEvent_t);
template size_t msm_scratch_bytes<fp2_t>(const MsmPlan&, bool);
template int msm_build_table<fp2_t>(const MsmPlan&, const Affine<fp2_t>*, Affine<fp2_t>*, cudaStream_t);

// psi on a Montgomery affine point: (conj(x) gx, conj(y) gy); the point at
// infinity (zeros) stays zeros
__device__ __forceinline__ g2_aff gls_psi(const g2_aff& p, const fp2_t& gx, const fp2_t& gy) {
    g2_aff q;
    q.x = fp2_t{p.x.c0, fe_neg(p.x.c1)} * gx;
    q.y = fp2_t{p.y.c0, fe_neg(p.y.c1)} * gy;
    return q;
}

// One thread per input point: k mod r (at most five subtractions of r from a
// 256-bit value), its four parts k = k0 + k1 lambda + k2 lambda^2 + k3
// lambda^3, and the points +-psi^t(Q) (t = 0..3) that carry the parts' signs:
// out[t n + i], with the magnitudes at osc[8 (t n + i)] (8 limbs, top 5 zero).
__global__ void __launch_bounds__(128) k_gls_prepare(const g2_aff* __restrict__ in, bool in_mont,
                                                     const uint32_t* __restrict__ sc, size_t n, fp2_t gx,
                                                     fp2_t gy, g2_aff* out, uint32_t* osc) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    fr_t k;
    const uint4* sp = reinterpret_cast<const uint4*>(sc + 8 * i);
    const uint4 s0 = __ldg(sp), s1 = __ldg(sp + 1);
    k.v[0] = s0.x; k.v[1] = s0.y; k.v[2] = s0.z; k.v[3] = s0.w;
    k.v[4] = s1.x; k.v[5] = s1.y; k.v[6] = s1.z; k.v[7] = s1.w;
    while (fe_geq_mod(k)) {
        uint32_t br = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const uint64_t d = (uint64_t)k.v[j] - mod_limb<FrCfg>(j) - br;
            k.v[j] = (uint32_t)d;
            br = (uint32_t)(d >> 63);
        }
    }
    uint32_t mag[4][3], neg[4];
    gls_split_limbs(k.v, mag, neg);  // parts below 2^66 for k < r
    g2_aff p = ld_vec(in + i);
    if (!in_mont) p = aff_to_mont(p);
#pragma unroll 1
    for (int t = 0; t < 4; t++) {
        if (t) p = gls_psi(p, gx, gy);
        g2_aff q = p;
        if (neg[t]) q.y = fe_neg(q.y);
        st_vec(out + (size_t)t * n + i, q);
        uint4* o = reinterpret_cast<uint4*>(osc + 8 * ((size_t)t * n + i));
        o[0] = make_uint4(mag[t][0], mag[t][1], mag[t][2], 0u);
        o[1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

int gls_prepare(const Affine<fp2_t>* in, bool in_mont, const uint32_t* sc, size_t n, Affine<fp2_t>* out,
                uint32_t* osc, cudaStream_t st) {
    const fp_t gx0 = {ACE_GLS_GX0}, gx1 = {ACE_GLS_GX1}, gy0 = {ACE_GLS_GY0}, gy1 = {ACE_GLS_GY1};
    const fp2_t gx{fe_to_mont(gx0), fe_to_mont(gx1)}, gy{fe_to_mont(gy0), fe_to_mont(gy1)};
    k_gls_prepare<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(in, in_mont, sc, n, gx, gy, out, osc);
    ::ace::note_launch();
    ACE_TRY_CUDA(cudaGetLastError());
    return ACE_OK;
}
}  // namespace ace
