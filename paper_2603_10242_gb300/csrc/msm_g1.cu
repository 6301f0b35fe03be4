// msm_g1.cu -- G1 instantiation of the Pippenger MSM, and the GLV inputs of
// G1 MSMs without window tables.
#define ACE_FIELD_MUL_CALL 1
#include "glv.cuh"
#include "msm_impl.cuh"

namespace ace {
template int msm_run<fp_t>(const MsmPlan&, const Affine<fp_t>*, bool, const uint32_t*, Arena&, Xyzz<fp_t>*,
                           Affine<fp_t>*, cudaStream_t, const MsmSorted*, MsmSorted*, cudaEvent_t);
template size_t msm_scratch_bytes<fp_t>(const MsmPlan&, bool);
template int msm_build_table<fp_t>(const MsmPlan&, const Affine<fp_t>*, Affine<fp_t>*, cudaStream_t);

// One thread per input point: k mod r (at most five subtractions of r from a
// 256-bit value), its GLV halves, and the points +-P and +-phi(P) =
// (beta x, +-y) that carry the halves' signs.
__global__ void __launch_bounds__(128) k_glv_prepare(const g1_aff* __restrict__ in, bool in_mont,
                                                     const uint32_t* __restrict__ sc, size_t n, fp_t beta,
                                                     g1_aff* out, uint32_t* osc) {
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
    uint32_t k1[4], k2[4], n1 = 0, n2 = 0;
    glv_split_limbs(k.v, k1, &n1, k2, &n2);  // halves below 2^127 for k < r
    g1_aff p = ld_vec(in + i);
    if (!in_mont) p = aff_to_mont(p);
    g1_aff a = p, b = p;
    b.x = p.x * beta;
    if (n1) a.y = fe_neg(a.y);
    if (n2) b.y = fe_neg(b.y);
    st_vec(out + i, a);
    st_vec(out + n + i, b);
    uint4* o1 = reinterpret_cast<uint4*>(osc + 8 * i);
    uint4* o2 = reinterpret_cast<uint4*>(osc + 8 * (n + i));
    o1[0] = make_uint4(k1[0], k1[1], k1[2], k1[3]);
    o1[1] = make_uint4(0u, 0u, 0u, 0u);
    o2[0] = make_uint4(k2[0], k2[1], k2[2], k2[3]);
    o2[1] = make_uint4(0u, 0u, 0u, 0u);
}

int glv_prepare(const Affine<fp_t>* in, bool in_mont, const uint32_t* sc, size_t n, Affine<fp_t>* out,
                uint32_t* osc, cudaStream_t st) {
    fp_t beta = {ACE_GLV_BETA};
    beta = fe_to_mont(beta);
    k_glv_prepare<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(in, in_mont, sc, n, beta, out, osc);
    ::ace::note_launch();
    ACE_TRY_CUDA(cudaGetLastError());
    return ACE_OK;
}
}  // namespace ace
