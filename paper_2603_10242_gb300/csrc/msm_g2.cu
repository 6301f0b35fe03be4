// msm_g2.cu -- G2 instantiation of the Pippenger MSM.
#define ACE_FIELD_MUL_CALL 1
#include "msm_impl.cuh"

namespace ace {
template int msm_run<fp2_t>(const MsmPlan&, const Affine<fp2_t>*, bool, const uint32_t*, Arena&, Xyzz<fp2_t>*,
                           Affine<fp2_t>*, cudaStream_t, const MsmSorted*, MsmSorted*, cudaEvent_t);
template size_t msm_scratch_bytes<fp2_t>(const MsmPlan&, bool);
template int msm_build_table<fp2_t>(const MsmPlan&, const Affine<fp2_t>*, Affine<fp2_t>*, cudaStream_t);
}  // namespace ace
