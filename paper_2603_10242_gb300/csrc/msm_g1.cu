// msm_g1.cu -- G1 instantiation of the Pippenger MSM.
#define ACE_FIELD_MUL_CALL 1
#include "msm_impl.cuh"

namespace ace {
template int msm_run<fp_t>(const MsmPlan&, const Affine<fp_t>*, bool, const uint32_t*, Arena&, Xyzz<fp_t>*,
                           Affine<fp_t>*, cudaStream_t, const MsmSorted*, MsmSorted*, cudaEvent_t);
template size_t msm_scratch_bytes<fp_t>(const MsmPlan&, bool);
template int msm_build_table<fp_t>(const MsmPlan&, const Affine<fp_t>*, Affine<fp_t>*, cudaStream_t);
}  // namespace ace
