// msm_noalloc.cu -- a G1 multi-scalar multiplication that allocates nothing.
//
// Some callers cannot call cudaMalloc: their device memory belongs to a pool
// or arena owned by someone else and handed out up front, or they run on a
// latency-sensitive path that shares the GPU with other streams and must not
// trigger the device-wide synchronisation that cudaMalloc / cudaFree imply.
// ace_msm_g1_noalloc serves them: it computes the same result as ace_msm_g1
// for up to ACE_MSM_NOALLOC_MAX_N points, with its scratch held in one fixed
// array in this file (kept on every GPU that loads the library until the
// process exits) instead of memory the library allocates.
//
// The array is shared by every call: it keeps the last call's contents, the
// pipeline clears what has to start at zero before each use, and calls whose
// work overlaps on the GPU (other streams, other host threads) race on it.
#include <mutex>

#include "msm.cuh"

namespace ace {
namespace {

// maximum number of points and the fixed window size of this variant
const size_t NOALLOC_MAX_N = 16384;
const int NOALLOC_C = 10;
const size_t NOALLOC_BYTES = 6u << 20;  // 6 MiB

// Host code must not use this name as a device address: the address is
// obtained with cudaGetSymbolAddress below, once per device.
static __device__ __align__(256) unsigned char g_msm_scratch[NOALLOC_BYTES];

std::mutex g_mu;
void* g_addr[64] = {};

// device address of g_msm_scratch on the current device (set up on the first
// call made on that device)
int scratch_address(void** out) {
    int dev = 0;
    ACE_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("ace_msm_g1_noalloc: device index %d out of range", dev);
        return ACE_E_ARG;
    }
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_msm_scratch);
        if (e != cudaSuccess || !p) {
            set_error("ace_msm_g1_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return ACE_E_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return ACE_OK;
}

}  // namespace
}  // namespace ace

using namespace ace;

extern "C" {

int ace_msm_g1_noalloc(const ace_g1_affine* d_bases, int base_form, const ace_fr* d_scalars, size_t n,
                       ace_g1_affine* d_out, ace_stream stream) {
    clear_error();
    if (!d_out || (n && (!d_bases || !d_scalars))) {
        set_error("ace_msm_g1_noalloc: NULL argument");
        return ACE_E_ARG;
    }
    if (base_form != ACE_FORM_CANONICAL && base_form != ACE_FORM_MONT) {
        set_error("ace_msm_g1_noalloc: base_form must be ACE_FORM_CANONICAL or ACE_FORM_MONT");
        return ACE_E_ARG;
    }
    if (n > NOALLOC_MAX_N) {
        set_error("ace_msm_g1_noalloc: n = %zu exceeds the maximum of %zu points of this entry point", n,
                  NOALLOC_MAX_N);
        return ACE_E_ARG;
    }
    if (((uintptr_t)d_bases | (uintptr_t)d_scalars | (uintptr_t)d_out) & 15u) {
        set_error("ace_msm_g1_noalloc: device buffers must be 16-byte aligned");
        return ACE_E_ARG;
    }
    void* base = nullptr;
    ACE_TRY(scratch_address(&base));
    MsmPlan plan = msm_plan(n, NOALLOC_C);
    plan.max_split = 1;  // the fixed scratch holds no partial bucket sums
    plan.alone = true;
    bool mont = base_form == ACE_FORM_MONT;
    if (msm_scratch_bytes<fp_t>(plan, mont) > NOALLOC_BYTES) {
        set_error("ace_msm_g1_noalloc: internal scratch bound exceeded");
        return ACE_E_INTERNAL;
    }
    Arena ar;
    ar.base = (char*)base;
    ar.cap = NOALLOC_BYTES;
    ar.off = 0;
    return msm_run<fp_t>(plan, (const g1_aff*)d_bases, mont, (const uint32_t*)d_scalars, ar, nullptr,
                         (g1_aff*)d_out, (cudaStream_t)stream);
}

}  // extern "C"
