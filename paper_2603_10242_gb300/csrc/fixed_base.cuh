// fixed_base.cuh -- batch scalar multiplication of the G1 / G2 generators (internal).
#pragma once
#include "curve.cuh"
#include "runtime.cuh"

namespace ace {
// generator in Montgomery form: G1 = (1, 2), G2 = the EIP-197 generator
template <class F>
Affine<F> generator_mont();
// d_out[i] = k_i G for canonical scalars k_i (n x 8 limbs); asynchronous on st
template <class F>
int fixed_base_mul(ace_ctx* ctx, const uint32_t* d_scalars, size_t n, Affine<F>* d_out, bool out_mont,
                   cudaStream_t st);
// 8-bit window table of an arbitrary base point: tab[w * 255 + d - 1] =
// d 2^(8w) P (32 x 255 Montgomery affine points), synchronous on st
template <class F>
int fixed_table_build(ace_ctx* ctx, const Affine<F>& base_mont, Affine<F>* d_tab, cudaStream_t st);

// k P from the window table of P (k: 8 little-endian limbs); one thread
template <class F>
__device__ __forceinline__ Xyzz<F> fixed_mul_tab(const Affine<F>* tab, const uint32_t* k) {
    Xyzz<F> acc = xyzz_inf<F>();
#pragma unroll 1
    for (int w = 0; w < 32; w++) {
        uint32_t d = (k[w >> 2] >> ((w & 3) * 8)) & 255u;
        if (d) acc = xyzz_add_aff(acc, tab[w * 255 + d - 1]);
    }
    return acc;
}
}  // namespace ace
