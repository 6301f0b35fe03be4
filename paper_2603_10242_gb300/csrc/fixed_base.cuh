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
}  // namespace ace
