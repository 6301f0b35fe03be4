// ntt.cuh -- number-theoretic transforms over Fr (internal).
//
// Domain H = {omega^i}, omega = 5^((r-1)/N) (5 is a non-residue mod r and
// 2^28 | r - 1); coset g H with g = 5.  A transform is a sequence of passes,
// each doing t stages (radix-2, or radix-4 pairs of stages) on groups of 2^t
// elements staged in shared memory (limb-planar layout with a swizzled word
// index, one 32-byte element per index).  Forward
// passes are decimation in frequency (natural order in, bit-reversed out);
// the transform that follows consumes bit-reversed input by decimation in
// time, so the QAP pipeline never permutes data.  Per-element factors (coset
// powers g^i, 1/N, Montgomery conversion) are applied while a pass loads or
// stores, from two small power tables.  These are the iNTT / coset NTT steps
// of the QAP quotient in Groth16.Prove (the paper's Section 3.1, Algorithm 1).
#pragma once
#include "curve.cuh"
#include "runtime.cuh"

namespace ace {

struct NttPlan {
    int log_n = 0;
    size_t n = 0;
    int h = 0;                // factor index split: e = (e_hi << h) | e_lo
    fr_t* tw_fwd = nullptr;   // omega^j, j < N/2 (Montgomery)
    fr_t* tw_inv = nullptr;   // omega^-j
    fr_t* cos_hi = nullptr;   // N^-1 g^(e_hi 2^h) (Montgomery)
    fr_t* cos_lo = nullptr;   // g^e_lo (Montgomery)
    fr_t* cg_hi = nullptr;    // g^(e_hi 2^h) (Montgomery)
    fr_t* icos_hi = nullptr;  // N^-1 g^-(e_hi 2^h) (Montgomery)
    fr_t* icos_lo = nullptr;  // g^-e_lo as a plain value: the product leaves Montgomery form
    fr_t* icos_lo_m = nullptr;  // g^-e_lo (Montgomery): with icos_hi, the factor for canonical data
    fr_t* ninv = nullptr;     // [N^-1] (Montgomery), single entry
    fr_t* one = nullptr;      // [1] (Montgomery), single entry
    fr_t* plain_one = nullptr;  // [1] as a plain value: multiplying by it leaves Montgomery form
    fr_t* rr = nullptr;       // [R^2 mod r] raw: multiplying by it enters Montgomery form
    fr_t zinv;                // (g^N - 1)^-1 (Montgomery)
    int smem_log = 11;        // log2 of the elements one block stages in shared memory (tunable)
    int radix = 4;            // 4: stages in radix-4 pairs, 2: radix-2 stages only (tunable)
    void* mem = nullptr;
    size_t bytes = 0;
};

// omega_N = 5^((r-1)/N) in Montgomery form (host)
fr_t root_of_unity_host(int log_n);
int ntt_get_plan(ace_ctx* ctx, int log_n, NttPlan** out);
// Stage form before tuning: radix-4 pairs from 2^18 elements up, where they
// were measured 2-6% faster; radix-2 below (13% faster at 2^16, where a
// transform is a few short passes and the radix-2 kernel's lower register
// count keeps more blocks resident)
inline int ntt_default_radix(int log_n) { return log_n >= 18 ? 4 : 2; }
void ntt_release_plans(ace_ctx* ctx);

// Factor applied to the element at position p: hi[e >> h] * lo[e & (2^h-1)]
// with e = p or e = bitrev(p); `single` uses hi[0] * lo[0] everywhere.
struct NttScale {
    const fr_t* hi = nullptr;
    const fr_t* lo = nullptr;
    int h = 0;
    int brev = 0;
    int single = 0;
};

// In-place transform of `count` consecutive arrays of N = 2^log_n elements.
// dif: natural -> bit-reversed (else bit-reversed -> natural); inverse
// selects omega^-1.  pre applies at the first load, post at the last store.
// fill_waves: narrow the blocks of a pass when that fills the GPU's last wave
// of blocks better (a transform with the GPU to itself); the prover's
// transforms share the GPU with its MSMs and keep the plan's width.
int ntt_run(const NttPlan& plan, fr_t* data, int count, bool dif, bool inverse, const NttScale& pre,
            const NttScale& post, cudaStream_t st,
            bool fill_waves = false);

// The same transform out of place: the first pass reads `in`, every pass
// writes `work` except the last, which writes `out` (at bit-reversed
// positions when out_brev: a DIF transform then leaves natural order).  Any
// two of the three may be the same array, except work and out when out_brev
// and the transform takes more than one pass (ACE_E_INTERNAL).
int ntt_run_io(const NttPlan& plan, const fr_t* in, fr_t* work, fr_t* out, bool out_brev, int count, bool dif,
               bool inverse, const NttScale& pre, const NttScale& post, cudaStream_t st, bool fill_waves = false);


}  // namespace ace
