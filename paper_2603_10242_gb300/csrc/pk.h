// pk.h -- device-resident Groth16 proving key (internal).
#pragma once
#include <vector>

#include "circuit.h"
#include "curve.cuh"
#include "msm.cuh"
#include "ntt.cuh"
#include "runtime.cuh"

namespace ace {

// fixed points of the key, Montgomery affine, kept together on the device
struct PkFixed {
    g1_aff alpha1, beta1, delta1;
    g2_aff beta2, delta2;
};

// one compacted MSM query: points whose setup scalar is non-zero, and the
// witness index each one multiplies
template <class F>
struct Query {
    uint32_t count = 0;
    uint32_t* d_idx = nullptr;        // count (witness indices)
    Affine<F>* d_pts = nullptr;       // plan.K x count: window table, window 0 = the points (Montgomery affine)
    std::vector<uint32_t> h_idx;      // host copy of the indices (ascending)
    MsmPlan plan;                     // tabled MSM plan for count points
};

}  // namespace ace

struct ace_pk {
    ace_ctx* ctx = nullptr;
    ace_circuit_params params;
    uint64_t N = 0, m = 0;
    int log_n = 0;
    // R1CS on the device (CSR; values in Montgomery form)
    uint32_t* d_rp[3] = {};
    uint32_t* d_col[3] = {};
    ace::fr_t* d_val[3] = {};
    uint64_t nnz[3] = {};
    uint32_t* d_row_order = nullptr;  // N rows by decreasing total length (sparse-product schedule)
    ace::Query<ace::fp_t> A, B1, L;
    ace::Query<ace::fp2_t> B2;   // same indices as B1
    ace::g1_aff* d_H = nullptr;  // window table of N points: H_i = [L'_i(tau) Z(tau)/delta]_1, coset Lagrange basis
    ace::MsmPlan H_plan;         // tabled plan of the H query
    ace::PkFixed* d_fixed = nullptr;
    // 8-bit window tables (32 x 255 points) of alpha1, beta1, delta1 and delta2
    ace::g1_aff* d_tab_alpha1 = nullptr;
    ace::g1_aff* d_tab_beta1 = nullptr;
    ace::g1_aff* d_tab_delta1 = nullptr;
    ace::g2_aff* d_tab_delta2 = nullptr;
    ace_vk vk;
    size_t bytes = 0;            // device bytes held
    std::vector<std::pair<void*, size_t>> allocs;
    // host copy of the circuit (for ace_pk_save)
    ace_circuit* circ = nullptr;
};

namespace ace {
int pk_alloc(ace_pk* pk, void** p, size_t bytes);
// rows 0..N-1 ordered by decreasing number of non-zeros in A, B and C
// together (ties: by the A length, then the B length, then the row), uploaded to
// pk->d_row_order: the sparse product takes rows in this order so that the
// lanes of a warp have equal work
int pk_row_order(ace_pk* pk, const Csr mat[3]);
// window tables of the fixed points (after d_fixed is set)
int pk_build_tables(ace_pk* pk, const PkFixed& f);
// allocate the window table of a query of `count` points (window 0 to be
// filled by the caller), set its plan
template <class F>
int pk_alloc_table(ace_pk* pk, uint32_t count, MsmPlan* plan, Affine<F>** tab);
// where a batch's proof leaves its MSM sums: res1 = S_H, S_A, S_B1, S_L;
// res2 = S_B2 (device)
struct MsmOut {
    g1_xyzz* res1;
    g2_xyzz* res2;
};
// one whole proof on proving slot `slot` at stream priority level `prio`
// (prove.cu); with msm_out, only its QAP and MSMs
// one_stream: every stage on the slot's main stream in turn (no auxiliary
// streams), for batches whose proofs overlap across slots instead
// alone: the proof has the GPU to itself (one proof per call); its MSM plans
// are marked so (MsmPlan::alone)
int prove_run(ace_ctx* ctx, int slot, int prio, const ace_pk* pk, const fr_t* d_z, const fr_t& r, const fr_t& s,
              uint32_t* d_proof, int32_t* d_status, cudaStream_t st_in, bool join,
              const MsmOut* msm_out = nullptr, bool one_stream = false, bool alone = false);
// ace_prove_batch on proving slots only, never on the batch-dimension
// kernels (prove.cu; for the batch autotuner)
int prove_batch_on_slots(ace_ctx* ctx, size_t k, const ace_pk* const* pks, const ace_fr* const* d_zs,
                         const ace_fr* rs, const ace_fr* ss, uint8_t* proofs, int32_t* status);
// device bytes of scratch arena `arena` of a slot proving with `pk`
size_t prove_slot_bytes(const ace_pk* pk, int arena);
}  // namespace ace
