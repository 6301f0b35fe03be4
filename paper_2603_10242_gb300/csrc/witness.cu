// witness.cu -- witnesses of many circuit instances on the device: the w_tx
// that every transaction's proof starts from (Section 3.3, Algorithm 3: each
// GenZKACEProof call proves one transaction's witness), computed for a whole
// block at once instead of on the host.
//
// The values are those of the host generator (circuit.cpp) for the same
// circuit and input seed, in the same variable order:
//   * the input stream (SplitMix64, seed, purpose 3) is counter based: word t
//     is mix(s0 + t gamma), so any word can be computed directly.  An Fr draw
//     takes attempts of 4 words (top 2 bits cleared) until one is below r;
//     one warp per instance finds the attempts that are accepted (ballot and
//     population count over 32 attempts at a time) and records them in order;
//   * one thread per permutation: its 3 input draws, then the 65 rounds (add
//     constants, x^5 S-boxes writing x^2, x^4, x^5, the Cauchy MDS layer);
//   * one thread per packing row: its bits (the low bit of one word each) and
//     y = sum 2^k b_k;
//   * one thread per instance: the chain x_{i+1} = x_i^2 + k_i from lane 0 of
//     the last permutation's output (or, without permutations, from one more
//     draw after the bits); the last chain value is z_1.
#include <string.h>

#include <vector>

#include "circuit.h"
#include "runtime.cuh"

namespace ace {
namespace {

const uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t sm_word(uint64_t s0, uint64_t t) {  // word t >= 1 of the stream
    uint64_t z = s0 + t * SM_GAMMA;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// candidate of attempt j (words 4 j + 1 .. 4 j + 4 after position base)
__device__ __forceinline__ fr_t sm_attempt(uint64_t s0, uint64_t base, uint64_t j) {
    fr_t x;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        uint64_t w = sm_word(s0, base + 4 * j + i + 1);
        if (i == 3) w &= 0x3FFFFFFFFFFFFFFFull;
        x.v[2 * i] = (uint32_t)w;
        x.v[2 * i + 1] = (uint32_t)(w >> 32);
    }
    return x;
}

struct WitCircuit {
    uint32_t n_perm, n_pack, pack_bits;
    uint64_t n_chain, m;
    const fr_t* rc;       // 65 x 3, Montgomery
    const fr_t* mds;      // 3 x 3, Montgomery
    const fr_t* chain_k;  // n_chain, Montgomery
};

// One warp per instance: att[q][i] = index of the attempt that yields draw i
// (i < D), after[q] = stream words used by the D draws.  err is set if the
// bounded search ends early (it cannot for any practical D: each attempt is
// accepted with probability r / 2^254 > 0.75).
__global__ void k_wit_draws(const uint64_t* seeds, uint32_t k, uint32_t D, uint32_t* att, uint64_t* after,
                            int32_t* err) {
    const uint32_t q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31;
    if (q >= k) return;
    const uint64_t s0 = seeds[q] ^ (3ull * SM_GAMMA);
    uint32_t cnt = 0;
    uint64_t j0 = 0;
    const uint64_t limit = 4ull * D + 4096;
    while (cnt < D && j0 < limit) {
        const uint64_t j = j0 + lane;
        fr_t v = sm_attempt(s0, 0, j);
        const bool acc = !fe_geq_mod(v);
        const uint32_t bal = __ballot_sync(0xffffffffu, acc);
        const uint32_t rank = __popc(bal & ((1u << lane) - 1u));
        if (acc && cnt + rank < D) att[(size_t)q * D + cnt + rank] = (uint32_t)j;
        cnt += __popc(bal);
        j0 += 32;
    }
    __syncwarp();  // the lane that stored the last draw's attempt may be another one
    if (lane == 0) {
        if (cnt < D) {
            atomicOr(err, 1);
            after[q] = 0;
        } else {
            after[q] = D ? 4ull * ((uint64_t)att[(size_t)q * D + D - 1] + 1) : 0;
        }
    }
}

// one thread per (instance, permutation)
__global__ void k_wit_perm(WitCircuit c, const uint64_t* seeds, uint32_t k, const uint32_t* att, fr_t* z,
                           fr_t* last) {
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (uint64_t)k * c.n_perm) return;
    const uint32_t q = (uint32_t)(g / c.n_perm), p = (uint32_t)(g % c.n_perm);
    const uint64_t s0 = seeds[q] ^ (3ull * SM_GAMMA);
    const uint32_t D = 3 * c.n_perm;
    fr_t* zq = z + (size_t)q * c.m;
    size_t pos = 2 + (size_t)p * (3 + ROWS_PER_PERM);
    fr_t lane[3];
    for (int l = 0; l < 3; l++) {
        fr_t v = sm_attempt(s0, 0, att[(size_t)q * D + 3 * p + l]);
        zq[pos++] = v;
        lane[l] = fe_to_mont(v);
    }
#pragma unroll 1
    for (int r = 0; r < PSN_ROUNDS; r++) {
        const bool full = r < PSN_FULL_HALF || r >= PSN_ROUNDS - PSN_FULL_HALF;
        for (int l = 0; l < 3; l++) lane[l] = lane[l] + c.rc[3 * r + l];
        for (int l = 0; l < (full ? 3 : 1); l++) {
            fr_t s = lane[l];
            fr_t x2 = fe_sqr(s);
            fr_t x4 = fe_sqr(x2);
            fr_t x5 = x4 * s;
            zq[pos++] = fe_from_mont(x2);
            zq[pos++] = fe_from_mont(x4);
            zq[pos++] = fe_from_mont(x5);
            lane[l] = x5;
        }
        fr_t nl[3];
        for (int i = 0; i < 3; i++) nl[i] = c.mds[3 * i] * lane[0] + c.mds[3 * i + 1] * lane[1] + c.mds[3 * i + 2] * lane[2];
        for (int i = 0; i < 3; i++) lane[i] = nl[i];
    }
    if (p + 1 == c.n_perm) last[q] = lane[0];
}

// one thread per (instance, packing row)
__global__ void k_wit_pack(WitCircuit c, const uint64_t* seeds, uint32_t k, const uint64_t* after, fr_t* z) {
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (uint64_t)k * c.n_pack) return;
    const uint32_t q = (uint32_t)(g / c.n_pack), row = (uint32_t)(g % c.n_pack);
    const uint64_t s0 = seeds[q] ^ (3ull * SM_GAMMA);
    fr_t* zq = z + (size_t)q * c.m;
    size_t pos = 2 + (size_t)c.n_perm * (3 + ROWS_PER_PERM) + (size_t)row * (c.pack_bits + 1);
    const uint64_t w0 = after[q] + (uint64_t)row * c.pack_bits;
    fr_t y = fe_zero<FrCfg>(), pw = fe_one<FrCfg>();
    for (uint32_t t = 0; t < c.pack_bits; t++) {
        const bool bit = (sm_word(s0, w0 + t + 1) & 1u) != 0;
        fr_t b = fe_zero<FrCfg>();
        b.v[0] = bit ? 1u : 0u;
        zq[pos++] = b;
        if (bit) y = y + pw;
        pw = pw + pw;
    }
    zq[pos] = fe_from_mont(y);
}

// one thread per instance: z_0, the chain start (without permutations) and
// the chain; the last chain value is z_1
__global__ void k_wit_chain(WitCircuit c, const uint64_t* seeds, uint32_t k, const uint64_t* after, const fr_t* last,
                            fr_t* z, int32_t* err) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= k) return;
    fr_t* zq = z + (size_t)q * c.m;
    zq[0] = fe_from_mont(fe_one<FrCfg>());
    size_t pos = 2 + (size_t)c.n_perm * (3 + ROWS_PER_PERM) + (size_t)c.n_pack * (c.pack_bits + 1);
    fr_t x;
    if (c.n_perm == 0) {
        const uint64_t s0 = seeds[q] ^ (3ull * SM_GAMMA);
        const uint64_t base = after[q] + (uint64_t)c.n_pack * c.pack_bits;
        fr_t v = fe_zero<FrCfg>();
        bool ok = false;
        for (uint64_t j = 0; j < 4096 && !ok; j++) {
            v = sm_attempt(s0, base, j);
            ok = !fe_geq_mod(v);
        }
        if (!ok) atomicOr(err, 1);
        zq[pos++] = v;
        x = fe_to_mont(v);
    } else {
        x = last[q];
    }
    for (uint64_t i = 0; i < c.n_chain; i++) {
        x = fe_sqr(x) + c.chain_k[i];
        if (i + 1 == c.n_chain)
            zq[1] = fe_from_mont(x);
        else
            zq[pos++] = fe_from_mont(x);
    }
}

}  // namespace
}  // namespace ace

using namespace ace;

extern "C" {

int ace_witness_many(ace_ctx* ctx, const ace_circuit* c, size_t k, const uint64_t* seeds, ace_fr* d_z,
                     ace_stream stream) {
    clear_error();
    if (!ctx || !c || (k && (!seeds || !d_z))) {
        set_error("ace_witness_many: NULL argument");
        return ACE_E_ARG;
    }
    if (k == 0) return ACE_OK;
    if (k > (1u << 24)) {
        set_error("ace_witness_many: k = %zu instances (at most 2^24)", k);
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = pick_stream(ctx, stream);
    const uint32_t D = 3 * c->p.n_perm;
    // constants (Montgomery), seeds, draw positions and per-instance words
    std::vector<fr_t> consts;
    consts.reserve(PSN_ROUNDS * 3 + 9 + c->n_chain);
    for (int r = 0; r < PSN_ROUNDS; r++)
        for (int l = 0; l < 3; l++) consts.push_back(c->rc[r][l]);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) consts.push_back(c->mds[i][j]);
    for (auto& x : c->chain_k) consts.push_back(x);
    const size_t bytes = consts.size() * sizeof(fr_t) + k * (8 + 8 + sizeof(fr_t)) + (size_t)k * D * 4 + 4096;
    ACE_TRY(arena_ensure(ctx, 2, bytes));
    Arena& a = ctx->scratch[2];
    fr_t* d_consts = (fr_t*)a.take(consts.size() * sizeof(fr_t));
    uint64_t* d_seeds = (uint64_t*)a.take(k * 8);
    uint64_t* d_after = (uint64_t*)a.take(k * 8);
    fr_t* d_last = (fr_t*)a.take(k * sizeof(fr_t));
    uint32_t* d_att = (uint32_t*)a.take((size_t)k * D * 4 + 4);
    int32_t* d_err = (int32_t*)a.take(16);
    if (!d_consts || !d_seeds || !d_after || !d_last || !d_att || !d_err) {
        set_error("ace_witness_many: scratch too small");
        return ACE_E_OOM;
    }
    ACE_TRY_CUDA(cudaMemcpyAsync(d_consts, consts.data(), consts.size() * sizeof(fr_t), cudaMemcpyHostToDevice, st));
    ACE_TRY_CUDA(cudaMemcpyAsync(d_seeds, seeds, k * 8, cudaMemcpyHostToDevice, st));
    ACE_TRY_CUDA(cudaMemsetAsync(d_err, 0, 4, st));
    WitCircuit wc;
    wc.n_perm = c->p.n_perm;
    wc.n_pack = c->p.n_pack;
    wc.pack_bits = c->p.pack_bits;
    wc.n_chain = c->n_chain;
    wc.m = c->m;
    wc.rc = d_consts;
    wc.mds = d_consts + PSN_ROUNDS * 3;
    wc.chain_k = d_consts + PSN_ROUNDS * 3 + 9;
    const uint32_t kk = (uint32_t)k;
    k_wit_draws<<<(unsigned)((k * 32 + 127) / 128), 128, 0, st>>>(d_seeds, kk, D, d_att, d_after, d_err);
    ::ace::note_launch();
    if (wc.n_perm) {
        const uint64_t n = (uint64_t)k * wc.n_perm;
        k_wit_perm<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(wc, d_seeds, kk, d_att, (fr_t*)d_z, d_last);
        ::ace::note_launch();
    }
    if (wc.n_pack) {
        const uint64_t n = (uint64_t)k * wc.n_pack;
        k_wit_pack<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(wc, d_seeds, kk, d_after, (fr_t*)d_z);
        ::ace::note_launch();
    }
    k_wit_chain<<<(unsigned)((k + 63) / 64), 64, 0, st>>>(wc, d_seeds, kk, d_after, d_last, (fr_t*)d_z, d_err);
    ::ace::note_launch();
    ACE_TRY_CUDA(cudaGetLastError());
    int32_t err = 0;
    // the host vector of constants must outlive its copy, and the draw search
    // reports its (practically impossible) failure
    ACE_TRY_CUDA(cudaMemcpyAsync(&err, d_err, 4, cudaMemcpyDeviceToHost, st));
    ACE_TRY_CUDA(cudaStreamSynchronize(st));
    if (err) {
        set_error("ace_witness_many: an input draw found no accepted attempt within its bound");
        return ACE_E_ARG;
    }
    return ACE_OK;
}

}  // extern "C"
