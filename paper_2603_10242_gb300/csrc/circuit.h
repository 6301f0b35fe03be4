// circuit.h -- host representation of the synthetic R1CS (internal).
//
// The circuit stands in for the ZK-ACE statement of the paper (Section 3.3,
// "ZK-ACE circuit specification", constraint (i): the identity commitment
// id_com = Poseidon(REV, salt, domain) of Section 2.1).  Recipe:
//   variables: z_0 = 1, z_1 = public output, then per permutation its three
//     inputs and (x2, x4, x5) per S-box, then per packing row its bits and y,
//     then (without permutations) the chain start, then chain values x_1..;
//   rows: 243 per permutation (3 per S-box: s*s = x2, x2*x2 = x4,
//     x4*s = x5; 8 full rounds with 3 S-boxes, 57 partial rounds with one;
//     round constants and the Cauchy MDS layer fold into linear
//     combinations), then packing rows (sum 2^k b_k) * z_0 = y, then chain
//     rows x_i * x_i = x_{i+1} - k_i z_0 (x_0 = lane 0 of the last
//     permutation's output, the last value is z_1), then A = z_0 and A = z_1,
//     then zero rows up to N.
//   seeds (SplitMix64 streams): round constants (purpose 1, 65 x 3), MDS
//     x_0..2, y_0..2 (purpose 2, redrawn until distinct with x_i + y_j != 0),
//     chain constants (purpose 10) from the circuit seed; permutation inputs
//     and bits (purpose 3) from the witness seed.
#pragma once
#include <stdint.h>

#include <vector>

#include "../../include/ace.h"
#include "field.cuh"

namespace ace {

static const int PSN_ROUNDS = 65;  // 4 full + 57 partial + 4 full
static const int PSN_FULL_HALF = 4;
static const int ROWS_PER_PERM = 243;

struct Csr {
    std::vector<uint32_t> rp;   // N + 1
    std::vector<uint32_t> col;  // nnz
    std::vector<fr_t> val;      // nnz, Montgomery form
};

struct SplitMix64 {
    uint64_t s;
    SplitMix64(uint64_t seed, uint64_t purpose) : s(seed ^ (purpose * 0x9E3779B97F4A7C15ull)) {}
    uint64_t next() {
        s += 0x9E3779B97F4A7C15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    // uniform element of Fr, canonical limbs
    fr_t fr_canon() {
        for (;;) {
            fr_t x;
            for (int i = 0; i < 4; i++) {
                uint64_t w = next();
                if (i == 3) w &= 0x3FFFFFFFFFFFFFFFull;
                x.v[2 * i] = (uint32_t)w;
                x.v[2 * i + 1] = (uint32_t)(w >> 32);
            }
            if (!fe_geq_mod(x)) return x;
        }
    }
    fr_t fr_mont() { return fe_to_mont(fr_canon()); }
};

}  // namespace ace

struct ace_circuit {
    ace_circuit_params p;
    uint64_t N = 0, m = 0, n_chain = 0;
    ace::Csr mat[3];  // A, B, C
    ace::fr_t rc[ace::PSN_ROUNDS][3];
    ace::fr_t mds[3][3];
    std::vector<ace::fr_t> chain_k;
};

namespace ace {
// witness in Montgomery form (m values)
int circuit_witness_mont(const ace_circuit* c, uint64_t input_seed, std::vector<fr_t>& z);
// (Az) o (Bz) == Cz on the host, rows split over threads
bool circuit_check(const ace_circuit* c, const std::vector<fr_t>& z_mont);
unsigned host_threads();
}  // namespace ace
