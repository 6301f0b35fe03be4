// circuit.cpp -- seeded synthetic R1CS and its witness (host), see circuit.h.
#include "circuit.h"

#include <stdarg.h>
#include <string.h>

#include <algorithm>
#include <thread>
#include <utility>

namespace ace {
void set_error(const char* fmt, ...);
void clear_error();
}  // namespace ace

namespace ace {
namespace {

typedef std::vector<std::pair<uint32_t, fr_t>> Lc;  // sorted by variable, no zero coefficients

void lc_normalise(Lc& a) {
    std::stable_sort(a.begin(), a.end(),
                     [](const std::pair<uint32_t, fr_t>& x, const std::pair<uint32_t, fr_t>& y) {
                         return x.first < y.first;
                     });
    Lc out;
    out.reserve(a.size());
    for (auto& t : a) {
        if (!out.empty() && out.back().first == t.first)
            out.back().second = out.back().second + t.second;
        else
            out.push_back(t);
    }
    a.clear();
    for (auto& t : out)
        if (!fe_is_zero(t.second)) a.push_back(t);
}

Lc lc_var(uint32_t v) { return Lc{{v, fe_one<FrCfg>()}}; }

struct Builder {
    ace_circuit* c;
    uint32_t next_var = 0;
    uint32_t rows = 0;

    uint32_t alloc() { return next_var++; }

    void row(const Lc* A, const Lc* B, const Lc* C) {
        const Lc* M[3] = {A, B, C};
        for (int k = 0; k < 3; k++) {
            Csr& m = c->mat[k];
            if (M[k])
                for (auto& t : *M[k]) {
                    m.col.push_back(t.first);
                    m.val.push_back(t.second);
                }
            m.rp[rows + 1] = (uint32_t)m.col.size();
        }
        rows++;
    }

    // s^5 as three rows; returns the x5 variable
    uint32_t sbox(const Lc& s) {
        uint32_t x2 = alloc();
        Lc l2 = lc_var(x2);
        row(&s, &s, &l2);
        uint32_t x4 = alloc();
        Lc l4 = lc_var(x4);
        row(&l2, &l2, &l4);
        uint32_t x5 = alloc();
        Lc l5 = lc_var(x5);
        row(&l4, &s, &l5);
        return x5;
    }

    Lc permutation() {
        Lc lane[3];
        for (int l = 0; l < 3; l++) lane[l] = lc_var(alloc());
        for (int r = 0; r < PSN_ROUNDS; r++) {
            bool full = r < PSN_FULL_HALF || r >= PSN_ROUNDS - PSN_FULL_HALF;
            for (int l = 0; l < 3; l++) {
                lane[l].push_back({0u, c->rc[r][l]});
                lc_normalise(lane[l]);
            }
            for (int l = 0; l < (full ? 3 : 1); l++) lane[l] = lc_var(sbox(lane[l]));
            Lc nl[3];
            for (int i = 0; i < 3; i++) {
                for (int j = 0; j < 3; j++)
                    for (auto& t : lane[j]) nl[i].push_back({t.first, t.second * c->mds[i][j]});
                lc_normalise(nl[i]);
            }
            for (int i = 0; i < 3; i++) lane[i].swap(nl[i]);
        }
        return lane[0];
    }
};

}  // namespace

unsigned host_threads() {
    unsigned t = std::thread::hardware_concurrency();
    return t ? (t > 64 ? 64 : t) : 4;
}

// Witness by direct evaluation of the permutation, packing and chain, in the
// variable order of the recipe.
int circuit_witness_mont(const ace_circuit* c, uint64_t input_seed, std::vector<fr_t>& z) {
    z.assign(c->m, fe_zero<FrCfg>());
    SplitMix64 rin(input_seed, 3);
    uint64_t pos = 0;
    z[pos++] = fe_one<FrCfg>();
    pos++;  // z_1 is the last chain value
    fr_t last = fe_zero<FrCfg>();
    for (uint32_t p = 0; p < c->p.n_perm; p++) {
        fr_t lane[3];
        for (int l = 0; l < 3; l++) {
            lane[l] = rin.fr_mont();
            z[pos++] = lane[l];
        }
        for (int r = 0; r < PSN_ROUNDS; r++) {
            bool full = r < PSN_FULL_HALF || r >= PSN_ROUNDS - PSN_FULL_HALF;
            for (int l = 0; l < 3; l++) lane[l] = lane[l] + c->rc[r][l];
            for (int l = 0; l < (full ? 3 : 1); l++) {
                fr_t s = lane[l];
                fr_t x2 = fe_sqr(s);
                fr_t x4 = fe_sqr(x2);
                fr_t x5 = x4 * s;
                z[pos++] = x2;
                z[pos++] = x4;
                z[pos++] = x5;
                lane[l] = x5;
            }
            fr_t nl[3];
            for (int i = 0; i < 3; i++)
                nl[i] = c->mds[i][0] * lane[0] + c->mds[i][1] * lane[1] + c->mds[i][2] * lane[2];
            for (int i = 0; i < 3; i++) lane[i] = nl[i];
        }
        last = lane[0];
    }
    for (uint32_t q = 0; q < c->p.n_pack; q++) {
        fr_t y = fe_zero<FrCfg>(), pw = fe_one<FrCfg>();
        for (uint32_t k = 0; k < c->p.pack_bits; k++) {
            bool bit = (rin.next() & 1u) != 0;
            z[pos++] = bit ? fe_one<FrCfg>() : fe_zero<FrCfg>();
            if (bit) y = y + pw;
            pw = pw + pw;
        }
        z[pos++] = y;
    }
    if (c->p.n_perm == 0) {
        last = rin.fr_mont();
        z[pos++] = last;
    }
    fr_t x = last;
    for (uint64_t i = 0; i < c->n_chain; i++) {
        x = fe_sqr(x) + c->chain_k[i];
        if (i + 1 == c->n_chain)
            z[1] = x;
        else
            z[pos++] = x;
    }
    if (pos != c->m) {
        set_error("witness: produced %llu values, circuit has %llu", (unsigned long long)pos,
                  (unsigned long long)c->m);
        return ACE_E_ARG;
    }
    return ACE_OK;
}

bool circuit_check(const ace_circuit* c, const std::vector<fr_t>& z) {
    const uint64_t N = c->N;
    unsigned nt = host_threads();
    std::vector<int> ok(nt, 1);
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; t++) {
        th.emplace_back([&, t]() {
            uint64_t lo = N * t / nt, hi = N * (t + 1) / nt;
            for (uint64_t i = lo; i < hi && ok[t]; i++) {
                fr_t v[3];
                for (int k = 0; k < 3; k++) {
                    const Csr& m = c->mat[k];
                    fr_t acc = fe_zero<FrCfg>();
                    for (uint32_t e = m.rp[i]; e < m.rp[i + 1]; e++) acc = acc + m.val[e] * z[m.col[e]];
                    v[k] = acc;
                }
                if (!fe_eq(v[0] * v[1], v[2])) ok[t] = 0;
            }
        });
    }
    for (auto& x : th) x.join();
    for (int v : ok)
        if (!v) return false;
    return true;
}

}  // namespace ace

using namespace ace;

extern "C" {

int ace_circuit_gen(const ace_circuit_params* p, ace_circuit** out) {
    clear_error();
    if (!p || !out) {
        set_error("ace_circuit_gen: NULL argument");
        return ACE_E_ARG;
    }
    *out = nullptr;
    if (p->log_n < 2 || p->log_n > 26) {
        set_error("ace_circuit_gen: log_n = %u outside [2, 26]", p->log_n);
        return ACE_E_ARG;
    }
    uint64_t N = 1ull << p->log_n;
    uint64_t fixed = 2 + (uint64_t)ROWS_PER_PERM * p->n_perm + p->n_pack;
    if (p->n_rows > N || p->n_rows < fixed + 1 || p->pack_bits > 253) {
        set_error("ace_circuit_gen: n_rows = %u must satisfy %llu <= n_rows <= %llu (and pack_bits <= 253)",
                  p->n_rows, (unsigned long long)(fixed + 1), (unsigned long long)N);
        return ACE_E_ARG;
    }
    ace_circuit* c = new ace_circuit();
    c->p = *p;
    c->N = N;
    c->n_chain = p->n_rows - fixed;
    c->m = 2 + (uint64_t)p->n_perm * (3 + ROWS_PER_PERM) + (uint64_t)p->n_pack * (p->pack_bits + 1) +
           (p->n_perm == 0 ? 1 : 0) + (c->n_chain - 1);
    if (c->m >= (1ull << 31)) {
        delete c;
        set_error("ace_circuit_gen: too many variables");
        return ACE_E_ARG;
    }
    for (int k = 0; k < 3; k++) c->mat[k].rp.assign(N + 1, 0);

    SplitMix64 g(p->seed, 1);
    for (int r = 0; r < PSN_ROUNDS; r++)
        for (int l = 0; l < 3; l++) c->rc[r][l] = g.fr_mont();
    SplitMix64 gm(p->seed, 2);
    for (;;) {
        fr_t x[3], y[3];
        for (auto& v : x) v = gm.fr_mont();
        for (auto& v : y) v = gm.fr_mont();
        bool ok = true;
        for (int i = 0; i < 3; i++)
            for (int j = i + 1; j < 3; j++) ok = ok && !fe_eq(x[i], x[j]) && !fe_eq(y[i], y[j]);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) ok = ok && !fe_is_zero(x[i] + y[j]);
        if (!ok) continue;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) c->mds[i][j] = fe_inv(x[i] + y[j]);
        break;
    }
    SplitMix64 gk(p->seed, 10);
    c->chain_k.resize(c->n_chain);
    for (auto& k : c->chain_k) k = gk.fr_mont();

    Builder b;
    b.c = c;
    b.alloc();  // z_0
    b.alloc();  // z_1
    // Every permutation has the same rows over its own block of
    // 3 + ROWS_PER_PERM variables (and z_0 for constants): build the first
    // one with linear combinations, then replicate its rows with the
    // variable block shifted.
    Lc chain_start;
    if (p->n_perm > 0) {
        const uint32_t v0 = b.next_var, r0 = b.rows;
        Lc out0 = b.permutation();
        const uint32_t nv = b.next_var - v0, nr = b.rows - r0;
        for (uint32_t q = 1; q < p->n_perm; q++) {
            const uint32_t shift = q * nv;
            for (uint32_t rr = 0; rr < nr; rr++) {
                for (int k = 0; k < 3; k++) {
                    Csr& m = c->mat[k];
                    uint32_t a = m.rp[r0 + rr], bnd = m.rp[r0 + rr + 1];
                    for (uint32_t e = a; e < bnd; e++) {
                        uint32_t v = m.col[e];
                        m.col.push_back(v == 0 ? 0u : v + shift);
                        m.val.push_back(m.val[e]);
                    }
                    m.rp[b.rows + 1] = (uint32_t)m.col.size();
                }
                b.rows++;
            }
            b.next_var += nv;
        }
        const uint32_t last_shift = (p->n_perm - 1) * nv;
        for (auto& t : out0) chain_start.push_back({t.first == 0 ? 0u : t.first + last_shift, t.second});
    }
    for (uint32_t q = 0; q < p->n_pack; q++) {
        Lc A;
        fr_t pw = fe_one<FrCfg>();
        for (uint32_t k = 0; k < p->pack_bits; k++) {
            A.push_back({b.alloc(), pw});
            pw = pw + pw;
        }
        Lc B = lc_var(0), C = lc_var(b.alloc());
        b.row(&A, &B, &C);
    }
    if (p->n_perm == 0) chain_start = lc_var(b.alloc());
    Lc x = chain_start;
    for (uint64_t i = 0; i < c->n_chain; i++) {
        uint32_t tgt = (i + 1 == c->n_chain) ? 1u : b.alloc();
        Lc C = lc_var(tgt);
        C.push_back({0u, fe_neg(c->chain_k[i])});
        lc_normalise(C);
        b.row(&x, &x, &C);
        x = lc_var(tgt);
    }
    for (uint32_t j = 0; j < 2; j++) {
        Lc A = lc_var(j);
        b.row(&A, nullptr, nullptr);
    }
    while (b.rows < N) b.row(nullptr, nullptr, nullptr);
    if (b.next_var != c->m) {
        set_error("ace_circuit_gen: internal variable count mismatch");
        delete c;
        return ACE_E_ARG;
    }
    for (int k = 0; k < 3; k++)
        if (c->mat[k].col.size() >= (1ull << 32)) {
            set_error("ace_circuit_gen: more than 2^32 non-zeros");
            delete c;
            return ACE_E_ARG;
        }
    *out = c;
    return ACE_OK;
}

int ace_circuit_free(ace_circuit* c) {
    delete c;
    return ACE_OK;
}

int ace_circuit_info(const ace_circuit* c, uint64_t info[ACE_INFO_LEN]) {
    if (!c || !info) {
        set_error("ace_circuit_info: NULL argument");
        return ACE_E_ARG;
    }
    memset(info, 0, sizeof(uint64_t) * ACE_INFO_LEN);
    info[ACE_INFO_N] = c->N;
    info[ACE_INFO_M] = c->m;
    info[ACE_INFO_ROWS] = c->p.n_rows;
    info[ACE_INFO_CHAIN] = c->n_chain;
    info[ACE_INFO_NNZ_A] = c->mat[0].col.size();
    info[ACE_INFO_NNZ_B] = c->mat[1].col.size();
    info[ACE_INFO_NNZ_C] = c->mat[2].col.size();
    return ACE_OK;
}

int ace_witness(const ace_circuit* c, uint64_t input_seed, ace_fr* z_out, size_t m) {
    clear_error();
    if (!c || !z_out) {
        set_error("ace_witness: NULL argument");
        return ACE_E_ARG;
    }
    if (m != c->m) {
        set_error("ace_witness: m = %zu but the circuit has %llu variables", m, (unsigned long long)c->m);
        return ACE_E_ARG;
    }
    std::vector<fr_t> z;
    int rc = circuit_witness_mont(c, input_seed, z);
    if (rc != ACE_OK) return rc;
    if (!circuit_check(c, z)) {
        set_error("ace_witness: generated witness does not satisfy the R1CS");
        return ACE_E_UNSAT;
    }
    for (size_t j = 0; j < m; j++) {
        fr_t v = fe_from_mont(z[j]);
        memcpy(z_out[j].l, v.v, 32);
    }
    return ACE_OK;
}

int ace_rs_from_seed(uint64_t seed, ace_fr* r, ace_fr* s) {
    if (!r || !s) {
        set_error("ace_rs_from_seed: NULL argument");
        return ACE_E_ARG;
    }
    SplitMix64 g(seed, 5);
    fr_t x;
    do { x = g.fr_canon(); } while (fe_is_zero(x));
    memcpy(r->l, x.v, 32);
    do { x = g.fr_canon(); } while (fe_is_zero(x));
    memcpy(s->l, x.v, 32);
    return ACE_OK;
}

}  // extern "C"
