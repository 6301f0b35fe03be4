// setup.cu -- toy Groth16 setup: the circuit-specific trusted setup the paper
// assumes (Section 9, "Trusted setup"), with seeded toxic waste.
//
// Scalars (host):  L_i(tau) = (tau^N - 1) omega^i / (N (tau - omega^i)) by
// batch inversion; u_j, v_j, w_j = sum_i {A,B,C}_ij L_i(tau) over the
// columns; L-query (beta u_j + alpha v_j + w_j)/delta (j > 1) and the
// verifying-key inputs with /gamma (j <= 1); H-query in the Lagrange basis
// of the coset g H (see below).
// Points (device): fixed-base multiplication of the generators, stored in
// Montgomery affine form; zero scalars are compacted out of the queries.
// Every query is kept with its MSM window table (window w holds 2^(c w) times
// the points).
//
// H query.  The quotient h = (A B - C) / Z has degree at most N - 2, so its N
// values on the coset g H = {x_i = g omega^i} determine it:
//   h(tau) = sum_i h(x_i) L'_i(tau),
//   L'_i(tau) = x_i (tau^N - g^N) / (N g^N (tau - x_i))
// (the Lagrange basis of g H, whose vanishing polynomial is X^N - g^N).  The
// key stores H_i = [L'_i(tau) Z(tau) / delta]_1 for i < N in natural order,
// so the prover feeds the coset values of h, which the QAP step produces
// anyway, straight into the H MSM: sum_i h(x_i) H_i = [h(tau) Z(tau) /
// delta]_1, the same point as sum_e h_e [tau^e Z(tau) / delta]_1 over the
// coefficients, without the last inverse transform.
#include <string.h>

#include <algorithm>
#include <thread>

#include "fixed_base.cuh"
#include "pk.h"

namespace ace {

int pk_build_tables(ace_pk* pk, const PkFixed& f) {
    const size_t T = 32 * 255;
    ACE_TRY(pk_alloc(pk, (void**)&pk->d_tab_alpha1, T * sizeof(g1_aff)));
    ACE_TRY(pk_alloc(pk, (void**)&pk->d_tab_beta1, T * sizeof(g1_aff)));
    ACE_TRY(pk_alloc(pk, (void**)&pk->d_tab_delta1, T * sizeof(g1_aff)));
    ACE_TRY(pk_alloc(pk, (void**)&pk->d_tab_delta2, T * sizeof(g2_aff)));
    cudaStream_t st = pk->ctx->stream;
    ACE_TRY(fixed_table_build<fp_t>(pk->ctx, f.alpha1, pk->d_tab_alpha1, st));
    ACE_TRY(fixed_table_build<fp_t>(pk->ctx, f.beta1, pk->d_tab_beta1, st));
    ACE_TRY(fixed_table_build<fp_t>(pk->ctx, f.delta1, pk->d_tab_delta1, st));
    ACE_TRY(fixed_table_build<fp2_t>(pk->ctx, f.delta2, pk->d_tab_delta2, st));
    return ACE_OK;
}

template <class F>
int pk_alloc_table(ace_pk* pk, uint32_t count, MsmPlan* plan, Affine<F>** tab) {
    *plan = msm_plan_tabled(count);
    void* p = nullptr;
    ACE_TRY(pk_alloc(pk, &p, (size_t)plan->K * count * sizeof(Affine<F>) + 16));
    *tab = (Affine<F>*)p;
    return ACE_OK;
}
template int pk_alloc_table<fp_t>(ace_pk*, uint32_t, MsmPlan*, Affine<fp_t>**);
template int pk_alloc_table<fp2_t>(ace_pk*, uint32_t, MsmPlan*, Affine<fp2_t>**);

int pk_alloc(ace_pk* pk, void** p, size_t bytes) {
    ACE_TRY(dev_alloc(pk->ctx, p, bytes));
    pk->allocs.push_back({*p, bytes});
    pk->bytes += bytes;
    return ACE_OK;
}

static fr_t pow_u64(fr_t a, uint64_t e) {
    uint32_t ex[8] = {(uint32_t)e, (uint32_t)(e >> 32), 0, 0, 0, 0, 0, 0};
    return fe_pow(a, ex);
}

static fr_t nonzero(SplitMix64& g) {
    fr_t x;
    do { x = g.fr_canon(); } while (fe_is_zero(x));
    return fe_to_mont(x);
}

template <class F>
static int upload(ace_pk* pk, const void* src, size_t bytes, F** out) {
    void* p = nullptr;
    ACE_TRY(pk_alloc(pk, &p, bytes ? bytes : 16));
    if (bytes) ACE_TRY_CUDA(cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice));
    *out = (F*)p;
    return ACE_OK;
}

int pk_row_order(ace_pk* pk, const Csr mat[3]) {
    const uint64_t N = mat[0].rp.size() - 1;
    std::vector<uint64_t> key(N);
    for (uint64_t i = 0; i < N; i++) {
        const uint64_t a = mat[0].rp[i + 1] - mat[0].rp[i], b = mat[1].rp[i + 1] - mat[1].rp[i],
                       c = mat[2].rp[i + 1] - mat[2].rp[i];
        // 21 bits per length (rows are far shorter than 2^21 terms)
        key[i] = ((a + b + c) << 42) | (std::min<uint64_t>(a, (1u << 21) - 1) << 21) | std::min<uint64_t>(b, (1u << 21) - 1);
    }
    std::vector<uint32_t> order(N);
    for (uint64_t i = 0; i < N; i++) order[i] = (uint32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return key[x] > key[y]; });
    return upload(pk, order.data(), N * 4, &pk->d_row_order);
}

// columns of one matrix: col_sum[j] = sum_i M_ij L_i, threads over column ranges
static void column_sums(const Csr& M, uint64_t N, uint64_t m, const std::vector<fr_t>& Lt, std::vector<fr_t>& out) {
    std::vector<uint32_t> cnt(m + 1, 0);
    for (uint32_t c : M.col) cnt[c + 1]++;
    for (uint64_t j = 0; j < m; j++) cnt[j + 1] += cnt[j];
    std::vector<uint32_t> rows(M.col.size());
    std::vector<fr_t> coef(M.col.size());
    std::vector<uint32_t> cur(cnt.begin(), cnt.end() - 1);
    for (uint64_t i = 0; i < N; i++)
        for (uint32_t e = M.rp[i]; e < M.rp[i + 1]; e++) {
            uint32_t p = cur[M.col[e]]++;
            rows[p] = (uint32_t)i;
            coef[p] = M.val[e];
        }
    out.assign(m, fe_zero<FrCfg>());
    unsigned nt = host_threads();
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; t++)
        th.emplace_back([&, t]() {
            for (uint64_t j = t; j < m; j += nt) {
                fr_t acc = fe_zero<FrCfg>();
                for (uint32_t p = cnt[j]; p < cnt[j + 1]; p++) acc = acc + coef[p] * Lt[rows[p]];
                out[j] = acc;
            }
        });
    for (auto& x : th) x.join();
}

template <class F>
static int build_query(ace_pk* pk, const std::vector<fr_t>& scal, uint64_t from, Query<F>& q, cudaStream_t st) {
    std::vector<uint32_t> idx;
    std::vector<fr_t> sc;
    for (uint64_t j = from; j < scal.size(); j++)
        if (!fe_is_zero(scal[j])) {
            idx.push_back((uint32_t)j);
            sc.push_back(fe_from_mont(scal[j]));
        }
    q.count = (uint32_t)idx.size();
    q.h_idx = idx;
    ACE_TRY(upload(pk, idx.data(), idx.size() * 4, &q.d_idx));
    ACE_TRY(pk_alloc_table<F>(pk, q.count, &q.plan, &q.d_pts));
    if (q.count) {
        fr_t* d_sc = nullptr;
        ACE_TRY_CUDA(cudaMalloc(&d_sc, sc.size() * sizeof(fr_t)));
        ACE_TRY_CUDA(cudaMemcpy(d_sc, sc.data(), sc.size() * sizeof(fr_t), cudaMemcpyHostToDevice));
        int rc = fixed_base_mul<F>(pk->ctx, (const uint32_t*)d_sc, q.count, q.d_pts, true, st);
        if (rc == ACE_OK) rc = msm_build_table<F>(q.plan, q.d_pts, q.d_pts, st);
        cudaError_t e = cudaStreamSynchronize(st);
        cudaFree(d_sc);
        ACE_TRY(rc);
        ACE_TRY_CUDA(e);
    }
    return ACE_OK;
}

template <class F>
static void canon_point(const Affine<F>& mont, void* out);
template <>
void canon_point<fp_t>(const g1_aff& p, void* out) {
    g1_aff c = aff_from_mont(p);
    memcpy(out, &c, sizeof c);
}
template <>
void canon_point<fp2_t>(const g2_aff& p, void* out) {
    g2_aff c = aff_from_mont(p);
    memcpy(out, &c, sizeof c);
}

}  // namespace ace

using namespace ace;

static void pk_release(ace_pk* pk) {
    if (!pk) return;
    ace_ctx* ctx = pk->ctx;
    if (ctx) {
        cudaSetDevice(ctx->device);
        cudaDeviceSynchronize();
        for (auto& a : pk->allocs) dev_free(ctx, a.first, a.second);
    }
    delete pk->circ;
    delete pk;
    if (ctx) ctx_unref(ctx);
}

extern "C" {

int ace_setup_toy(ace_ctx* ctx, const ace_circuit* c, uint64_t toxic_seed, ace_pk** pk_out, ace_vk* vk_out) {
    clear_error();
    if (!ctx || !c || !pk_out) {
        set_error("ace_setup_toy: NULL argument");
        return ACE_E_ARG;
    }
    *pk_out = nullptr;
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const uint64_t N = c->N, m = c->m;
    const int log_n = (int)c->p.log_n;
    ace_pk* pk = new ace_pk();
    pk->ctx = ctx;
    ctx_ref(ctx);
    pk->params = c->p;
    pk->N = N;
    pk->m = m;
    pk->log_n = log_n;
    pk->circ = new ace_circuit(*c);
    int rc = ACE_OK;
#define SETUP_TRY(expr)                 \
    do {                                \
        rc = (expr);                    \
        if (rc != ACE_OK) {             \
            pk_release(pk);             \
            return rc;                  \
        }                               \
    } while (0)

    // toxic waste
    SplitMix64 g(toxic_seed, 4);
    fr_t tau, one = fe_one<FrCfg>();
    for (;;) {
        tau = nonzero(g);
        if (!fe_eq(pow_u64(tau, N), one)) break;
    }
    fr_t alpha = nonzero(g), beta = nonzero(g), gamma = nonzero(g), delta = nonzero(g);

    // Lagrange basis at tau
    fr_t omega = root_of_unity_host(log_n);
    fr_t zt = pow_u64(tau, N) - one;
    fr_t ninv = fe_inv(pow_u64(fe_from_u32<FrCfg>(2), (uint64_t)log_n));
    std::vector<fr_t> Lt(N), den(N), pre(N);
    {
        fr_t w = one;
        for (uint64_t i = 0; i < N; i++) {
            Lt[i] = w;  // omega^i for now
            den[i] = tau - w;
            w = w * omega;
        }
        fr_t acc = one;
        for (uint64_t i = 0; i < N; i++) {
            pre[i] = acc;
            acc = acc * den[i];
        }
        acc = fe_inv(acc);
        for (uint64_t i = N; i-- > 0;) {
            fr_t inv_i = acc * pre[i];
            acc = acc * den[i];
            den[i] = inv_i;
        }
        fr_t zn = zt * ninv;
        for (uint64_t i = 0; i < N; i++) Lt[i] = zn * Lt[i] * den[i];
    }
    std::vector<fr_t> u, v, w;
    column_sums(c->mat[0], N, m, Lt, u);
    column_sums(c->mat[1], N, m, Lt, v);
    column_sums(c->mat[2], N, m, Lt, w);
    fr_t dinv = fe_inv(delta), ginv = fe_inv(gamma);
    std::vector<fr_t> lq(m);
    for (uint64_t j = 0; j < m; j++) lq[j] = (beta * u[j] + alpha * v[j] + w[j]) * (j <= 1 ? ginv : dinv);

    // R1CS on the device
    for (int k = 0; k < 3; k++) {
        const Csr& M = c->mat[k];
        pk->nnz[k] = M.col.size();
        SETUP_TRY(upload(pk, M.rp.data(), M.rp.size() * 4, &pk->d_rp[k]));
        SETUP_TRY(upload(pk, M.col.data(), M.col.size() * 4, &pk->d_col[k]));
        SETUP_TRY(upload(pk, M.val.data(), M.val.size() * sizeof(fr_t), &pk->d_val[k]));
    }
    SETUP_TRY(pk_row_order(pk, c->mat));
    // queries
    SETUP_TRY(build_query<fp_t>(pk, u, 0, pk->A, st));
    SETUP_TRY(build_query<fp_t>(pk, v, 0, pk->B1, st));
    SETUP_TRY(build_query<fp2_t>(pk, v, 0, pk->B2, st));
    {
        std::vector<fr_t> lq2(lq);
        lq2[0] = fe_zero<FrCfg>();
        lq2[1] = fe_zero<FrCfg>();
        SETUP_TRY(build_query<fp_t>(pk, lq2, 0, pk->L, st));
    }
    // H query in the Lagrange basis of the coset g H (natural order):
    // H_i = K x_i / (tau - x_i) with K = (tau^N - g^N) Z(tau) / (N g^N delta),
    // or, when tau lies on the coset (tau = x_k), H_i = [i = k] Z(tau)/delta
    {
        std::vector<fr_t> hs(N);
        const fr_t gc = fe_from_u32<FrCfg>(5), gn = pow_u64(gc, N), tn = pow_u64(tau, N);
        std::vector<fr_t> xs(N), dx(N), pre2(N);
        fr_t x = gc, acc = one;
        bool on_coset = false;
        for (uint64_t i = 0; i < N; i++) {
            xs[i] = x;
            dx[i] = tau - x;
            if (fe_is_zero(dx[i])) on_coset = true;
            x = x * omega;
        }
        if (on_coset) {
            for (uint64_t i = 0; i < N; i++) hs[i] = fe_is_zero(dx[i]) ? fe_from_mont(zt * dinv) : fe_zero<FrCfg>();
        } else {
            for (uint64_t i = 0; i < N; i++) {
                pre2[i] = acc;
                acc = acc * dx[i];
            }
            acc = fe_inv(acc);
            for (uint64_t i = N; i-- > 0;) {
                fr_t inv_i = acc * pre2[i];
                acc = acc * dx[i];
                dx[i] = inv_i;
            }
            const fr_t K = (tn - gn) * zt * ninv * fe_inv(gn) * dinv;
            for (uint64_t i = 0; i < N; i++) hs[i] = fe_from_mont(K * xs[i] * dx[i]);
        }
        fr_t* d_sc = nullptr;
        SETUP_TRY(upload(pk, hs.data(), N * sizeof(fr_t), &d_sc));
        SETUP_TRY(pk_alloc_table<fp_t>(pk, (uint32_t)N, &pk->H_plan, &pk->d_H));
        SETUP_TRY(fixed_base_mul<fp_t>(ctx, (const uint32_t*)d_sc, N, pk->d_H, true, st));
        SETUP_TRY(msm_build_table<fp_t>(pk->H_plan, pk->d_H, pk->d_H, st));
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("setup: H query kernel failed");
            pk_release(pk);
            return ACE_E_CUDA;
        }
    }
    // fixed points and verifying key
    {
        fr_t g1s[6] = {fe_from_mont(alpha), fe_from_mont(beta), fe_from_mont(delta),
                       fe_from_mont(lq[0]), fe_from_mont(lq[1]), fe_zero<FrCfg>()};
        fr_t g2s[3] = {fe_from_mont(beta), fe_from_mont(gamma), fe_from_mont(delta)};
        fr_t *d1 = nullptr, *d2 = nullptr;
        SETUP_TRY(upload(pk, g1s, sizeof g1s, &d1));
        SETUP_TRY(upload(pk, g2s, sizeof g2s, &d2));
        g1_aff* o1 = nullptr;
        g2_aff* o2 = nullptr;
        SETUP_TRY(pk_alloc(pk, (void**)&o1, 6 * sizeof(g1_aff)));
        SETUP_TRY(pk_alloc(pk, (void**)&o2, 3 * sizeof(g2_aff)));
        SETUP_TRY(fixed_base_mul<fp_t>(ctx, (const uint32_t*)d1, 6, o1, true, st));
        SETUP_TRY(fixed_base_mul<fp2_t>(ctx, (const uint32_t*)d2, 3, o2, true, st));
        g1_aff h1[6];
        g2_aff h2[3];
        if (cudaMemcpyAsync(h1, o1, sizeof h1, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(h2, o2, sizeof h2, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("setup: fixed points failed");
            pk_release(pk);
            return ACE_E_CUDA;
        }
        PkFixed f;
        f.alpha1 = h1[0];
        f.beta1 = h1[1];
        f.delta1 = h1[2];
        f.beta2 = h2[0];
        f.delta2 = h2[2];
        SETUP_TRY(upload(pk, &f, sizeof f, &pk->d_fixed));
        SETUP_TRY(pk_build_tables(pk, f));
        canon_point<fp_t>(h1[0], &pk->vk.alpha1);
        canon_point<fp2_t>(h2[0], &pk->vk.beta2);
        canon_point<fp2_t>(h2[1], &pk->vk.gamma2);
        canon_point<fp2_t>(h2[2], &pk->vk.delta2);
        canon_point<fp_t>(h1[3], &pk->vk.ic[0]);
        canon_point<fp_t>(h1[4], &pk->vk.ic[1]);
    }
#undef SETUP_TRY
    if (vk_out) *vk_out = pk->vk;
    *pk_out = pk;
    return ACE_OK;
}

int ace_pk_free(ace_pk* pk) {
    pk_release(pk);
    return ACE_OK;
}

int ace_pk_info(const ace_pk* pk, uint64_t info[ACE_INFO_LEN]) {
    if (!pk || !info) {
        set_error("ace_pk_info: NULL argument");
        return ACE_E_ARG;
    }
    memset(info, 0, sizeof(uint64_t) * ACE_INFO_LEN);
    info[ACE_INFO_N] = pk->N;
    info[ACE_INFO_M] = pk->m;
    info[ACE_INFO_ROWS] = pk->params.n_rows;
    info[ACE_INFO_NNZ_A] = pk->nnz[0];
    info[ACE_INFO_NNZ_B] = pk->nnz[1];
    info[ACE_INFO_NNZ_C] = pk->nnz[2];
    info[ACE_INFO_M_A] = pk->A.count;
    info[ACE_INFO_M_B] = pk->B1.count;
    info[ACE_INFO_M_L] = pk->L.count;
    info[ACE_INFO_DEVICE_BYTES] = pk->bytes;
    return ACE_OK;
}

int ace_pk_point(const ace_pk* pk, int query, size_t index, void* out) {
    clear_error();
    if (!pk || !out || query < 0 || query > 4) {
        set_error("ace_pk_point: bad argument");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(pk->ctx->device));
    if (query == 4) {
        if (index >= pk->N) {
            set_error("ace_pk_point: H index %zu out of range", index);
            return ACE_E_ARG;
        }
        g1_aff p;
        ACE_TRY_CUDA(cudaMemcpy(&p, pk->d_H + index, sizeof p, cudaMemcpyDeviceToHost));
        canon_point<fp_t>(p, out);
        return ACE_OK;
    }
    if (index >= pk->m) {
        set_error("ace_pk_point: index %zu out of range", index);
        return ACE_E_ARG;
    }
    const std::vector<uint32_t>& idx = query == 0 ? pk->A.h_idx : query == 3 ? pk->L.h_idx : pk->B1.h_idx;
    auto it = std::lower_bound(idx.begin(), idx.end(), (uint32_t)index);
    bool present = it != idx.end() && *it == index;
    size_t k = it - idx.begin();
    if (query == 2) {
        if (!present) {
            memset(out, 0, sizeof(g2_aff));
            return ACE_OK;
        }
        g2_aff p;
        ACE_TRY_CUDA(cudaMemcpy(&p, pk->B2.d_pts + k, sizeof p, cudaMemcpyDeviceToHost));
        canon_point<fp2_t>(p, out);
        return ACE_OK;
    }
    if (!present) {
        memset(out, 0, sizeof(g1_aff));
        return ACE_OK;
    }
    const g1_aff* src = (query == 0 ? pk->A.d_pts : query == 3 ? pk->L.d_pts : pk->B1.d_pts) + k;
    g1_aff p;
    ACE_TRY_CUDA(cudaMemcpy(&p, src, sizeof p, cudaMemcpyDeviceToHost));
    canon_point<fp_t>(p, out);
    return ACE_OK;
}

}  // extern "C"
