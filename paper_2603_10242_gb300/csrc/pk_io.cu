// pk_io.cu -- persistence of a proving key: setup at 2^20 and above is the
// expensive step, so a serving process reloads the key instead of redoing it.
//
// File layout (little-endian): "ACEPK001" | u32 version (2) | u32 header
// words | header (params, N, m, nnz[3], query counts) | circuit (CSR of A, B,
// C; round constants; MDS; chain constants) | queries (indices, Montgomery
// affine points) | H query (coset Lagrange basis; version 1 files held the
// monomial basis and are refused) | fixed points | verifying key.  Each array
// is preceded by its byte count (u64).
#include <stdio.h>
#include <string.h>

#include "pk.h"

namespace ace {
namespace {

const char MAGIC[8] = {'A', 'C', 'E', 'P', 'K', '0', '0', '1'};
const uint32_t VERSION = 2;

struct Writer {
    FILE* f;
    bool ok = true;
    void raw(const void* p, size_t n) {
        if (ok && n && fwrite(p, 1, n, f) != n) ok = false;
    }
    void arr(const void* p, size_t n) {
        uint64_t b = n;
        raw(&b, 8);
        raw(p, n);
    }
};
struct Reader {
    FILE* f;
    bool ok = true;
    void raw(void* p, size_t n) {
        if (ok && n && fread(p, 1, n, f) != n) ok = false;
    }
    template <class T>
    bool arr(std::vector<T>& v) {
        uint64_t b = 0;
        raw(&b, 8);
        if (!ok || b % sizeof(T) || b > (1ull << 40)) return ok = false;
        v.resize(b / sizeof(T));
        raw(v.data(), b);
        return ok;
    }
};

template <class T>
bool dev_to_host(const T* d, size_t n, std::vector<T>& h) {
    h.resize(n);
    return n == 0 || cudaMemcpy(h.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost) == cudaSuccess;
}

// upload window 0 of a query table and build the other windows
template <class F>
int table_to_dev(ace_pk* pk, const std::vector<Affine<F>>& h, MsmPlan* plan, Affine<F>** d) {
    ACE_TRY(pk_alloc_table<F>(pk, (uint32_t)h.size(), plan, d));
    if (h.empty()) return ACE_OK;
    ACE_TRY_CUDA(cudaMemcpy(*d, h.data(), h.size() * sizeof(Affine<F>), cudaMemcpyHostToDevice));
    ACE_TRY(msm_build_table<F>(*plan, *d, *d, pk->ctx->stream));
    ACE_TRY_CUDA(cudaStreamSynchronize(pk->ctx->stream));
    return ACE_OK;
}

template <class T>
int host_to_dev(ace_pk* pk, const std::vector<T>& h, T** d) {
    void* p = nullptr;
    ACE_TRY(pk_alloc(pk, &p, h.size() * sizeof(T) + 16));
    if (!h.empty()) ACE_TRY_CUDA(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    *d = (T*)p;
    return ACE_OK;
}

}  // namespace
}  // namespace ace

using namespace ace;

extern "C" {

int ace_pk_save(const ace_pk* pk, const char* path) {
    clear_error();
    if (!pk || !path || !pk->circ) {
        set_error("ace_pk_save: bad argument");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(pk->ctx->device));
    ACE_TRY_CUDA(cudaDeviceSynchronize());
    FILE* f = fopen(path, "wb");
    if (!f) {
        set_error("ace_pk_save: cannot open %s", path);
        return ACE_E_ARG;
    }
    Writer w{f};
    w.raw(MAGIC, 8);
    w.raw(&VERSION, 4);
    uint64_t hdr[9] = {pk->N, pk->m, pk->nnz[0], pk->nnz[1], pk->nnz[2], pk->A.count, pk->B1.count, pk->L.count,
                       pk->circ->n_chain};
    uint32_t nh = 9;
    w.raw(&nh, 4);
    w.raw(&pk->params, sizeof pk->params);
    w.raw(hdr, sizeof hdr);
    const ace_circuit* c = pk->circ;
    for (int k = 0; k < 3; k++) {
        w.arr(c->mat[k].rp.data(), c->mat[k].rp.size() * 4);
        w.arr(c->mat[k].col.data(), c->mat[k].col.size() * 4);
        w.arr(c->mat[k].val.data(), c->mat[k].val.size() * sizeof(fr_t));
    }
    w.arr(c->rc, sizeof c->rc);
    w.arr(c->mds, sizeof c->mds);
    w.arr(c->chain_k.data(), c->chain_k.size() * sizeof(fr_t));
    std::vector<g1_aff> g1;
    std::vector<g2_aff> g2;
    bool ok = true;
    w.arr(pk->A.h_idx.data(), pk->A.h_idx.size() * 4);
    ok = ok && dev_to_host(pk->A.d_pts, pk->A.count, g1);
    w.arr(g1.data(), g1.size() * sizeof(g1_aff));
    w.arr(pk->B1.h_idx.data(), pk->B1.h_idx.size() * 4);
    ok = ok && dev_to_host(pk->B1.d_pts, pk->B1.count, g1);
    w.arr(g1.data(), g1.size() * sizeof(g1_aff));
    ok = ok && dev_to_host(pk->B2.d_pts, pk->B2.count, g2);
    w.arr(g2.data(), g2.size() * sizeof(g2_aff));
    w.arr(pk->L.h_idx.data(), pk->L.h_idx.size() * 4);
    ok = ok && dev_to_host(pk->L.d_pts, pk->L.count, g1);
    w.arr(g1.data(), g1.size() * sizeof(g1_aff));
    ok = ok && dev_to_host(pk->d_H, pk->N, g1);
    w.arr(g1.data(), g1.size() * sizeof(g1_aff));
    std::vector<PkFixed> fx;
    ok = ok && dev_to_host(pk->d_fixed, 1, fx);
    w.arr(fx.data(), sizeof(PkFixed));
    w.arr(&pk->vk, sizeof pk->vk);
    bool good = w.ok && ok;
    if (fclose(f) != 0) good = false;
    if (!good) {
        set_error("ace_pk_save: write to %s failed", path);
        return ACE_E_ARG;
    }
    return ACE_OK;
}

int ace_pk_load(ace_ctx* ctx, const char* path, ace_pk** pk_out, ace_vk* vk_out) {
    clear_error();
    if (!ctx || !path || !pk_out) {
        set_error("ace_pk_load: NULL argument");
        return ACE_E_ARG;
    }
    *pk_out = nullptr;
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    FILE* f = fopen(path, "rb");
    if (!f) {
        set_error("ace_pk_load: cannot open %s", path);
        return ACE_E_ARG;
    }
    Reader r{f};
    char magic[8];
    uint32_t ver = 0, nh = 0;
    r.raw(magic, 8);
    r.raw(&ver, 4);
    r.raw(&nh, 4);
    if (!r.ok || memcmp(magic, MAGIC, 8) != 0 || ver != VERSION || nh != 9) {
        fclose(f);
        set_error("ace_pk_load: %s is not a version-%u proving key", path, VERSION);
        return ACE_E_ARG;
    }
    ace_pk* pk = new ace_pk();
    pk->ctx = ctx;
    ctx_ref(ctx);
    uint64_t hdr[9];
    r.raw(&pk->params, sizeof pk->params);
    r.raw(hdr, sizeof hdr);
    ace_circuit* c = new ace_circuit();
    pk->circ = c;
    c->p = pk->params;
    pk->N = c->N = hdr[0];
    pk->m = c->m = hdr[1];
    c->n_chain = hdr[8];
    pk->log_n = (int)pk->params.log_n;
    std::vector<fr_t> rcv, mdsv;
    for (int k = 0; k < 3; k++) {
        r.arr(c->mat[k].rp);
        r.arr(c->mat[k].col);
        r.arr(c->mat[k].val);
    }
    r.arr(rcv);
    r.arr(mdsv);
    r.arr(c->chain_k);
    std::vector<uint32_t> ia, ib, il;
    std::vector<g1_aff> pa, pb, pl, ph;
    std::vector<g2_aff> pb2;
    std::vector<PkFixed> fx;
    std::vector<uint8_t> vkb;
    r.arr(ia);
    r.arr(pa);
    r.arr(ib);
    r.arr(pb);
    r.arr(pb2);
    r.arr(il);
    r.arr(pl);
    r.arr(ph);
    r.arr(fx);
    r.arr(vkb);
    fclose(f);
    bool ok = r.ok && rcv.size() == 65 * 3 && mdsv.size() == 9 && fx.size() == 1 && vkb.size() == sizeof(ace_vk) &&
              ph.size() == pk->N && pa.size() == ia.size() && pb.size() == ib.size() && pb2.size() == ib.size() &&
              pl.size() == il.size() && c->mat[0].rp.size() == pk->N + 1;
    auto fail = [&](int code) {
        ace_pk_free(pk);
        return code;
    };
    if (!ok) {
        set_error("ace_pk_load: %s is truncated or inconsistent", path);
        return fail(ACE_E_ARG);
    }
    memcpy(c->rc, rcv.data(), sizeof c->rc);
    memcpy(c->mds, mdsv.data(), sizeof c->mds);
    memcpy(&pk->vk, vkb.data(), sizeof pk->vk);
    int rc = ACE_OK;
    for (int k = 0; k < 3 && rc == ACE_OK; k++) {
        pk->nnz[k] = c->mat[k].col.size();
        rc = host_to_dev(pk, c->mat[k].rp, &pk->d_rp[k]);
        if (rc == ACE_OK) rc = host_to_dev(pk, c->mat[k].col, &pk->d_col[k]);
        if (rc == ACE_OK) rc = host_to_dev(pk, c->mat[k].val, &pk->d_val[k]);
    }
    if (rc == ACE_OK) rc = pk_row_order(pk, c->mat);
    pk->A.count = (uint32_t)ia.size();
    pk->A.h_idx = ia;
    pk->B1.count = pk->B2.count = (uint32_t)ib.size();
    pk->B1.h_idx = pk->B2.h_idx = ib;
    pk->L.count = (uint32_t)il.size();
    pk->L.h_idx = il;
    if (rc == ACE_OK) rc = host_to_dev(pk, ia, &pk->A.d_idx);
    if (rc == ACE_OK) rc = table_to_dev(pk, pa, &pk->A.plan, &pk->A.d_pts);
    if (rc == ACE_OK) rc = host_to_dev(pk, ib, &pk->B1.d_idx);
    if (rc == ACE_OK) rc = table_to_dev(pk, pb, &pk->B1.plan, &pk->B1.d_pts);
    if (rc == ACE_OK) rc = host_to_dev(pk, ib, &pk->B2.d_idx);
    if (rc == ACE_OK) rc = table_to_dev(pk, pb2, &pk->B2.plan, &pk->B2.d_pts);
    if (rc == ACE_OK) rc = host_to_dev(pk, il, &pk->L.d_idx);
    if (rc == ACE_OK) rc = table_to_dev(pk, pl, &pk->L.plan, &pk->L.d_pts);
    if (rc == ACE_OK) rc = table_to_dev(pk, ph, &pk->H_plan, &pk->d_H);
    if (rc == ACE_OK) rc = host_to_dev(pk, fx, &pk->d_fixed);
    if (rc == ACE_OK) rc = pk_build_tables(pk, fx[0]);
    if (rc != ACE_OK) return fail(rc);
    if (vk_out) *vk_out = pk->vk;
    *pk_out = pk;
    return ACE_OK;
}

}  // extern "C"
