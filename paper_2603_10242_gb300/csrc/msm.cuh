// msm.cuh -- Pippenger multi-scalar multiplication for G1 and G2 (internal).
//
// sum_i k_i P_i for affine P_i (Montgomery form) and canonical Fr scalars k_i:
//   1. signed c-bit digits of every scalar; scalars 0 contribute nothing and
//      scalars 1 go to an extra "ones" window of up to B virtual buckets
//      (their sum is that window's plain total), so the frequent {0,1}
//      witness values neither cost K additions nor pile onto one bucket;
//   2. counting sort of (bucket, point) pairs: histogram, exclusive scan,
//      scatter;
//   3. one mixed XYZZ addition per entry into its bucket;
//   4. per window sum_b b S_b: running sums over segments of L buckets
//      (16; 4 for one MSM whose windows hold at most 2^13 buckets, where the
//      segment chain is the reduction's latency) give W_j (weights 1..L
//      inside segment j) and S_j; one thread per
//      segment adds j L S_j to W_j (at most c - 1 doublings), and block-wide
//      trees sum the M segments of every window (256 to 1 per pass);
//   5. Horner over windows (c doublings each) plus the ones-window total.
// With precomputed window tables of the bases (the proving key's queries),
// every window's digits share one bucket set and step 5 is a single sum.
// These are the G1/G2 multi-scalar multiplications of Groth16.Prove (the
// paper's Section 3.1, Algorithm 1), computed for the A, B1, L and H queries
// on G1 and the B query on G2.
#pragma once
#include "curve.cuh"
#include "runtime.cuh"

namespace ace {

struct MsmPlan {
    size_t n = 0;
    int c = 0;       // window bits
    int K = 0;       // digit windows, ceil(255 / c)
    uint32_t B = 0;  // buckets per window, 2^(c-1)
    int lambda = 0;  // log2 of the segment length L
    uint32_t L = 0;
    uint32_t M = 0;  // segments per window, B / L
    // tabled: the bases come with precomputed window tables
    // tab[w n + i] = 2^(c w) P_i, so all K digit windows share one set of
    // buckets (no Horner over windows)
    bool tabled = false;
    // batch > 1: that many MSMs over the same n points, each with its own n
    // scalars (scalars and results laid out one MSM after another) and its
    // own bucket sets; every reduction step runs over all of them at once
    uint32_t batch = 1;
    // most threads one bucket's entries may be split among (1: no split)
    uint32_t max_split = 16;
    // glv (G1 without window tables): n counts the points P_i and phi(P_i)
    // of n / 2 input points, whose scalars are the 128-bit halves of the GLV
    // split (glv.cuh); K = ceil(128 / c) windows
    bool glv = false;
    // gls (G2 without window tables): n counts the points psi^t(Q_i), t < 4,
    // of n / 4 input points, whose scalars are the four parts of the split by
    // the endomorphism psi (glv.cuh, below 2^66); K = ceil(67 / c) windows
    bool gls = false;
    int bits() const { return glv ? 128 : gls ? 67 : 255; }
    // virtual buckets the ones window uses (a power of two <= B, about n / 64):
    // scalar 1 of point i goes to bucket i mod B1.  Enough buckets to spread
    // the additions over many threads, few enough that the window's plain sum
    // in the reduction stays short (its other buckets are empty)
    uint32_t B1 = 0;
    // a call that has the GPU to itself (one MSM, one proof): its reduction
    // runs on four lanes per segment while that still fits about one wave of
    // the GPU (see msm_impl.cuh); batched and served proofs leave it off
    bool alone = false;
    uint32_t ones_mask() const { return (B1 ? B1 : B) - 1u; }
    uint32_t bucket_windows() const { return tabled ? 1u : (uint32_t)K; }
    uint32_t windows() const { return bucket_windows() + 1; }  // + ones window
    uint32_t keys_per() const { return windows() * B; }         // keys of one MSM
    uint32_t keys() const { return batch * keys_per(); }
    uint32_t all_windows() const { return batch * windows(); }
    size_t scalars() const { return (size_t)batch * n; }
};

// c chosen by the cost model  max(n K madd + 2 K 2^(c-1) add, the top window's
// longest bucket run in sequence)  (force_c > 0 overrides)
MsmPlan msm_plan(size_t n, int force_c = 0);
// plan for tabled bases: cost n K madd + 2 2^(c-1) add, c <= 20
MsmPlan msm_plan_tabled(size_t n, int force_c = 0);
// G1 plan over the GLV split of n points (2 n virtual points, 128-bit scalars)
MsmPlan msm_plan_glv(size_t n, int force_c = 0);
// G2 plan over the four-way split of n points by psi (4 n virtual points,
// scalars below 2^66)
MsmPlan msm_plan_gls(size_t n, int force_c = 0);
// make p a plan for `batch` MSMs over the same points (segments of 16
// buckets again when batch > 1; see plan_for)
void msm_plan_set_batch(MsmPlan& p, uint32_t batch);
// GLV inputs of a G1 MSM: for i < n, out[i] = +-P_i and out[n + i] =
// +-phi(P_i) (Montgomery affine), osc[i] = |k1|, osc[n + i] = |k2| (8 limbs,
// canonical) with k_i mod r = k1 + k2 lambda and the signs moved onto the
// points.  in: n affine points (Montgomery if in_mont); sc: n scalars < 2^256.
int glv_prepare(const Affine<fp_t>* in, bool in_mont, const uint32_t* sc, size_t n, Affine<fp_t>* out,
                uint32_t* osc, cudaStream_t st);
// psi inputs of a G2 MSM: for i < n and t < 4, out[t n + i] = +-psi^t(Q_i)
// (Montgomery affine) and osc[t n + i] = |k_t| (8 limbs, canonical) with
// k_i mod r = k_0 + k_1 lambda + k_2 lambda^2 + k_3 lambda^3 and the signs
// moved onto the points.  in: n affine points (Montgomery if in_mont); sc: n
// scalars < 2^256.
int gls_prepare(const Affine<fp2_t>* in, bool in_mont, const uint32_t* sc, size_t n, Affine<fp2_t>* out,
                uint32_t* osc, cudaStream_t st);
// window table of n Montgomery affine points: tab[w n + i] = 2^(c w) pts[i]
// for w < K (pts may be tab itself, i.e. window 0 already in place)
template <class F>
int msm_build_table(const MsmPlan& plan, const Affine<F>* pts, Affine<F>* tab, cudaStream_t st);

template <class F, class A>
struct MsmBufs {
    uint32_t* offsets;   // keys + 1
    uint32_t* cursor;    // keys
    uint32_t* scan_tmp;  // scan block sums
    uint32_t* entries;   // n K
    uint32_t* order;     // keys, bucket keys by decreasing size
    uint32_t* size_bins; // SIZE_BINS + 1
    Xyzz<F>* buckets;    // keys
    Xyzz<F>* partial;    // keys x split (split parts per bucket), or buckets itself
    Xyzz<F>* segW;       // windows M
    Xyzz<F>* segS;       // windows M
    Affine<F>* conv;     // n (when bases arrive canonical, or the GLV points)
    uint32_t* gsc;       // n x 8 (GLV scalar halves only)
    template <class Alloc>
    bool carve(Alloc& a, const MsmPlan& p, bool need_conv);
};

// The sorted (bucket, point) entries of one MSM: bucket offsets (keys + 1),
// entries, bucket order.  A second MSM with the same scalars and plan over
// other bases (the B query on G1 and on G2) reuses them instead of sorting.
struct MsmSorted {
    const uint32_t* offsets = nullptr;
    const uint32_t* entries = nullptr;
    const uint32_t* order = nullptr;
};

// Run one MSM (plan.batch of them over the same bases).  d_bases: n affine
// points; base_mont says whether they are in Montgomery form.  Writes the
// XYZZ results (Montgomery, plan.batch of them) to d_res if non-null and the
// canonical affine results to d_out if non-null.  Scratch comes from `ar`
// (size it with msm_scratch_bytes).  Asynchronous on st.
// pre: sorted entries of an earlier MSM with the same scalars and plan (then
// d_scalars is not read; the caller orders st after that sort).  sorted /
// sorted_ev: hand out this run's sorted entries, and record sorted_ev on st
// when they are complete; they stay valid while `ar` is not reused.
template <class F>
int msm_run(const MsmPlan& plan, const Affine<F>* d_bases, bool base_mont, const uint32_t* d_scalars,
            Arena& ar, Xyzz<F>* d_res, Affine<F>* d_out, cudaStream_t st, const MsmSorted* pre = nullptr,
            MsmSorted* sorted = nullptr, cudaEvent_t sorted_ev = nullptr);
template <class F>
size_t msm_scratch_bytes(const MsmPlan& plan, bool base_mont);

// exclusive prefix sum of n u32 values in place; tmp holds ceil(n/1024)+1 words
int scan_exclusive_u32(uint32_t* d, size_t n, uint32_t* tmp, cudaStream_t st);
size_t scan_tmp_words(size_t n);

}  // namespace ace

namespace ace {
// buckets are processed in decreasing order of size so that the threads of a
// warp carry similar numbers of additions; sizes >= SIZE_BINS - 1 share a bin
static const uint32_t SIZE_BINS = 512;
// order[] = keys sorted by decreasing bucket size (counting sort on sizes)
int bucket_order(const uint32_t* offsets, uint32_t keys, uint32_t* bins, uint32_t* scan_tmp, uint32_t* order,
                 cudaStream_t st);
// digits of n scalars into (key, entry) pairs: histogram (SCATTER = false)
// or placement; tabled plans put every window's digit in one bucket set with
// entry w n + i
template <bool SCATTER>
void launch_digits(const MsmPlan& plan, const uint32_t* sc, uint32_t* cnt, uint32_t* entries, cudaStream_t st);
}  // namespace ace
