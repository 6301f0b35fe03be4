/*
 * ace.h -- C ABI of the GB300 (sm_103a) Groth16/BN254 prover library (libace.so).
 *
 * The library computes the proof of the paper's Phase 2: Groth16.Prove(C, w,
 * pub) run off the critical path on the builder's GPU (Section 3.1,
 * Algorithm 1 ProveAsync; Section 3.3, Algorithm 3 GPUProofPipeline Stage 1),
 * over BN254 (Section 3.3, "ZK-ACE circuit specification"), producing the
 * single 256-byte proof of Section 3.3 / Appendix B, checked by the three-
 * pairing verification of Section 3.4 (Algorithm 4).  The paper treats Groth16
 * as a black box; the QAP / setup / prover algebra follows Groth 2016, which
 * it cites.
 *
 * Conventions
 *  - Every function returns int: ACE_OK (0) or a negative ACE_E_* code.
 *    ace_verify returns 1 (valid), 0 (invalid) or a negative code.
 *    Nothing aborts, traps or prints; ace_last_error() returns the message of
 *    the last failure on the calling thread.
 *  - Field elements (ace_fr, ace_fp) are 8 little-endian 32-bit limbs in
 *    CANONICAL form (value < modulus) unless an argument says ACE_FORM_MONT
 *    (Montgomery form x * 2^256 mod p).  G1 affine = {x, y}; G2 affine =
 *    {x.c0, x.c1, y.c0, y.c1} over Fp2 = Fp[u]/(u^2+1).  The point at infinity
 *    is all-zero coordinates ((0,0) is on neither curve).
 *  - Proof bytes (256): A.x | A.y | B.x.c0 | B.x.c1 | B.y.c0 | B.y.c1 | C.x | C.y,
 *    each 32-byte little-endian canonical.
 *  - Arguments named d_* are DEVICE pointers on the context's device; all
 *    others are host pointers.  The caller owns every buffer it passes; the
 *    library never frees caller memory.  Opaque handles are owned by the
 *    library and released by the matching *_free / *_destroy call.
 *  - `stream` is a cudaStream_t (NULL = the context's own stream).  Device
 *    work is enqueued on that stream; functions that return results in host
 *    memory synchronise it before returning.
 *  - A context is not thread-safe: use one context per host thread.
 */
#ifndef ACE_H
#define ACE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ACE_OK 0
#define ACE_E_ARG (-1)          /* invalid argument (size, pointer, non-canonical value) */
#define ACE_E_OOM (-2)          /* device or host allocation failed */
#define ACE_E_CUDA (-3)         /* a CUDA call failed (message in ace_last_error) */
#define ACE_E_UNSAT (-4)        /* witness does not satisfy the R1CS */
#define ACE_E_NOT_ON_CURVE (-5) /* an input point is not on the curve */
#define ACE_E_TIMEOUT (-6)      /* a bounded device wait expired */
#define ACE_E_BUSY (-7)         /* admission refused / result not ready */
#define ACE_E_INTERNAL (-8)     /* an internal bound of the library was exceeded (a library fault, not a bad argument) */

#define ACE_FORM_CANONICAL 0
#define ACE_FORM_MONT 1

typedef struct CUstream_st* ace_stream; /* == cudaStream_t */
typedef struct ace_ctx ace_ctx;
typedef struct ace_circuit ace_circuit;
typedef struct ace_pk ace_pk;
typedef struct ace_server ace_server;

typedef struct { uint32_t l[8]; } ace_fr;
typedef struct { uint32_t l[8]; } ace_fp;
typedef struct { ace_fp x, y; } ace_g1_affine;
typedef struct { ace_fp x[2], y[2]; } ace_g2_affine;

/* Verifying key for l = 1 public input: ic[0] + x_1 ic[1] is the input term. */
typedef struct {
    ace_g1_affine alpha1;
    ace_g2_affine beta2, gamma2, delta2;
    ace_g1_affine ic[2];
} ace_vk;

/* Seeded synthetic R1CS over Fr with N = 2^log_n rows:
 *   n_perm Poseidon-style permutations (width 3, x^5 S-box, 8 full + 57
 *   partial rounds; the identity commitment of Section 2.1, Definition "ZK
 *   Identity Commitment", constraint (i) of the ZK-ACE circuit), 243 rows each;
 *   n_pack bit-packing rows (sum_k 2^k b_k) * 1 = y with pack_bits seeded bits;
 *   a chain of squaring gates x_{i+1} = x_i^2 + k_i filling rows up to n_rows - 2;
 *   two input-consistency rows (A = z_0, A = z_1); rows n_rows..N-1 are zero.
 * One public input (l = 1): z_1, the last chain value.
 * Requires 2 <= log_n <= 26, n_rows <= N, pack_bits <= 253 and
 * n_rows >= 243 n_perm + n_pack + 3. */
typedef struct {
    uint32_t log_n;
    uint32_t n_rows;
    uint32_t n_perm;
    uint32_t n_pack;
    uint32_t pack_bits;
    uint64_t seed;
} ace_circuit_params;

/* info[] layout of ace_circuit_info / ace_pk_info */
enum {
    ACE_INFO_N = 0,      /* QAP domain size */
    ACE_INFO_M = 1,      /* witness length (z_0 = 1, z_1 public, private ...) */
    ACE_INFO_ROWS = 2,   /* rows carrying constraints */
    ACE_INFO_CHAIN = 3,  /* chain rows */
    ACE_INFO_NNZ_A = 4,
    ACE_INFO_NNZ_B = 5,
    ACE_INFO_NNZ_C = 6,
    ACE_INFO_M_A = 7,    /* pk: non-zero A-query points (after compaction) */
    ACE_INFO_M_B = 8,    /* pk: non-zero B-query points */
    ACE_INFO_M_L = 9,    /* pk: non-zero L-query points */
    ACE_INFO_DEVICE_BYTES = 10, /* pk: device memory held */
    ACE_INFO_LEN = 12
};

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * memory the context's caches and scratch may hold (0 = no bound); calls
 * that would exceed it return ACE_E_OOM. */
int ace_ctx_create(ace_ctx** out, int device, size_t hbm_budget_bytes);
/* Releases the context.  Proving keys and servers made on it keep it alive:
 * with any of them left, the context is freed when the last one is freed
 * (so the order in which a caller releases them does not matter). */
int ace_ctx_destroy(ace_ctx* ctx);
/* Message of the last error on this thread ("" if none).  Never NULL. */
const char* ace_last_error(void);
/* Bytes of device memory currently held by the context (caches + scratch). */
int ace_ctx_device_bytes(const ace_ctx* ctx, size_t* out);

/* ---- circuit and witness (host) ----------------------------------------- */

/* Build the seeded synthetic R1CS described at ace_circuit_params (host):
 * the circuit C of Groth16.Prove(C, w, pub) in the builder's proving stage
 * (Section 3.1, Algorithm 1; Section 3.3, Algorithm 3), made of the
 * Poseidon-style identity-commitment gadget (Section 2.1, Definition "ZK
 * Identity Commitment"; Appendix B, the constraint group of the commitment)
 * plus packing rows and a squaring chain.  *out is lib-owned (free with
 * ace_circuit_free).  ACE_E_ARG if the parameters break the requirements
 * listed at ace_circuit_params; ACE_E_OOM if host memory runs out. */
int ace_circuit_gen(const ace_circuit_params* p, ace_circuit** out);
int ace_circuit_free(ace_circuit* c);
int ace_circuit_info(const ace_circuit* c, uint64_t info[ACE_INFO_LEN]);

/* Witness z (m canonical Fr values) for the circuit: Groth16.Prove's w_tx
 * input (Section 3.1, Algorithm 1).  Private inputs are drawn from input_seed
 * (SplitMix64, purpose 3).  Checks the R1CS on the host; ACE_E_UNSAT if it
 * fails (cannot happen for a generated witness), ACE_E_ARG if m is wrong. */
int ace_witness(const ace_circuit* c, uint64_t input_seed, ace_fr* z_out, size_t m);

/* ---- setup -------------------------------------------------------------- */

/* Toy trusted setup (the circuit-specific trusted setup of Section 9, "Trusted setup") with toxic
 * waste tau, alpha, beta, gamma, delta drawn from toxic_seed (SplitMix64,
 * purpose 4; zero rejected; tau^N = 1 rejected).  The proving key is built on
 * the device and stays resident there; vk_out (host) receives the verifying
 * key.  Points whose scalar is zero are compacted out of the MSM inputs. */
int ace_setup_toy(ace_ctx* ctx, const ace_circuit* c, uint64_t toxic_seed, ace_pk** pk_out,
                  ace_vk* vk_out);
int ace_pk_free(ace_pk* pk);
int ace_pk_info(const ace_pk* pk, uint64_t info[ACE_INFO_LEN]);
/* Copy one proving-key point to host memory (affine, canonical).
 * query: 0 A_j = [u_j(tau)]1, 1 B1_j = [v_j(tau)]1, 2 B2_j = [v_j(tau)]2 (out is
 * an ace_g2_affine), 3 L_j = [(beta u_j + alpha v_j + w_j)(tau)/delta]1 (j > 1),
 * 4 H_i = [L'_i(tau) Z(tau)/delta]1 (i < N), L'_i the Lagrange basis of the
 * coset g H = {5 omega^i} (the prover multiplies it by the quotient's values
 * on that coset); j indexes the witness, i the domain.  Infinity is returned
 * as zeros. */
int ace_pk_point(const ace_pk* pk, int query, size_t index, void* out);

/* ---- hot path ----------------------------------------------------------- */

/* QAP quotient of Groth16.Prove (Section 3.1, Algorithm 1; the QAP of Groth
 * 2016): h = (A(X) B(X) - C(X)) / (X^N - 1) where A, B, C interpolate
 * Az, Bz, Cz on H = {omega^i}, omega = 5^((r-1)/N).  Steps: sparse products,
 * 3 inverse NTTs, 3 coset NTTs on g H (g = 5), pointwise (a b - c)/(g^N - 1),
 * coset inverse NTT.  d_z: m canonical Fr (device); d_h_out: N canonical Fr
 * (device), natural coefficient order, h_{N-1} = 0.  Asynchronous on stream.
 * Scratch is drawn from the context.  (ace_prove stops before the last step:
 * its H query is in the Lagrange basis of g H and takes the coset values.) */
int ace_qap_h(ace_ctx* ctx, const ace_pk* pk, const ace_fr* d_z, ace_fr* d_h_out, ace_stream stream);

/* The multi-scalar multiplications of Groth16.Prove (Section 3.1, Algorithm
 * 1): sum_i k_i P_i over G1 (Pippenger: signed c-bit
 * digits, bucket sort, bucket accumulation, bucket and window reduction).
 * d_bases: n affine points in base_form (ACE_FORM_CANONICAL or _MONT);
 * d_scalars: n canonical Fr; d_out: one affine canonical point (device).
 * n may be 0 (result is infinity).  Asynchronous on stream.  For n < 2^30
 * the G1 scalars are split by the GLV endomorphism, k = k1 + k2 lambda with
 * 128-bit halves over P_i and (beta x_i, y_i), which halves the digit
 * windows; any 256-bit scalar is then taken modulo r.  Scratch (buckets,
 * sorted digits, 2n prepared points and scalar halves) is drawn from the
 * context. */
int ace_msm_g1(ace_ctx* ctx, const ace_g1_affine* d_bases, int base_form, const ace_fr* d_scalars,
               size_t n, ace_g1_affine* d_out, ace_stream stream);
/* Same over G2 (coordinates in Fp2): the B query of the proof.  For
 * n <= 2^16 the scalars are split four ways by the endomorphism psi of G2
 * (k = k0 + k1 lambda + k2 lambda^2 + k3 lambda^3, parts below 2^66, over
 * the points psi^t(Q_i)), which cuts the digit windows from 17 to 7; any
 * 256-bit scalar is then taken modulo r.  Larger MSMs use full-width
 * scalars.  Scratch (buckets, sorted digits, 4n prepared points and parts)
 * is drawn from the context. */
int ace_msm_g2(ace_ctx* ctx, const ace_g2_affine* d_bases, int base_form, const ace_fr* d_scalars,
               size_t n, ace_g2_affine* d_out, ace_stream stream);

/* G1 MSM that allocates no device memory, for callers that cannot call
 * cudaMalloc (their device memory is owned by a pool handed out up front, or
 * they must not trigger the device-wide synchronisation that allocation and
 * freeing imply).  The paper has no counterpart; this is a library service.
 * Same arguments and result as ace_msm_g1, without a context: it runs on the
 * current device, on `stream` (NULL = the legacy default stream).  n must be
 * at most 16384 (ACE_E_ARG otherwise; ACE_E_INTERNAL if the library's own
 * scratch bound were exceeded, which its fixed plan rules out).  Its scratch is one fixed 6 MiB device
 * array inside the library, present on every GPU that loads the library
 * until the process exits; the first call on a device looks up that array's
 * address (make that first call before any stream capture).  Every call
 * shares the array and leaves its contents behind (the call clears what must
 * start at zero), so calls whose work overlaps on the GPU race. */
int ace_msm_g1_noalloc(const ace_g1_affine* d_bases, int base_form, const ace_fr* d_scalars, size_t n,
                       ace_g1_affine* d_out, ace_stream stream);

/* Fixed-base batch k_i * G1 (resp. G2 generator) for canonical Fr scalars;
 * writes n affine points in out_form.  Used for setup and for MSM inputs. */
int ace_g1_fixed_base(ace_ctx* ctx, const ace_fr* d_scalars, size_t n, ace_g1_affine* d_out,
                      int out_form, ace_stream stream);
int ace_g2_fixed_base(ace_ctx* ctx, const ace_fr* d_scalars, size_t n, ace_g2_affine* d_out,
                      int out_form, ace_stream stream);

/* Groth16 proof for witness d_z (m canonical Fr, device) with prover
 * randomness r, s (host, canonical):
 *   A = [alpha]1 + sum z_j A_j + r [delta]1,  B = [beta]2 + sum z_j B2_j + s [delta]2,
 *   C = sum_{j>1} z_j L_j + sum h_i H_i + s A + r B1 - r s [delta]1,
 *   B1 = [beta]1 + sum z_j B1_j + s [delta]1.
 * proof_out (host, 256 bytes) as described above; the call synchronises.
 * The proof is taken to have the GPU to itself: a bucket reduction with
 * few enough segments runs on four lanes per segment (lower latency, more
 * instructions), which batched proofs do not use.  Same bytes either way.
 * ACE_E_UNSAT if (Az) o (Bz) != Cz (checked on the device). */
int ace_prove(ace_ctx* ctx, const ace_pk* pk, const ace_fr* d_z, const ace_fr* r, const ace_fr* s,
              uint8_t proof_out[256], ace_stream stream);
/* Same, but writes the 256 proof bytes to device memory d_proof_out and does
 * not synchronise (for graph capture and overlap). UNSAT is then reported by
 * the int at d_status (device): 0 ok, 1 unsat. */
int ace_prove_async(ace_ctx* ctx, const ace_pk* pk, const ace_fr* d_z, const ace_fr* r, const ace_fr* s,
                    uint8_t* d_proof_out, int32_t* d_status, ace_stream stream);

/* Prover randomness (r, s) drawn from seed (SplitMix64, purpose 5, zero rejected). */
int ace_rs_from_seed(uint64_t seed, ace_fr* r, ace_fr* s);

/* Groth16 verification on the host: 1 iff
 * e(A, B) = e(alpha1, beta2) e(ic[0] + sum x_j ic[j], gamma2) e(C, delta2)
 * (the three-pairing check of Section 3.3 / Section 3.4).  n_pub must be 1. */
int ace_verify(const ace_vk* vk, const ace_fr* pub, size_t n_pub, const uint8_t proof[256]);

/* Batch verification of k proofs of one verifying key (the validators'
 * check, Section 3.4 Algorithm 4, for many proofs at once): returns 1 iff
 *   prod_i e(rho_i A_i, B_i) e(-(sum rho_i) alpha1, beta2)
 *          e(-(sum rho_i)(ic[0] + ...) , gamma2) e(-(sum rho_i C_i), delta2) = 1
 * with IC folded as (sum rho_i) ic[0] + (sum rho_i x_i) ic[1], and every B_i
 * in the order-r subgroup; 0 if some proof is invalid (then at least one is,
 * except with probability about k 2^-128), negative on malformed input.
 * rho_i are 128-bit values drawn from SplitMix64(seed, purpose 12): a
 * verifier facing adversarial provers must pass a seed they cannot predict.
 * pubs: k public inputs (host, canonical); proofs: k x 256 bytes (host);
 * k <= 2^20 per call (about 1.5 KB of device scratch per proof).
 * The per-proof work (subgroup check, rho_i A_i, rho_i C_i, Miller loop) runs
 * on the device, the final exponentiation on the host. */
int ace_verify_batch(ace_ctx* ctx, const ace_vk* vk, size_t k, const ace_fr* pubs, const uint8_t* proofs,
                     uint64_t seed);

/* NTT of N = 2^log_n canonical Fr values in natural order, in place on the
 * device: the transforms of the QAP step of Groth16.Prove (Section 3.1,
 * Algorithm 1; H = {omega^i}, omega = 5^((r-1)/N), coset g H with g = 5).
 * The values must be canonical (below r): the passes transform them as they
 * are, with no conversion, and a larger value gives an undefined result.
 * Each pass picks its block width to fill the GPU's last wave of blocks.
 * kind: 0 forward (coefficients -> values on H), 1 inverse, 2 coset forward
 * (coefficients -> values on g H), 3 coset inverse.  1 <= log_n <= 28.
 * Scratch: N elements from the context. */
int ace_ntt(ace_ctx* ctx, ace_fr* d_data, uint32_t log_n, int kind, ace_stream stream);

/* The transform passes the QAP step is built from, without scaling: `count`
 * consecutive arrays of N Montgomery-form values, in place.  dif != 0:
 * natural -> bit-reversed order (decimation in frequency), else bit-reversed
 * -> natural (decimation in time); inverse != 0 uses omega^-1. */
int ace_ntt_mont(ace_ctx* ctx, ace_fr* d_data, uint32_t log_n, int count, int dif, int inverse,
                 ace_stream stream);

/* ace_msm_g1 with the window size forced to c (6 <= c <= 20), without the
 * GLV split (full-width scalars, K = ceil(255 / c) windows). */
int ace_msm_g1_window(ace_ctx* ctx, const ace_g1_affine* d_bases, int base_form, const ace_fr* d_scalars,
                      size_t n, int c, ace_g1_affine* d_out, ace_stream stream);
/* ace_msm_g1 (GLV split, K = ceil(128 / c) windows over 2n points) with the
 * window size forced to c (6 <= c <= 20); n < 2^30.  A diagnostic of this
 * library; the paper has no counterpart. */
int ace_msm_g1_glv_window(ace_ctx* ctx, const ace_g1_affine* d_bases, int base_form, const ace_fr* d_scalars,
                          size_t n, int c, ace_g1_affine* d_out, ace_stream stream);
/* ace_msm_g2 (scalars split four ways by psi, K = ceil(67 / c) windows over
 * 4n points) with the window size forced to c (6 <= c <= 20); n < 2^29.  A
 * diagnostic of this library; the paper has no counterpart. */
int ace_msm_g2_gls_window(ace_ctx* ctx, const ace_g2_affine* d_bases, int base_form, const ace_fr* d_scalars,
                          size_t n, int c, ace_g2_affine* d_out, ace_stream stream);

/* ---- diagnostics and measurement ------------------------------------------- */

/* Element-wise device arithmetic on canonical inputs, for unit-level checks.
 * field: 0 Fp, 1 Fr, 2 Fp2 (16 limbs per element); op: 0 a+b, 1 a-b, 2 a*b,
 * 3 a^2, 4 a^-1 (0 for a = 0).  n elements each. */
int ace_debug_field_op(int field, int op, const void* d_a, const void* d_b, void* d_out, size_t n,
                       ace_stream stream);
/* group: 1 G1, 2 G2 (affine canonical points); op: 0 P+Q, 1 P+Q mixed, 2 2P,
 * 3 k P with k from d_k (canonical 256-bit). */
int ace_debug_curve_op(int group, int op, const void* d_a, const void* d_b, const ace_fr* d_k, void* d_out,
                       size_t n, ace_stream stream);
/* Host: the library's optimal-ate pairing e(P, Q) after final exponentiation,
 * as 6 Fp2 coefficients (w^0, w^2, w^4, w^1, w^3, w^5), canonical. */
int ace_debug_pairing(const uint8_t g1[64], const uint8_t g2[128], uint8_t out[384]);
/* The same pairing by Miller-loop form 0 (affine, the single verifier's) or 1
 * (homogeneous projective, the loop the batch verifier runs on the device),
 * or form 2 (affine, with the final exponentiation's hard part by plain
 * square-and-multiply instead of the base-p joint exponentiation), computed
 * on the host. */
int ace_debug_pairing_form(int form, const uint8_t g1[64], const uint8_t g2[128], uint8_t out[384]);
/* Host: the GLV split the prover uses for s S_A + r S_B1: k = k1 + k2 lambda
 * (mod r), lambda = 0xb3c4d79d41a917585bfc41088d8daaa78b17ea66b99c90dd, a
 * cube root of unity with (beta x, y) = lambda (x, y) on G1.  out[0..3] = |k1|,
 * out[4] = 1 if k1 < 0, out[5..8] = |k2|, out[9] = 1 if k2 < 0 (|k_i| < 2^128). */
int ace_debug_glv_split(const ace_fr* k, uint32_t out[10]);
/* Host: the width-5 NAF the prover walks for each GLV half in s S_A + r S_B1:
 * out[i] (i < 132, least significant first) in {0, +-1, +-3, ..., +-15}
 * with sum_i out[i] 2^i = k, where k = k[0] + 2^32 k[1] + 2^64 k[2] + 2^96 k[3]
 * (below 2^128), and at most one non-zero digit in any five consecutive ones.
 * ACE_E_ARG for NULL pointers. */
int ace_debug_wnaf5(const uint32_t k[4], int8_t out[132]);
/* Host: the split ace_msm_g2 applies to each scalar, by the endomorphism
 * psi(x, y) = (conj(x) gx, conj(y) gy) of G2 (multiplication by
 * lambda = 6 x^2 on G2, x = 4965661367192848881 the BN parameter):
 * k = k0 + k1 lambda + k2 lambda^2 + k3 lambda^3 (mod r) with |k_i| < 2^66.
 * out[4 i .. 4 i + 2] = |k_i| (3 little-endian 32-bit limbs), out[4 i + 3] =
 * 1 if k_i < 0.  ACE_E_ARG for NULL pointers or k >= r. */
int ace_debug_gls_split(const ace_fr* k, uint32_t out[16]);
/* Host: the MSM plan the library picks for n points (no device call); a
 * diagnostic of this library, the paper has no counterpart.
 * kind: 0 full-width scalars without window tables (ace_msm_g1 for
 * n >= 2^30, ace_msm_g2 for n > 2^16), 1 window tables (proving-key
 * queries), 2 the GLV split of ace_msm_g1, 3 the four-way psi split of
 * ace_msm_g2.  force_c: 0 for the library's window (the cost model's; for
 * kind 3 a measured constant), else 6..20.
 * out: [c, K digit windows, buckets per window 2^(c-1), bucket windows + 1
 * (the {0,1} window), segment length L, segments per window M, virtual
 * buckets of the {0,1} window, points (2n for the GLV split, 4n for the psi
 * split, low 32 bits)].  ACE_E_ARG for a bad kind or force_c. */
int ace_debug_msm_plan(size_t n, int kind, int force_c, uint32_t out[8]);
/* Measured 32-bit multiply-add throughput of the device (operations/s):
 * mode 0 mad.lo, 1 mad.hi, 2 carry-chained lo/hi pairs, 3 mad.wide.u32
 * (one 32 x 32 -> 64-bit limb product with 64-bit accumulate per operation). */
int ace_debug_imad_rate(ace_ctx* ctx, int mode, double* ops_per_s);

/* Nanoseconds per step of a single-thread dependent chain: what = 0 Fp
 * Montgomery products, 1 G1 XYZZ additions (the latency that sequential
 * reductions and final combinations pay). */
int ace_debug_chain_latency(ace_ctx* ctx, int what, double* ns_per_step);

/* Montgomery products per second over all SMs and single-thread latency
 * (ns) of product form 0 (32-bit low/high multiply-add chains), form 1
 * (64-bit wide multiply-adds, one carry chain per row) or form 2 (plain 64-bit
 * products, two carry chains per row); digest: 4 words of output (optional)
 * for comparing the forms. */
int ace_debug_mul_rate(ace_ctx* ctx, int form, double* per_s, double* latency_ns, uint32_t* digest);

/* Kernel launches issued by the library in this process so far. */
int ace_launch_count(uint64_t* out);
/* Kernel timing: when enabled (and reset), the hot kernels are bracketed
 * with CUDA events on the stream they run on.  ace_profile_read synchronises
 * the device and returns, for one kind, the length of the union of the
 * bracketed intervals (ms), the launches and the work units:
 * kind 0 G1 bucket accumulation (units: mixed additions), 1 the same on G2,
 * 2 NTT passes (units: radix-2 butterflies), 3 sparse products (units:
 * non-zeros), 4 MSM digit sort (units: scalars), 5 MSM bucket reduction
 * (units: buckets), 6 proof-assembly scalar multiplications (units: launches).
 * A bracket of kinds 4 and 5 spans several kernels of one MSM. */
int ace_profile_enable(int on);
int ace_profile_read(int kind, double* ms, uint64_t* launches, uint64_t* units);
/* The total length of the same intervals (ms): launches that overlap one
 * another count once each, so sum_ms / launches is the average launch
 * duration. */
int ace_profile_read_sum(int kind, double* sum_ms);
/* Measurement mode (no counterpart in the paper): with on != 0, proofs made
 * on ctx afterwards run every stage on their slot's main stream in turn
 * instead of spreading the MSMs over auxiliary streams, so that the profiled
 * intervals of the stages do not overlap and add up to the proof's time.
 * The proof bytes do not change.  ACE_E_ARG for a NULL context. */
int ace_debug_serial_proofs(ace_ctx* ctx, int on);

/* ---- batching and serving ------------------------------------------------ */

/* k independent proofs in one call: the parallel map of the builder's
 * proving stage (Section 3.3, Algorithm 3 ParallelMap, which proves many
 * independent circuits at once), here over proofs of any mix of keys and
 * sizes.  pks[i] and d_zs[i] (device, pks[i]'s m canonical values, 16-byte
 * aligned) give proof i, rs[i] and ss[i] its randomness (host, canonical).
 * Proofs go round-robin over the context's proving slots (up to 16;
 * ace_autotune_batch_slots chooses their number and whether each proof's
 * MSMs spread over its slot's auxiliary streams or all its stages run on one
 * stream), so consecutive proofs overlap on the device.  When a call has
 * more proofs than slots, the fixed-base terms of all proofs run in one
 * launch beside the first MSMs and the variable-base terms and the assembly
 * in one launch each at the end; otherwise each proof finishes on its slot
 * as a lone proof does.  A call of one proof runs it as ace_prove does (its
 * MSMs on the auxiliary streams, latency-first reductions).  A call of at
 * least 8 proofs that all share one key
 * with N <= 2^18 runs instead on the batch-dimension kernels of
 * ace_prove_many (one launch per stage for all of them, the witnesses first
 * copied into one contiguous staging buffer held by the context).
 * Proof i goes to proofs + 256 i (host); status[i] (host) is 0, or 1 if
 * witness i does not satisfy its R1CS.  Synchronous.  ACE_E_ARG for NULL
 * pointers or non-canonical r, s; ACE_E_OOM if the slots' scratch cannot be
 * allocated.  Each proof equals the one ace_prove makes with the same inputs. */
int ace_prove_batch(ace_ctx* ctx, size_t k, const ace_pk* const* pks, const ace_fr* const* d_zs,
                    const ace_fr* rs, const ace_fr* ss, uint8_t* proofs, int32_t* status);
/* The same with the witnesses in HOST memory (h_zs[i]: pks[i]'s m canonical
 * values; page-locked memory lets the copies overlap the proving, pageable
 * memory works but the copy then blocks the calling thread).  Each witness
 * is copied into its proving slot's staging buffer (one per slot, sized for
 * the slot's largest witness, held by the context) once the slot's previous
 * proof is done, so a call moves exactly sum_i 32 m_i bytes to the device and
 * 256 k + 4 k bytes back.  Same results, status and errors as ace_prove_batch. */
int ace_prove_batch_host(ace_ctx* ctx, size_t k, const ace_pk* const* pks, const ace_fr* const* h_zs,
                         const ace_fr* rs, const ace_fr* ss, uint8_t* proofs, int32_t* status);

/* Proof server with continuous batching: block-proof jobs are proved as
 * they arrive (the builder loop of Section 3.3, Algorithm 3).  A job starts
 * as soon as one of `slots` proving slots is idle and the device memory it
 * needs (witness + scratch of its key's size) fits hbm_budget_bytes (0 = the
 * memory of `slots` jobs of max_pk's size); running jobs overlap on the
 * device.  A job not started within max_queue_wait_s (> 0) seconds of its
 * submission ends with ACE_E_TIMEOUT.  Slot scratch is sized for max_pk at
 * creation.  While the server exists, one server thread owns the context:
 * do not use the context from other threads (submit / poll / wait are
 * thread-safe).  Latency is measured from submission to proof bytes on the
 * host. */
int ace_server_create(ace_ctx* ctx, const ace_pk* max_pk, int slots, size_t hbm_budget_bytes,
                      double max_queue_wait_s, ace_server** out);
/* Queue one proof of witness z_host (host, m canonical Fr; pinned memory
 * recommended; must stay valid until the job's result is collected) under
 * key pk (m <= max_pk's m) with randomness r, s. */
int ace_server_submit(ace_server* srv, const ace_pk* pk, const ace_fr* z_host, const ace_fr* r, const ace_fr* s,
                      uint64_t* job_id);
/* ACE_E_BUSY while the job runs; otherwise its result (ACE_OK with the 256
 * proof bytes, ACE_E_UNSAT, ACE_E_TIMEOUT, ...) and latency in ms, after
 * which the job id is released. */
int ace_server_poll(ace_server* srv, uint64_t job_id, uint8_t proof_out[256], double* latency_ms);
/* Like ace_server_poll but blocks up to timeout_s (<= 0: no limit);
 * ACE_E_BUSY if the job is still running when the time is up. */
int ace_server_wait(ace_server* srv, uint64_t job_id, uint8_t proof_out[256], double* latency_ms, double timeout_s);
/* submitted, collected, timeouts, waiting, peak running jobs, peak admitted
 * device bytes, budget, slots */
int ace_server_stats(ace_server* srv, uint64_t out[8]);
/* Finishes the jobs already submitted, then stops the server thread. */
int ace_server_destroy(ace_server* srv);
/* Host-only check of the server's admission logic on a virtual clock: jobs
 * with the given arrival time, run time and memory on `slots` slots and a
 * memory budget; returns each job's start / finish time and status (0, -2
 * never fits, -6 timed out) and peaks[0] = most jobs running at once,
 * peaks[1] = most memory admitted at once; prio_out (optional): each job's
 * stream-priority level (jobs already running when it started). */
int ace_debug_scheduler_sim(int slots, size_t budget, size_t n, const double* arrival, const double* duration,
                            const size_t* mem, double max_wait, double* start_out, double* finish_out,
                            int32_t* status_out, uint64_t* peaks, int32_t* prio_out);

/* Witnesses of k instances of circuit c on the device, instance q from input
 * seed seeds[q] (host array): the same values, in the same order, as
 * ace_witness(c, seeds[q]) (the w_tx each transaction's proof starts from,
 * Section 3.3, Algorithm 3).  d_z: k x m canonical values (device, caller
 * owned), laid out as ace_prove_many expects.  The R1CS is not checked here
 * (the provers check it and report it per proof).  Synchronises `stream`.
 * Scratch: the circuit's constants and k x 3 n_perm draw positions. */
int ace_witness_many(ace_ctx* ctx, const ace_circuit* c, size_t k, const uint64_t* seeds, ace_fr* d_z,
                     ace_stream stream);

/* Many proofs of ONE key in one pass: the per-transaction proofs of a block
 * (every transaction proves the same circuit; Section 3.3, Algorithm 3
 * ParallelMap over the block's transactions).  Every stage runs once for
 * all k proofs (one sparse-product launch, NTT launches over 3k arrays, MSMs
 * whose k bucket sets share the key's point tables), in chunks that keep the
 * scratch within 24 GB (the environment variable ACE_MANY_MAX_CHUNK caps the
 * proofs per chunk further).  d_z: k witnesses of pk's m values each, contiguous
 * (k x m ace_fr, canonical, 16-byte aligned, device); rs, ss: k canonical
 * values each (host); proofs (host, k x 256 bytes) and status (host, k: 0 ok,
 * 1 the witness does not satisfy the R1CS).  Synchronous; each proof equals
 * the one ace_prove makes with the same (z, r, s). */
int ace_prove_many(ace_ctx* ctx, const ace_pk* pk, size_t k, const ace_fr* d_z, const ace_fr* rs, const ace_fr* ss,
                   uint8_t* proofs, int32_t* status);

/* ---- autotuning ------------------------------------------------------------ */

/* Measure candidate MSM window sizes c for the generic G1 MSM at
 * n = 2^log_min .. 2^log_max (6 <= log_min <= log_max <= 24) on synthetic
 * inputs and keep the fastest per size in the context (ace_msm_g1 then uses
 * it).  report (optional, 5 doubles per size): log_n, chosen c, its ms,
 * cost-model c, its ms. */
int ace_autotune_msm(ace_ctx* ctx, uint32_t log_min, uint32_t log_max, double* report);
/* Measure the NTT pass width (2^10, 2^11 or 2^12 elements per block in shared
 * memory) and stage form (radix-2 stages, or stages in radix-4 pairs) for
 * N = 2^log_min .. 2^log_max (8..24) on three arrays and keep the fastest
 * pair per size.  report (optional, 5 per size): log_n, chosen width, its
 * ms, ms at width 2^11 with the untuned form, chosen radix (2 or 4). */
int ace_autotune_ntt(ace_ctx* ctx, uint32_t log_min, uint32_t log_max, double* report);
/* Time batches of k proofs of (pk, d_z) over 1..max_slots proving slots, in
 * two stage layouts (a proof's MSMs spread over its slot's auxiliary
 * streams, or every stage of a proof on one stream with proofs overlapping
 * across slots only), and keep for ace_prove_batch, among the configurations
 * within 1% of the fastest, the one-stream layout first and then the fewest
 * slots (fewer kernels share the SMs and fewer slots hold scratch, at the same
 * throughput).  The proofs do not change.  1 <= max_slots <= 16 (ACE_E_ARG
 * otherwise).  report (optional, 2 x max_slots doubles): ms per batch for
 * 1..max_slots slots with the auxiliary streams, then the same with one
 * stream per proof. */
int ace_autotune_batch_slots(ace_ctx* ctx, const ace_pk* pk, const ace_fr* d_z, int k, int max_slots,
                             double* report);
/* Save / load the tuned choices (JSON keyed by the GPU name; loading a file
 * tuned on another GPU fails with ACE_E_ARG and changes nothing). */
int ace_autotune_save(ace_ctx* ctx, const char* path);
int ace_autotune_load(ace_ctx* ctx, const char* path);

/* ---- persistence ---------------------------------------------------------- */

/* Save / load a proving key (with its circuit) to a versioned file.  A
 * library service with no counterpart in the paper, which requires a
 * circuit-specific trusted setup (Section 9, "Trusted setup") and says
 * nothing about storing its output: the file holds a header (magic,
 * format version), the circuit, window 0 of every query table and the fixed
 * points; loading checks the header and sizes, rebuilds the window tables on
 * the device and returns the key (pk_out, lib-owned, free with ace_pk_free)
 * and its verifying key (vk_out, caller-owned, optional).  ACE_E_ARG for a
 * missing, truncated or mismatched file; ACE_E_OOM if the key does not fit. */
int ace_pk_save(const ace_pk* pk, const char* path);
int ace_pk_load(ace_ctx* ctx, const char* path, ace_pk** pk_out, ace_vk* vk_out);

#ifdef __cplusplus
}
#endif
#endif /* ACE_H */
