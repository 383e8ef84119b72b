/*
 * zkvc.h -- C ABI of a GB300 (sm_103a) prover for zkVC's CRPC matrix-multiplication
 * circuit under Groth16 over BN254.
 *
 * zkVC ("zkVC: Fast Zero-Knowledge Proof for Private and Verifiable Computing",
 * arXiv 2504.12217) proves Y = X W with the Constraint-reduced Polynomial Circuit (CRPC,
 * Sec. III-A) and Prefix-Sum Query (PSQ, Sec. III-B), and runs Groth16 Gen / Prove /
 * Verify (Sec. II) as its zkVC-G backend (Sec. IV).  This library exposes that problem
 * statement (setup / prove / verify on a matmul shape) and the kernels underneath it.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Field elements cross the ABI in canonical (non-Montgomery) form: 32 bytes,
 *    little-endian, value < modulus.  Fr is the BN254 scalar field (order r), Fp the base
 *    field (modulus p).
 *  - G1 points are affine x || y (64 bytes); G2 points are x.c0 || x.c1 || y.c0 || y.c1
 *    (128 bytes) with Fp2 = Fp[i]/(i^2 + 1).  The point at infinity is all zero bytes.
 *  - "d_" pointers are CUDA device pointers owned by the caller; other pointers are host
 *    pointers owned by the caller.  Handles (zkvc_pk, zkvc_vk) are owned by the library.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Unless a
 *    function says it synchronises, work is only enqueued on `stream`.
 *  - Every function returns ZKVC_OK (0) or a negative status; zkvc_last_error() then
 *    describes the failure (thread-local, valid until the next call on that thread).
 *  - Workspaces are caller-provided device buffers of at least the size the matching
 *    *_workspace_bytes() function reports; the library never allocates inside a call
 *    that takes a workspace, except for a per-device domain table built once on first
 *    use of each NTT size (so warm up before capturing such a call in a CUDA graph).
 */
#ifndef ZKVC_H_
#define ZKVC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define ZKVC_OK 0
#define ZKVC_EINVAL (-1)   /* bad argument: shape, size, pointer, encoding              */
#define ZKVC_ENOMEM (-2)   /* a device or host allocation failed                        */
#define ZKVC_ECUDA (-3)    /* a CUDA runtime call failed                                 */
#define ZKVC_ETIMEOUT (-4) /* a bounded device-side wait ran out                         */
#define ZKVC_EUNSAT (-5)   /* the witness does not satisfy the CRPC constraints          */
#define ZKVC_EIO (-6)      /* serialisation: short buffer, bad header or checksum        */

/* Description of the last failure on the calling thread ("" after success). */
const char* zkvc_last_error(void);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int zkvc_version(void);

/* Number of CUDA kernels the library has launched in this process so far (all devices,
 * all threads); a diagnostic for launch-count accounting. */
uint64_t zkvc_kernel_launches(void);

/* Stage timers for the prover: when enabled, zkvc_prove records CUDA events on the
 * streams of its stages and accumulates their elapsed times after its final
 * synchronisation.  Stages 0..7: witness, ntt, msm_g1 (the H-query MSM),
 * msm_g1_bucket_accum (its accumulation kernel), msm_g2 (with the encoding of B),
 * msm_g2_bucket_accum, combine (the encoding of C after the joins), msm_g1_small (the
 * small-digit G1 run with what follows it on its stream: the chain-mode scalar
 * multiplications or the encoding of A).  The two bucket_accum stages time the
 * bucket-accumulation kernel alone and count its units (bucket terms, one mixed point
 * addition each).  zkvc_profile_span gives a stage's mean begin and end offsets (ms) from
 * the begin of the witness stage of the same proof: the proof's timeline across its
 * streams.  Enabling resets the counters.  A single-threaded diagnostic: not for
 * concurrent provers.  Out-of-range stages return ZKVC_EINVAL.
 */
void zkvc_profile_enable(int on);
int zkvc_profile_read(int stage, const char** name, double* ms, uint64_t* calls, uint64_t* units);
int zkvc_profile_span(int stage, double* start_ms, double* end_ms);

/* Integer-pipe throughput microbenchmark: the measured peak of the 32-bit multiply-add
 * (IMAD) that every Montgomery product of the prover is made of (BN254 field arithmetic
 * of the groth16 backend, Sec. IV; the roofline denominator of the MSM and NTT kernels).
 * A 32 x 32 -> 64-bit product counts as two IMADs (its low and high words), as in the
 * 264 of a CIOS product.  form 0: sixteen independent mad.lo.u32 chains per thread;
 * 1: the CIOS row of the field code (a carry chain of eight mad.lo and eight mad.hi);
 * 2: sixteen independent mad.hi.u32 chains; 3: eight independent mad.wide.u32 chains
 * (64-bit accumulators); 4: two carry chains of eight mad.lo; 5 to 8: two independent
 * chains of whole Fp Montgomery products per thread (264 IMADs each): 5 CIOS with
 * carry-chain rows, 6 CIOS with 64-bit accumulators, 7 product scanning with 96-bit
 * column accumulators in mad.lo.cc / madc.hi.cc (the product the kernels use), 8 the same
 * with mul.wide and additions; 9 and 10: latency, one warp running one dependent chain
 * of products per thread (9: the kernels' product, 10: the 64-bit-accumulator CIOS); each
 * checked against the CIOS product on every thread (ZKVC_ECUDA if any result differs).  A full-occupancy grid over every SM runs `iters` iterations (16 IMADs per
 * thread for forms 0 .. 4), once untimed (iters / 8) and once timed with CUDA events on
 * `stream`; the call synchronises.  Outputs (any may be null): IMADs per second, the
 * timed launch in ms and the SM count used.  ZKVC_EINVAL for a form outside 0 .. 10 or
 * iters outside [1, 2^24].
 */
int zkvc_imad_rate(int form, uint32_t iters, double* imad_per_s, double* ms, int* sms, void* stream);

/* ------------------------------------------------------------------ field kernels
 * Elementwise products of n canonical elements: d_out[i] = d_a[i] * d_b[i] mod the
 * field's modulus (Fr: scalar field r; Fp: base field p; Fp2: pairs c0 || c1, 64 bytes
 * per element, with i^2 = -1).  Inputs must be canonical.  d_out may alias d_a or d_b.
 * These are the Montgomery multiplication kernels of the prover (BN254 arithmetic of the
 * groth16 backend, Sec. IV) exposed for verification.
 */
int zkvc_fr_mul(const uint8_t* d_a, const uint8_t* d_b, uint8_t* d_out, size_t n, void* stream);
int zkvc_fp_mul(const uint8_t* d_a, const uint8_t* d_b, uint8_t* d_out, size_t n, void* stream);
int zkvc_fp2_mul(const uint8_t* d_a, const uint8_t* d_b, uint8_t* d_out, size_t n, void* stream);

/* Elementwise inverses d_out[i] = d_a[i]^-1 mod r (fr) or mod p (fp), 0 -> 0, for n
 * canonical 32-byte little-endian elements in device memory; d_out may alias d_a.  The
 * inversion of the prover's affine conversions (the Groth16 proof encodes A, B and C in
 * affine coordinates, Sec. II): a binary GCD that takes 30 steps at a time on 62-bit
 * stand-ins of the operands (17 rounds).  Returns ZKVC_EINVAL on a null pointer with n > 0.
 */
int zkvc_fr_inv(const uint8_t* d_a, uint8_t* d_out, size_t n, void* stream);
int zkvc_fp_inv(const uint8_t* d_a, uint8_t* d_out, size_t n, void* stream);

/* The host-side GLV split of the chain-mode scalar multiplications (G1 of BN254 has the
 * endomorphism phi(x, y) = (beta x, y) = lambda (x, y)): k (32 bytes little-endian,
 * k < r) = k1 + k2 lambda (mod r) with |k1|, |k2| < 2^127, by rounding against a short
 * basis of the lattice {(x, y) : x + y lambda = 0 mod r} (Gallant, Lambert, Vanstone).
 * out: |k1| (16 bytes little-endian), sign of k1 (1 byte: 1 = negative), then |k2| and
 * its sign (34 bytes).  Host only; ZKVC_EINVAL on a null pointer.
 */
int zkvc_glv_split(const uint8_t k[32], uint8_t out[34]);

/* ------------------------------------------------------------------ witness matmul
 * Y = X W for int8 X (a x n, row-major) and W (n x b, row-major) into int32 Y (a x b,
 * row-major), exactly -- the matrix product whose correctness zkVC proves (Sec. II) and
 * the first step of the prover's witness.  It runs on the tensor cores (tcgen05, bf16
 * operands, fp32 accumulation in passes of 256 products, each pass exact) and returns
 * when Y is written (synchronises `stream`).  All pointers are device memory owned by
 * the caller.  ZKVC_EINVAL for a null pointer or a shape below 1; ZKVC_ETIMEOUT if a
 * tensor-core wait ran out (Y is then not written).
 */
int zkvc_matmul_i8(const int8_t* d_X, const int8_t* d_W, int32_t* d_Y, int a, int n, int b, void* stream);

/* ------------------------------------------------------------------ NTT over Fr
 * In-place transform of N = 2^log_n canonical Fr elements in natural order
 * (1 <= log_n <= 28), over the domain H = <omega_N>, omega_N = 5^((r-1)/2^28)^(2^28/N),
 * and the coset gH with g = 5 -- the domain on which the QAP of the CRPC R1CS is
 * interpolated (Sec. II) and whose coset carries the quotient h(x):
 *   ZKVC_NTT_FORWARD        v_k = sum_i a_i omega^(ik)
 *   ZKVC_NTT_INVERSE        a_i = N^-1 sum_k v_k omega^(-ik)
 *   ZKVC_NTT_COSET_FORWARD  v_k = sum_i a_i g^i omega^(ik)
 *   ZKVC_NTT_COSET_INVERSE  a_i = g^-i N^-1 sum_k v_k omega^(-ik)
 * No workspace; the first call for a given log_n on a device builds and caches that
 * domain's tables (allocates and synchronises).
 */
#define ZKVC_NTT_FORWARD 0
#define ZKVC_NTT_INVERSE 1
#define ZKVC_NTT_COSET_FORWARD 2
#define ZKVC_NTT_COSET_INVERSE 3
int zkvc_ntt(uint8_t* d_data, uint32_t log_n, int kind, void* stream);

/* ------------------------------------------------------------------ MSM
 * Variable-base multi-scalar multiplication out = sum_i s_i P_i (Pippenger, signed
 * c-bit windows, bucket sort and parallel reduction) -- the kernel behind the A, B, L
 * and H queries of Groth16 Prove (Sec. II).
 *   d_points   n affine points (64 bytes each for G1, 128 for G2), canonical, on the curve
 *              (not checked); infinity allowed, as all-zero bytes
 *   d_scalars  n scalars, 32-byte little-endian integers; values at or above r are
 *              reduced mod r (an endomorphism split follows in both groups: GLV with
 *              phi(x, y) = (beta x, y) on G1, psi on G2, halves below 2^127)
 *   d_ws       device workspace of zkvc_msm_workspace_bytes(n, group) bytes
 *   out        host buffer of 64 (G1) or 128 (G2) bytes; the call synchronises `stream`
 * group = 1 for G1, 2 for G2.  n may be 0 (out = infinity); n above ZKVC_MSM_MAX_POINTS
 * returns ZKVC_EINVAL (there the 2n split scalars take eight 16-bit windows each: 16 n
 * digits, whose 32-bit term indices must stay at or below 2^31), and
 * zkvc_msm_workspace_bytes returns 0 for it.
 */
#define ZKVC_MSM_MAX_POINTS (1u << 27)
size_t zkvc_msm_workspace_bytes(size_t n, int group);
int zkvc_msm_g1(const uint8_t* d_points, const uint8_t* d_scalars, size_t n, void* d_ws, size_t ws_bytes,
                uint8_t out[64], void* stream);
int zkvc_msm_g2(const uint8_t* d_points, const uint8_t* d_scalars, size_t n, void* d_ws, size_t ws_bytes,
                uint8_t out[128], void* stream);

/* Fixed-base multiplication of the group generators: d_points[i] = [k_i] G for n
 * canonical Fr scalars (device), written as canonical affine points (64 bytes for G1,
 * 128 for G2).  The comb of 32 byte-windows that Gen (Sec. II) uses to build proving
 * keys, exposed for callers that need many generator multiples.  Workspace:
 * zkvc_generator_mul_workspace_bytes(n, group).  The first call on a device builds and
 * caches the comb tables (allocates and synchronises).
 */
size_t zkvc_generator_mul_workspace_bytes(size_t n, int group);
int zkvc_g1_generator_mul(const uint8_t* d_scalars, size_t n, uint8_t* d_points, void* d_ws, size_t ws_bytes,
                          void* stream);
int zkvc_g2_generator_mul(const uint8_t* d_scalars, size_t n, uint8_t* d_points, void* d_ws, size_t ws_bytes,
                          void* stream);

/* Allocation-free variant of zkvc_msm_g1, for callers that cannot allocate device memory
 * (runtimes without a device allocator, or processes whose device memory another
 * framework reserved up front for its own pool).  The paper has no counterpart; it is a
 * deployment convenience of this library.
 *   - Same arguments and result as zkvc_msm_g1, minus the workspace: the scratch is one
 *     8 MiB array in device memory, part of the library image, held on every GPU that
 *     loads the library until the process exits.
 *   - n <= ZKVC_MSM_NOALLOC_MAX_POINTS; larger n returns ZKVC_EINVAL.
 *   - Calls no allocator (CUDA's or any framework's).  Like zkvc_msm_g1 it uploads its
 *     bucket tables from host memory, synchronises `stream` and copies the result to
 *     `out` (host memory) before it returns.
 *   - The first call on a device (with that device current) looks up the array's device
 *     address and caches it per device and CUDA context; make that first call before any
 *     stream capture.
 *   - All calls share the array, which keeps the previous call's contents (each call
 *     initialises what it reads).  Calls whose GPU work overlaps race on it: issue them
 *     one at a time.
 */
#define ZKVC_MSM_NOALLOC_MAX_POINTS 4096
int zkvc_msm_g1_noalloc(const uint8_t* d_points, const uint8_t* d_scalars, size_t n, uint8_t out[64], void* stream);

/* ------------------------------------------------------------------ Groth16 over CRPC
 * The circuit (Sec. III-A general CRPC equation with Sec. III-B prefix sums) for
 * Y = X W, X of a x n and W of n x b (int8), has n multiplication constraints
 *     row k < n-1:  a_k b_k = S_k - S_(k-1)        (S_(-1) = 0)
 *     row n-1:      a_(n-1) b_(n-1) = Y(z) - S_(n-2)
 * with a_k = sum_i z^(ib) x_ik, b_k = sum_j z^j w_kj, Y(z) = sum_ij z^(ib+j) y_ij, plus
 * l + 1 public-input rows (A = [variable v], v = 0 .. l).  Variables: 0 = one, then X
 * row-major and Y row-major (public, l = a n + a b), then W row-major and S_0 .. S_(n-2)
 * (private).  Integers enter Fr as v >= 0 -> v, v < 0 -> r - |v|.  The QAP domain has
 * N = 2^ceil(log2(n + l + 1)) points.
 */
typedef struct zkvc_pk zkvc_pk; /* proving key: resident on the device that built it */
typedef struct zkvc_vk zkvc_vk; /* verifying key: host memory                         */

/* Gen (Sec. II).  toxic = tau || alpha || beta || gamma || delta || z, six canonical Fr
 * values (192 bytes, host); z is the CRPC evaluation point of Sec. III-A.  Rejected with
 * ZKVC_EINVAL: non-canonical values, tau^N = 1, alpha..delta = 0, z in {0, 1}.  Allocates
 * the key on the current device, synchronises `stream`, and returns library-owned
 * handles (release with zkvc_pk_free / zkvc_vk_free).
 */
int zkvc_setup(int a, int n, int b, const uint8_t toxic[192], void* stream, zkvc_pk** pk, zkvc_vk** vk);
void zkvc_pk_free(zkvc_pk* pk);
void zkvc_vk_free(zkvc_vk* vk);

/* Shape of a proving key, its domain size log2 N and its stored base counts. */
int zkvc_pk_info(const zkvc_pk* pk, int* a, int* n, int* b, uint32_t* log_domain, size_t* g1_bases,
                 size_t* g2_bases);

/* Copies proving-key entries [start, start + count) of one query to host memory as
 * canonical affine encodings (64 bytes for G1, 128 for G2), in variable order:
 *   ZKVC_Q_A   [A_v(tau)]1, v = 0 .. l          ZKVC_Q_B1 / B2  [B_v(tau)]1,2 for W
 *   ZKVC_Q_L   [(beta A + alpha B + C)_v(tau)/delta]1, W variables then S variables
 *   ZKVC_Q_H   [tau^j t(tau)/delta]1, j = 0 .. N-2
 *   ZKVC_Q_ALPHA1 .. ZKVC_Q_DELTA2  the single points [alpha]1, [beta]1, [beta]2,
 *                                   [delta]1, [delta]2 (start = 0, count = 1)
 * Synchronises the device.  Make the key's device current first.
 */
#define ZKVC_Q_A 0
#define ZKVC_Q_B1 1
#define ZKVC_Q_B2 2
#define ZKVC_Q_L 3
#define ZKVC_Q_H 4
#define ZKVC_Q_ALPHA1 5
#define ZKVC_Q_BETA1 6
#define ZKVC_Q_BETA2 7
#define ZKVC_Q_DELTA1 8
#define ZKVC_Q_DELTA2 9
int zkvc_pk_export(const zkvc_pk* pk, int query, size_t start, size_t count, uint8_t* out);

/* Verifying-key entries: IC_v = [(beta A + alpha B + C)_v(tau)/gamma]1 (v = 0 .. l) and
 * the points [alpha]1, [beta]2, [gamma]2, [delta]2.  Host copy, no device work.
 */
int zkvc_vk_info(const zkvc_vk* vk, int* a, int* n, int* b);
#define ZKVC_VK_IC 0
#define ZKVC_VK_ALPHA1 1
#define ZKVC_VK_BETA2 2
#define ZKVC_VK_GAMMA2 3
#define ZKVC_VK_DELTA2 4
int zkvc_vk_export(const zkvc_vk* vk, int query, size_t start, size_t count, uint8_t* out);

/* Builds a verifying key for shape (a, n, b) from canonical encodings (host memory,
 * copied): [alpha]1, [beta]2, [gamma]2, [delta]2 and IC_0 .. IC_l (n_ic = l + 1 points of
 * 64 bytes).  No device work.  Release with zkvc_vk_free.
 */
int zkvc_vk_import(int a, int n, int b, const uint8_t alpha1[64], const uint8_t beta2[128], const uint8_t gamma2[128],
                   const uint8_t delta2[128], const uint8_t* ic, size_t n_ic, zkvc_vk** vk);

/* Verify (Sec. II): decides e(A, B) = e(alpha, beta) e(IC(x), gamma) e(C, delta) with the
 * public input x = X (a x n int8, row-major) then Y (a x b int32, row-major), host
 * pointers.  Runs on the host (optimal-ate pairing over BN254), no device work.
 * Returns ZKVC_OK with *ok = 1 for a valid proof and *ok = 0 otherwise -- including
 * proofs whose points are not canonical, not on the curve, or (B) not in the order-r
 * subgroup.  ZKVC_EIO for a malformed key.  With a key of no public inputs
 * (ZKVC_PUBLIC_NONE) X and Y are not read and may be NULL.
 */
int zkvc_verify(const zkvc_vk* vk, const int8_t* X, const int32_t* Y, const uint8_t proof[256], int* ok);

/* Verification on the GPU, batched (Sec. II: Verify).  Proof i is checked against
 * verifying key vks[i] (keys may repeat) with its public inputs X[i] (a x n int8) and Y[i]
 * (a x b int32), host pointers (ignored for keys without public inputs; X and Y may then
 * be NULL).  proofs: count x 256 bytes (host).  ok[i] (host) receives 1 for a valid proof
 * and 0 otherwise, with the host verifier's rules: canonical coordinates, points on their
 * curves, B in the order-r subgroup, and the pairing equation.  IC(x) of all proofs is one
 * merged GPU MSM; each proof's four Miller loops and final exponentiation run on the GPU.
 * Allocates temporary device memory, waits for the result (bounded by
 * zkvc_set_wait_timeout_ms).  ZKVC_EIO for a malformed key.
 *
 * zkvc_pairing: e(P_i, Q_i) for n canonical G1 points (d_P, n x 64 bytes) and G2 points
 * (d_Q, n x 128), device pointers; d_out receives n x 384 bytes, 12 canonical Fp values per
 * pairing in the tower basis Fp12 = Fp6[w]/(w^2 - v), Fp6 = Fp2[v]/(v^3 - (9 + i)):
 * (c0.c0, c0.c1, c0.c2, c1.c0, c1.c1, c1.c2), each Fp2 element as c0 then c1.  Exposed for
 * verification of the pairing itself; enqueued on `stream` only.
 */
int zkvc_verify_batch(const zkvc_vk* const* vks, const int8_t* const* X, const int32_t* const* Y, const uint8_t* proofs,
                      int count, int* ok, void* stream);
int zkvc_pairing(const uint8_t* d_P, const uint8_t* d_Q, size_t n, uint8_t* d_out, void* stream);

/* Key files: a versioned header (magic, version, shape, counts), the payload, and an
 * FNV-1a-64 checksum of the payload.  pk files hold the device representation of this
 * library version (Montgomery-form bases with their precomputed windows) so that a key
 * built once by zkvc_setup can be reloaded instead of recomputed; vk files hold the
 * canonical encodings.  zkvc_pk_load allocates the key on the current device and
 * synchronises; ZKVC_EIO for a missing, truncated, corrupt or mismatched file.
 */
int zkvc_pk_save(const zkvc_pk* pk, const char* path);
int zkvc_pk_load(const char* path, void* stream, zkvc_pk** pk);
int zkvc_vk_save(const zkvc_vk* vk, const char* path);
int zkvc_vk_load(const char* path, zkvc_vk** vk);

/* Prove (Sec. II) for the key's shape.
 *   d_X   a x n int8, row-major (device)          d_W  n x b int8, row-major (device)
 *   rs    r || s, two canonical Fr values (64 bytes, host): the prover's randomness
 *   d_Y   a x b int32 output (device): receives Y = X W, the proven product
 *   d_ws  device workspace of zkvc_prove_workspace_bytes(pk) bytes
 *   proof 256-byte host output: A (G1, 64) || B (G2, 128) || C (G1, 64), canonical affine
 * Synchronises `stream`.  ZKVC_EUNSAT if the device-side checks find the witness does
 * not satisfy the constraints (the PSQ chain must close against Y(z) and h must have
 * degree < N - 1).  The proof is a deterministic function of (pk, X, W, r, s).
 * When a key is proven twice in a row with the same d_X, d_W, d_Y, d_ws, mode and
 * tuning, the second call captures the proof's launch sequence as a CUDA graph (kept with
 * the key, freed by zkvc_pk_free) and later calls with those buffers replay it; other
 * calls, and every call while the stage timers are on, enqueue directly.  The bytes are
 * the same either way.
 */
size_t zkvc_prove_workspace_bytes(const zkvc_pk* pk);
int zkvc_prove(const zkvc_pk* pk, const int8_t* d_X, const int8_t* d_W, const uint8_t rs[64], int32_t* d_Y,
               void* d_ws, size_t ws_bytes, uint8_t proof[256], void* stream);

/* The same proof computed two ways (identical bytes).  Groth16's C holds s A + r B1 - r s
 * [delta]1 (Sec. II), which needs A and B1 first.
 *   ZKVC_PROVE_FOLD   (zkvc_prove's mode unless tuning chose chain) expands s A and r B1 by linearity into
 *                     fixed-base terms sum (s w_v) [A_v]1 + sum (r w_e) [B_e]1 + ..., so
 *                     no serial doubling chain remains: lowest latency for one proof,
 *                     but 16 signed digits per witness entry instead of one.
 *   ZKVC_PROVE_CHAIN  computes A and B1 with small-scalar MSMs and then s A and r B1 as
 *                     two variable-base multiplications beside the H MSM (the scalars
 *                     split by the GLV endomorphism, four 127-bit halves on four lane
 *                     quads): about 2.5x less MSM work per proof, so more proofs per
 *                     second when several proofs share the GPU.
 * Workspace sizes differ per mode.  zkvc_prove uses the key's mode (tuning value 6),
 * ZKVC_PROVE_FOLD unless zkvc_pk_autotune or zkvc_pk_set_tuning chose chain, and
 * zkvc_prove_workspace_bytes follows it. */
/* Latency tuning of the one-proof prover for a key: zkvc_pk_autotune times whole proofs
 * of the given inputs (device X, W; host rs) in `mode` while it varies the launch shape
 * -- ZKVC_PK_TUNING_LEN values: the terms per level-0 chunk of each MSM run (small-scalar
 * G1, rest G1, H, G2; 0 = the default rule: about two chunks per bucket, at least 16 terms
 * and about 40 k chunks), log2 of the NTT elements per block (8..11; 0 = 10), when the side MSM starts (the
 * full-scalar "rest" MSM in fold mode, the small-digit MSM in chain mode: 0 at once, 1
 * after the NTTs, 2 after the H MSM's bucket accumulation), the mode zkvc_prove uses
 * (ZKVC_PROVE_FOLD or ZKVC_PROVE_CHAIN), when the G2 MSM starts (0, 1), and whether the H
 * and the small-digit runs accumulate on quads of lanes (0, 1) --
 * keeps the fastest in the key and writes it to tuning (may be NULL): a joint grid over
 * the small-digit and G2 chunks first, then two sweeps of coordinate descent over all
 * values, then the four fastest settings seen timed twice more (the lowest mean of three
 * wins).  Each timing is the median of nine proofs, each started after a 256 MiB write (a
 * cold L2, as for a proof of fresh inputs).  `mode` is the mode to tune, or ZKVC_PROVE_AUTO to tune both and keep
 * the faster.  It allocates and frees its own workspace and the 256 MiB buffer and
 * synchronises `stream`; the key must not be proving meanwhile.
 * Afterwards zkvc_prove_workspace_bytes reflects the chosen chunks (smaller chunks need
 * more workspace).  zkvc_pk_set_tuning / zkvc_pk_get_tuning impose or read the setting
 * (ZKVC_EINVAL for a chunk above 1024, an NTT block outside 2^8..2^11, a start outside
 * its range or a mode other than fold or chain).  Proof bytes
 * never depend on it.  Keys of zkvc_setup only.
 * Tuning cache: every result is also stored in a process-wide cache keyed by the shape
 * (a, n, b), the requested mode, the GPU's name and its SM count; zkvc_pk_autotune on a
 * key with a cached entry applies it without timing (and returns it in tuning), unless
 * `mode` carries ZKVC_TUNE_FRESH.  zkvc_tune_cache_save / zkvc_tune_cache_load write and
 * merge a text file of entries (ZKVC_EIO for an unreadable or malformed file, which then
 * changes nothing; entries are validated as zkvc_pk_set_tuning validates a setting);
 * zkvc_tune_cache_clear empties the cache.  Host only, thread-safe. */
#define ZKVC_PK_TUNING_LEN 10
#define ZKVC_TUNE_FRESH 0x10 /* zkvc_pk_autotune: ignore the tuning cache, tune again */
int zkvc_pk_autotune(zkvc_pk* pk, int mode, const int8_t* d_X, const int8_t* d_W, const uint8_t rs[64], void* stream,
                     uint32_t tuning[ZKVC_PK_TUNING_LEN]);
int zkvc_pk_set_tuning(zkvc_pk* pk, const uint32_t tuning[ZKVC_PK_TUNING_LEN]);
int zkvc_pk_get_tuning(const zkvc_pk* pk, uint32_t tuning[ZKVC_PK_TUNING_LEN]);
int zkvc_tune_cache_save(const char* path);
int zkvc_tune_cache_load(const char* path);
int zkvc_tune_cache_clear(void);

#define ZKVC_PROVE_FOLD 0
#define ZKVC_PROVE_CHAIN 1
#define ZKVC_PROVE_AUTO 2 /* zkvc_pk_autotune only: tune both modes, keep the faster */
size_t zkvc_prove_workspace_bytes_mode(const zkvc_pk* pk, int mode);
/* Proof of a claimed product: the statement of zkVC's use case (Sec. I; Gen / Prove of
 * Sec. II) in which a server claims Y = X W and proves it.  Like zkvc_prove, but Y is an
 * input: dY_claimed (int32, a x b, row-major, device, read only) enters the witness as it
 * is, nothing computes X W.  If it is not X W the constraints cannot all hold: the call
 * returns ZKVC_EUNSAT (the PSQ chain does not close against Y(z), or, for circuits
 * without it, the quotient has degree N - 1) and the proof bytes are meaningless.  Works
 * with keys of zkvc_setup (in the key's tuned mode, enqueued directly, never from the
 * captured graph) and of zkvc_setup_circuit; workspace as for zkvc_prove.  Synchronises
 * `stream`.
 */
int zkvc_prove_claimed(const zkvc_pk* pk, const int8_t* d_X, const int8_t* d_W, const int32_t* d_Y_claimed,
                       const uint8_t rs[64], void* d_ws, size_t ws_bytes, uint8_t proof[256], void* stream);

int zkvc_prove_mode(const zkvc_pk* pk, int mode, const int8_t* d_X, const int8_t* d_W, const uint8_t rs[64],
                    int32_t* d_Y, void* d_ws, size_t ws_bytes, uint8_t proof[256], void* stream);

/* ------------------------------------------------------------------ circuit variants
 * The paper's ablation (Sec. V, Table II) compares four R1CS encodings of the same
 * matmul, and its verify timing suggests few public inputs.  zkvc_setup_circuit builds a
 * key for any of them on a generic sparse-R1CS layout (variables one | X | Y | W |
 * auxiliary, circuit rows then input-consistency rows):
 *   ZKVC_CIRCUIT_CRPC_PSQ  CRPC (Sec. III-A) with the PSQ chain (Sec. III-B): n rows,
 *                          auxiliary S_0..S_(n-2) -- the same circuit as zkvc_setup
 *   ZKVC_CIRCUIT_CRPC      CRPC without PSQ: rows a_k b_k = p_k, then
 *                          (p_0 + ... + p_(n-1)) * 1 = Y(z); auxiliary p_k
 *   ZKVC_CIRCUIT_PSQ       PSQ without CRPC: per output y_ij the chain
 *                          x_ik w_kj = S_ijk - S_ij(k-1), closing on y_ij (a b n rows)
 *   ZKVC_CIRCUIT_VANILLA   x_ik w_kj = p_ijk per product (a b n rows, Sec. III-A's count)
 *                          and (sum_k p_ijk) * 1 = y_ij per output
 *   ZKVC_CIRCUIT_SOFTMAX   CRPC + PSQ, then the nonlinear gadgets of Sec. III-C on each
 *                          row of Y (read as fixed point with ZKVC_GADGET_FRAC_BITS
 *                          fractional bits): the row maximum x_max verified by
 *                          x_max >= y_ij (32-bit decompositions of d = x_max - y_ij) and
 *                          prod_j (x_max - y_ij) = 0 (a chain of products), then e^x at
 *                          x = -d approximated by 0 below T = -2^ZKVC_GADGET_EXP_SQUARINGS
 *                          and by (1 + x/2^n)^(2^n), n = ZKVC_GADGET_EXP_SQUARINGS,
 *                          above: a 33-bit decomposition compares with T, the bits of d
 *                          from n up give the division by 2^n, n squarings give the
 *                          power.  71 rows per entry plus max(1, b - 1) per row of Y.
 *   ZKVC_CIRCUIT_GELU      CRPC + PSQ, then GELU(x) ~ x^2/8 + x/4 + 1/2 (Sec. III-C) on
 *                          every entry of Y, exactly at scale 2^(2F + 3): one row
 *                          y * y = G - 2^(F+1) y - 2^(2F+2) per entry.
 *                          Requires |y| < 2^31 (int8 products with n < 2^16 are).
 *                          The gadgets' outputs are auxiliary (private) variables.
 * and public_io ZKVC_PUBLIC_XY (X and Y public) or ZKVC_PUBLIC_NONE (only the constant
 * one is public; the verifier then takes no X or Y).  toxic and the error behaviour are
 * those of zkvc_setup (z is unused by the circuits without CRPC but still checked).
 * zkvc_prove / zkvc_prove_mode on such a key run the generic prover (the two
 * multiplications s A and r B1 are variable-base, as in ZKVC_PROVE_CHAIN, whichever mode
 * is asked); zkvc_prove_workspace_bytes sizes it.  zkvc_pk_export on such a key indexes
 * ZKVC_Q_A / B1 / B2 / L by variable (all-zero bytes where the query has no entry), H by
 * position.  pk files, batches and the server take zkvc_setup keys only.
 * zkvc_pk_circuit reports a key's circuit, public-input mode, rows and variables.
 */
#define ZKVC_CIRCUIT_CRPC_PSQ 0
#define ZKVC_CIRCUIT_CRPC 1
#define ZKVC_CIRCUIT_PSQ 2
#define ZKVC_CIRCUIT_VANILLA 3
#define ZKVC_CIRCUIT_SOFTMAX 4
#define ZKVC_CIRCUIT_GELU 5
#define ZKVC_GADGET_FRAC_BITS 12
#define ZKVC_GADGET_EXP_SQUARINGS 3
#define ZKVC_PUBLIC_XY 0
#define ZKVC_PUBLIC_NONE 1
int zkvc_setup_circuit(int a, int n, int b, int circuit, int public_io, const uint8_t toxic[192], void* stream,
                       zkvc_pk** pk, zkvc_vk** vk);
int zkvc_pk_circuit(const zkvc_pk* pk, int* circuit, int* public_io, uint64_t* rows, uint64_t* vars);

/* ------------------------------------------------------------------ batched proving
 * Many proofs of uneven shapes in one launch sequence (the paper proves the matmul
 * layers of a network, Sec. V, each as its own CRPC circuit; batching them is this
 * library's throughput form of Prove).  A batch is built once for an ordered list of
 * proving keys (repeats allowed, all on the current device) and then proves one
 * instance per key per call.  Proofs are byte-identical to zkvc_prove's for the same
 * (pk, X, W, r, s).
 *
 * zkvc_batch_create allocates every device buffer the batch needs (ZKVC_ENOMEM if the
 * device cannot hold them) plus pinned host staging, and synchronises.  Flags:
 *   ZKVC_BATCH_AUTOTUNE  the first zkvc_batch_prove times candidate MSM chunk sizes,
 *                        block sizes and NTT tile sizes on its own inputs and keeps the
 *                        fastest before capturing (adds a few batch-times once);
 *   ZKVC_BATCH_EAGER     launch the sequence every call instead of capturing it once as
 *                        a CUDA graph and replaying it.
 * The keys must outlive the batch.  A batch is used by one thread at a time.
 *
 * zkvc_batch_prove(b, d_X[i], d_W[i], rs, d_Y[i], proofs, status, stream):
 *   d_X[i], d_W[i]  instance i's int8 matrices (device, row-major, shapes of key i);
 *   rs              count x 64 bytes (host): r || s of each instance, canonical Fr;
 *   d_Y[i]          instance i's a x b int32 output (device);
 *   proofs          count x 256 bytes (host output), in key order;
 *   status          optional count ints (host output): per-instance ZKVC_OK, ZKVC_EINVAL
 *                   (non-canonical r or s) or ZKVC_EUNSAT.
 * The inputs are read after the caller's earlier work on `stream`; the call returns when
 * the proofs are on the host, waiting at most zkvc_set_wait_timeout_ms (ZKVC_ETIMEOUT
 * then: the batch's work keeps running and the next call on the batch waits for it).
 * Returns the first failing instance's status.
 *
 * zkvc_batch_get_tuning / zkvc_batch_set_tuning read or impose the launch shape as
 * ZKVC_BATCH_TUNING_LEN integers: for the small G1, main G1 and G2 MSM runs in turn
 * (chunk terms per thread, accumulation threads per block), then the
 * NTT's log2 elements per block.  Setting re-captures on the next prove.
 *
 * zkvc_batch_terms reports the bucket terms (point additions) of the last call's three
 * MSM runs, for throughput accounting.
 *
 * zkvc_prove_batch is a one-shot form (create eagerly, prove, free).
 */
typedef struct zkvc_batch zkvc_batch;
#define ZKVC_BATCH_AUTOTUNE 1
#define ZKVC_BATCH_EAGER 2
#define ZKVC_BATCH_TUNING_LEN 7

int zkvc_batch_create(const zkvc_pk* const* pks, int count, int flags, zkvc_batch** batch);
void zkvc_batch_free(zkvc_batch* batch);
int zkvc_batch_info(const zkvc_batch* batch, int* count, size_t* device_bytes, uint64_t* graph_launches);
int zkvc_batch_get_tuning(const zkvc_batch* batch, int32_t* params, int n);
/* Bucket terms (nonzero signed digits, one point addition each) of the last call's
 * small G1, main G1 and G2 runs; synchronises the batch's stream. */
int zkvc_batch_terms(const zkvc_batch* batch, uint64_t terms[3]);
int zkvc_batch_set_tuning(zkvc_batch* batch, const int32_t* params, int n);
int zkvc_batch_prove(zkvc_batch* batch, const int8_t* const* d_X, const int8_t* const* d_W, const uint8_t* rs,
                     int32_t* const* d_Y, uint8_t* proofs, int* status, void* stream);
int zkvc_prove_batch(const zkvc_pk* const* pks, const int8_t* const* d_X, const int8_t* const* d_W, const uint8_t* rs,
                     int count, int32_t* const* d_Y, uint8_t* proofs, int* status, void* stream);

/* ------------------------------------------------------------------ proof server
 * Continuous batching of proof requests (the paper's use case, Sec. I: a client sends X
 * and receives Y with a proof; here many clients share one GPU).  The server keeps the
 * given proving keys resident (they must outlive it) and preallocates `mem_budget` bytes
 * of device memory for per-request state.  `slots` worker threads, each with its own CUDA
 * stream, take requests in arrival order: the head of the queue is admitted as soon as a
 * worker is idle and its footprint (zkvc_server_request_bytes: prove workspace plus X, W
 * and Y) fits in the unused budget, so requests that arrive while others run overlap
 * with them on the device.  A request that can never fit completes with ZKVC_ENOMEM.
 * Policy: ZKVC_SERVER_ADAPTIVE proves a request that finds the GPU idle with
 * ZKVC_PROVE_FOLD (lowest latency) and one admitted beside others with ZKVC_PROVE_CHAIN
 * (less work per proof); ZKVC_SERVER_FOLD / _CHAIN force one mode.  ZKVC_SERVER_MERGE
 * adds batching across requests: a worker that finds two or more requests queued takes
 * the longest prefix of the queue (at most 64 requests) whose batch fits in the largest
 * free block of the budget and proves it with the batched prover's launch sequence
 * (zkvc_batch_*: batched NTTs, merged multi-instance MSM runs; run eagerly with default
 * launch shapes, over the server's own memory); a request alone in the queue takes the
 * one-proof path as under ZKVC_SERVER_ADAPTIVE.  Results are the same bytes as
 * zkvc_prove's under every policy.
 *
 * zkvc_server_submit copies X (a x n int8, host) and W (n x b int8, host) and rs (64
 * bytes, host) of key `key` and returns a ticket at once.  zkvc_server_wait blocks up to
 * timeout_ms for a ticket: ZKVC_ETIMEOUT if it is not done (the ticket stays valid),
 * otherwise ZKVC_OK with *status = the request's status, the proof (256 bytes) and Y
 * (a x b int32) copied out when it succeeded (either may be NULL), and times_ms = {queue,
 * prove, total} milliseconds from submission; the ticket is then released.
 * zkvc_server_free stops the workers after their current requests; queued requests are
 * dropped.  Submit, wait and stats may be called from any thread.
 */
typedef struct zkvc_server zkvc_server;
#define ZKVC_SERVER_ADAPTIVE 0
#define ZKVC_SERVER_FOLD 1
#define ZKVC_SERVER_CHAIN 2
#define ZKVC_SERVER_MERGE 3

int zkvc_server_create(const zkvc_pk* const* pks, int npk, int slots, size_t mem_budget, int policy,
                       zkvc_server** server);
void zkvc_server_free(zkvc_server* server);
int zkvc_server_submit(zkvc_server* server, int key, const int8_t* X, const int8_t* W, const uint8_t rs[64],
                       uint64_t* ticket);
int zkvc_server_wait(zkvc_server* server, uint64_t ticket, int timeout_ms, uint8_t proof[256], int32_t* Y,
                     double times_ms[3], int* status);
int zkvc_server_stats(zkvc_server* server, uint64_t* completed, int* in_flight, int* queued, size_t* bytes_in_use,
                      size_t* peak_bytes, uint64_t* chain_mode);
/* Requests proven in merged batches, and the batches (ZKVC_SERVER_MERGE), since creation. */
int zkvc_server_merge_stats(zkvc_server* server, uint64_t* merged_requests, uint64_t* batches);
size_t zkvc_server_request_bytes(const zkvc_pk* pk, int mode);

/* Diagnostic knob for the bounded device-side waits (the fault handling that a
 * production prover needs; no counterpart in the paper): the time limit, in ns, of the
 * tensor-core witness matmul's waits for its MMAs in kernels launched from now on (the
 * one-proof and generic provers, the server and zkvc_matmul_i8; default 200 ms; captured
 * graphs keep the value of their capture).  0 makes the first wait give up at once, which
 * exercises the timeout path: the kernel flags the timeout, waits for its outstanding MMAs
 * with the full 200 ms limit, frees its tensor memory and returns, and the call reports
 * ZKVC_ETIMEOUT.  Always ZKVC_OK.
 */
int zkvc_set_device_wait_limit_ns(uint64_t ns);

/* Deadline of the library's host-side waits for device work (batched proving and the
 * proof server), in milliseconds (default 60000).  A wait that runs out returns
 * ZKVC_ETIMEOUT instead of blocking forever. */
int zkvc_set_wait_timeout_ms(int ms);

#ifdef __cplusplus
}
#endif

#endif /* ZKVC_H_ */
