// Groth16 Prove for the CRPC + PSQ matmul circuit (zkVC Sec. II: Prove; Sec. III-A: CRPC;
// Sec. III-B: PSQ), as one stream-ordered chain of kernels:
//
//  1. Y = X W exactly (int8 x int8 -> int32), the computation being proven.
//  2. CRPC evaluations a_k = sum_i z^(ib) x_ik, b_k = sum_j z^j w_kj and
//     Y(z) = sum_i z^(ib) sum_j z^j y_ij (block reductions of small-integer x Fr products).
//  3. PSQ prefix sums S_k = S_(k-1) + a_k b_k (one-block scan); the closing constraint
//     S_(n-2) + a_(n-1) b_(n-1) = Y(z) is checked on the device (ZKVC_EUNSAT otherwise).
//  4. QAP evaluations on the domain: A_ev = (a_k | 1, X, Y), B_ev = (b_k), C_ev = (a_k b_k).
//  5. h = (A B - C) / t via INTT (DIF, bit-reversed out, scaled by g^i / N), coset NTT
//     (DIT back to natural order), pointwise division by g^N - 1, coset INTT (DIF, scaled
//     by g^-i / N).  h stays in bit-reversed order; the H query is stored in that order.
//     h at natural index N - 1 must vanish (checked).
//  6. One merged G1 MSM with two outputs and one G2 MSM (on a side stream, overlapping
//     steps 1-6).  By linearity the randomised Groth16 elements become fixed-base sums:
//        A = [alpha]1 + sum_v w_v [A_v]1 + r [delta]1
//        B = [beta]2  + sum_W w_e [B_e]2 + s [delta]2
//        C = sum_priv w_i [L_i]1 + sum_j h_j [H_j]1 + s A + r B1 - r s [delta]1
//          = sum w_i [L_i]1 + sum h_j [H_j]1 + s [alpha]1 + r [beta]1 + r s [delta]1
//            + sum_v (s w_v) [A_v]1 + sum_W (r w_e) [B_e]1,
//     so no variable-base multiplication (and no serial doubling chain) remains: every
//     base is a proving-key point stored with its 2^(16 w) multiples.
//  7. Affine conversion (one inversion per point, in parallel) and the canonical
//     256-byte encoding A || B || C.
#include <algorithm>
#include <array>
#include <optional>
#include <mutex>
#include <new>
#include <cstring>

#include "coop.cuh"
#include "sliced.cuh"
#include "glv.h"
#include "groth16.h"
#include "msm.h"
#include "witness.cuh"

namespace zkvc {

// ------------------------------------------------------------------ witness
// block k < n: a_k and b_k
__global__ void __launch_bounds__(256) k_crpc_ab(const int8_t* __restrict__ X, const int8_t* __restrict__ W,
                                                 const Fr* __restrict__ zA, const Fr* __restrict__ zB, int a, int n, int b,
                                                 Fr* ak, Fr* bk) {
  __shared__ Fr sh[256];
  crpc_ab_row(X, W, zA, zB, a, n, b, blockIdx.x, ak, bk, sh);
}

// block i < a: z^(ib) sum_j z^j y_ij
__global__ void __launch_bounds__(256) k_crpc_y(const int32_t* __restrict__ Y, const Fr* __restrict__ zA,
                                                const Fr* __restrict__ zB, int b, Fr* part) {
  __shared__ Fr sh[256];
  crpc_y_row(Y, zA, zB, b, blockIdx.x, part, sh);
}

// One block of 1024 threads: products, prefix sums, closing check, first n evaluations.
__global__ void __launch_bounds__(1024) k_psq(const Fr* __restrict__ ak, const Fr* __restrict__ bk,
                                              const Fr* __restrict__ ypart, int a, int n, Fr* S, Fr* Aev, Fr* Bev,
                                              Fr* Cev, int* flags) {
  __shared__ Fr sh[1024];
  psq_chain(ak, bk, ypart, a, n, S, Aev, Bev, Cev, flags, sh);
}

// domain rows n .. N-1
__global__ void k_domain_rest(const int8_t* __restrict__ X, const int32_t* __restrict__ Y, int n, uint32_t an,
                              uint32_t l, size_t N, Fr* Aev, Fr* Bev, Fr* Cev) {
  size_t k = n + size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= N) return;
  domain_rest_row(X, Y, n, an, l, k, Aev, Bev, Cev);
}

__global__ void k_check_h(const Fr* H, size_t N, int* flags) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && !ld_field(H + (N - 1)).is_zero()) atomicOr(flags, 2);
}

// rs[0] = r, rs[1] = s (canonical, from the caller); rs[2] = r s, rs[3] = -r s (canonical)
__global__ void k_randomness(Fr* rs, int* flags) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Fr r = ld_field(rs), s = ld_field(rs + 1);
  if (!canonical_fr(r) || !canonical_fr(s)) atomicOr(flags, 4);
  Fr rsv = f_mul(f_to_mont(r), s);  // (r R) s / R = r s, canonical
  st_field(rs + 2, rsv);
  st_field(rs + 3, f_neg(rsv));
}

// Chain mode: s A and r B1 (small-run outputs 0 and 2) with the scalars split by the GLV
// endomorphism on the host (gs[0] = s, gs[1] = r): four warps compute s1 A, s2 phi(A),
// r1 B1 and r2 phi(B1) side by side (phi(x, y) = (beta x, y)) in limb-sliced arithmetic
// (sliced.cuh: eight lanes per product, four products per warp), then two warps add the
// pairs.  Meanwhile the fifth warp encodes A (bytes 0..63 of the proof: its inversion
// overlaps the chains).  Then the H-free part of C, small[1] + s A + r B1, goes to cpart.
// (proof and cpart may be null: the generic engine encodes A and C itself.)  One block
// of 160 threads.
__global__ void __launch_bounds__(160) k_chains(const GlvScalar* __restrict__ gs, const G1J* __restrict__ small,
                                                G1J* chain, G1J* cpart, uint8_t* proof) {
  __shared__ G1J T[4][16];
  __shared__ G1J part[4];
  const int w = threadIdx.x >> 5;
  if (threadIdx.x == 128 && proof) encode_g1(ld_field(small), proof);
  if (w < 4) {
    SlG1 P = sl_ld(small + (w < 2 ? 0 : 2));
    if (w & 1) {  // beta in Montgomery form: beta R^2 R^-1
      const int j = sl_limb();
      uint32_t beta = 0, r2 = 0;
#pragma unroll
      for (int i = 0; i < 8; i++) {
        beta |= glv_beta_limb(i) & (0u - uint32_t(j == i));
        r2 |= r2_limb<FpCfg>(i) & (0u - uint32_t(j == i));
      }
      P.X = sl_mul(P.X, sl_mul(beta, r2));
    }
    sl_st(part + w, sl_mul_half(P, gs[w >> 1].h[w & 1], T[w]));
  }
  __syncthreads();
  if (w == 0 || w == 2) sl_st(part + w, sl_padd(sl_ld(part + w), sl_ld(part + w + 1)));
  __syncthreads();
  if (w == 0) {
    const SlG1 sA = sl_ld(part), rB = sl_ld(part + 2);
    sl_st(chain, sA);
    sl_st(chain + 1, rB);
    if (cpart) sl_st(cpart, sl_padd(sl_ld(small + 1), sl_padd(sA, rB)));
  }
}

// sw[v] = s w_v for v = 0 .. l (one, X, Y), sa[k] = s a_k and rb[k] = r b_k (k < n), in
// Montgomery form: the scalars of the C terms s sum_v w_v [L_(n+v)]1, s sum_k a_k [L_k]1
// and r sum_k b_k [L_k]1 (s A and r B1 expanded by linearity over the CRPC rows).
__global__ void k_scaled_witness(const int8_t* __restrict__ X, const int32_t* __restrict__ Y, const Fr* __restrict__ ak,
                                 const Fr* __restrict__ bk, const Fr* __restrict__ rs, uint32_t an, uint32_t l, uint32_t n,
                                 Fr* sw, Fr* sa, Fr* rb) {
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= l) {
    Fr s = f_to_mont(ld_field(rs + 1));
    Fr w = t == 0 ? Fr::one() : (t <= an ? f_from_int<FrCfg>(X[t - 1]) : f_from_int<FrCfg>(Y[t - 1 - an]));
    st_field(sw + t, f_mul(s, w));
  } else if (t < l + 1 + n) {
    uint32_t k = t - l - 1;
    st_field(sa + k, f_mul(f_to_mont(ld_field(rs + 1)), ld_field(ak + k)));
  } else if (t < l + 1 + 2 * n) {
    uint32_t k = t - l - 1 - n;
    st_field(rb + k, f_mul(f_to_mont(ld_field(rs)), ld_field(bk + k)));
  }
}

// Proof encoding.  A = small[0]; C = small[1] + x[0] + y[0] + (chain ? chain[0] + chain[1]
// : 0), where (x, y) are the rest and H results (fold mode) or the main result and
// infinity (chain mode).  Thread 0 converts A and C with one shared inversion; thread 32
// (another warp) converts B concurrently.
// The proof is encoded piecewise as its parts become ready, so that only C's last
// addition and inversion follow the H MSM: B on the G2 stream, A (and the part of C
// without the H and rest terms) on the small-digit stream, the rest term on its own
// stream, and C on the main stream after the joins.
__global__ void k_encode_a(const G1J* small, const G1J* chain, G1J* cpart, uint8_t* proof) {
  if (threadIdx.x != 0) return;
  G1J c = ld_field(small + 1);
  if (chain) c = p_add(c, p_add(ld_field(chain), ld_field(chain + 1)));
  st_field(cpart, c);
  encode_g1(ld_field(small), proof);
}

__global__ void k_encode_b(const G2J* res2, uint8_t* proof) {
  if (threadIdx.x == 0) encode_b(ld_field(res2), proof);
}

__global__ void k_add_into(G1J* acc, const G1J* x) {
  const G1J r = p_add_quad(ld_field(acc), ld_field(x));
  if (threadIdx.x == 0) st_field(acc, r);
}

// C = cpart + H, then its canonical affine encoding (bytes 192..255), on one warp in
// limb-sliced arithmetic: the addition, ZZ ZZZ and the products of the affine conversion
// (x = X ZZZ / (ZZ ZZZ), y = Y ZZ / (ZZ ZZZ), then out of Montgomery form) run sliced,
// the inversion in lane 0.
__global__ void __launch_bounds__(32) k_encode_c(const G1J* cpart, const G1J* h, uint8_t* proof) {
  __shared__ uint32_t zs[8], inv[8];
  const SlG1 C = sl_padd(sl_ld(cpart), sl_ld(h));
  const int j = sl_limb(), grp = sl_group();
  uint8_t* out = proof + 192;
  if (sl_is_zero(C.ZZ)) {  // infinity encodes as zeros
    for (int i = threadIdx.x; i < 64; i += 32) out[i] = 0;
    return;
  }
  const uint32_t z = sl_mul(C.ZZ, C.ZZZ);
  if (grp == 0) zs[j] = z;
  __syncwarp();
  if (threadIdx.x == 0) {
    Fp zf;
#pragma unroll
    for (int i = 0; i < 8; i++) zf.v[i] = zs[i];
    const Fp iv = f_inv(zf);
#pragma unroll
    for (int i = 0; i < 8; i++) inv[i] = iv.v[i];
  }
  __syncwarp();
  const uint32_t m = sl_mul(inv[j], sl_pick(C.ZZZ, C.ZZ, C.ZZZ, C.ZZ));
  const uint32_t a = sl_mul(sl_pick(C.X, C.Y, C.X, C.Y), m);  // group 0: x, group 1: y (Montgomery)
  const uint32_t c = sl_mul(a, j == 0 ? 1u : 0u);             // times R^-1: canonical
  if (grp < 2) {
    uint8_t* o = out + 32 * grp + 4 * j;
    o[0] = (uint8_t)c;
    o[1] = (uint8_t)(c >> 8);
    o[2] = (uint8_t)(c >> 16);
    o[3] = (uint8_t)(c >> 24);
  }
}


// ------------------------------------------------------------------ plans and workspace
struct ProveBufs {
  Fr *ak, *bk, *yz, *S, *ev, *rs, *sw, *sa, *rb;
  int* flags;
  G1J *res_small, *res_rest, *res_h, *res_chain, *cpart;
  GlvScalar* glv;
  G2J* res2;
  uint8_t* proof;
  void *ws_small, *ws_rest, *ws_h, *ws2;
  size_t ws_small_bytes, ws_rest_bytes, ws_h_bytes, ws2_bytes;
};

static MsmSeg seg_of(const Region& r, uint32_t first, uint32_t count, uint32_t out, int kind, const void* sc,
                     uint32_t skip = 0xffffffffu) {
  MsmSeg s{};
  s.base_off = r.off + uint64_t(first) * r.nwin;
  s.count = count;
  s.nwin = r.nwin;
  s.out = out;
  s.kind = kind;
  s.scalars = sc;
  s.skip = skip;
  return s;
}

// The MSM runs of one proof.  Fold mode (four runs on four streams):
//   small (G1, 8-bit digits): output 0 = A = [alpha]1 + the input rows of one, X, Y +
//               sum_k a_k [L_k]1 + r [delta]1; output 1 = the CRPC part of C:
//               sum_k b_k [alpha L_k / delta]1 (L over W) + s sum_k a_k [L_k]1 +
//               r sum_k b_k [L_k]1;
//   rest  (G1, 16-bit digits): the rest of C known right after the witness: L over S,
//               s w_v over the input rows, s alpha, r beta, r s delta;
//   h     (G1): the H part of C, after the NTTs;
//   g2:         output 0 = B = [beta]2 + sum_k b_k [L_k]2 + s [delta]2.
// "rest" does not depend on h, so it overlaps the NTTs; only "h" follows them.
// Chain mode (three runs): small adds output 2 = B1 = [beta]1 + sum_k b_k [L_k]1 +
// s [delta]1 and drops the s and r terms from output 1; "h" also takes L over S and
// -r s [delta]1; there is no "rest"; two variable-base multiplications s A and r B1
// complete C = L + H + s A + r B1 - r s delta.
struct Plans {
  MsmPlan small, rest, h, g2;
};

static void plans(const zkvc_pk* pk, int mode, const int8_t* dX, const int32_t* dY, const Fr* ak, const Fr* bk,
                  const Fr* S, const Fr* h, const Fr* rs, const Fr* sw, const Fr* sa, const Fr* rb, Plans* P) {
  const Shape& sh = pk->shape;
  const Region* g = pk->lay.g1;
  const uint32_t an = sh.a * sh.n, ab = sh.a * sh.b, n = sh.n;
  const bool chain = mode == ZKVC_PROVE_CHAIN;
  P->small.outs = {{8, 1, 0, 0}, {8, 1, 0, 0}};
  P->small.segs = {
      seg_of(g[R1_AIN], 0, 1, 0, SK_ONE, nullptr),
      seg_of(g[R1_AIN], 1, an, 0, SK_I8, dX),
      seg_of(g[R1_AY8], 0, ab, 0, SK_I32, dY),
      seg_of(g[R1_ALPHA], 0, 1, 0, SK_ONE, nullptr),
      seg_of(g[R1_DELTA8], 0, 1, 0, SK_FR_CANON, rs + 0),
      seg_of(g[R1_LK], 0, n, 0, SK_FR_MONT, ak),
      seg_of(g[R1_ALK], 0, n, 1, SK_FR_MONT, bk),
  };
  P->h.outs = {{ZKVC_C1, 1, 0, 0}};
  P->h.segs = {seg_of(g[R1_H], 0, (uint32_t)sh.N, 0, SK_FR_MONT, h, (uint32_t)sh.N - 1)};
  if (chain) {
    P->small.outs.push_back({8, 1, 0, 0});
    P->small.segs.push_back(seg_of(g[R1_LK], 0, n, 2, SK_FR_MONT, bk));
    P->small.segs.push_back(seg_of(g[R1_BETA], 0, 1, 2, SK_ONE, nullptr));
    P->small.segs.push_back(seg_of(g[R1_DELTA8], 0, 1, 2, SK_FR_CANON, rs + 1));
    P->h.segs.push_back(seg_of(g[R1_LS], 0, (uint32_t)(sh.n - 1), 0, SK_FR_MONT, S));
    P->h.segs.push_back(seg_of(g[R1_DELTA], 0, 1, 0, SK_FR_CANON, rs + 3));
  } else {
    P->small.segs.push_back(seg_of(g[R1_LK], 0, n, 1, SK_FR_MONT, sa));
    P->small.segs.push_back(seg_of(g[R1_LK], 0, n, 1, SK_FR_MONT, rb));
    P->rest.outs = {{ZKVC_C1, 1, 0, 0}};
    P->rest.segs = {
        seg_of(g[R1_LS], 0, (uint32_t)(sh.n - 1), 0, SK_FR_MONT, S),
        seg_of(g[R1_AIN], 0, sh.l + 1, 0, SK_FR_MONT, sw),
        seg_of(g[R1_ALPHA], 0, 1, 0, SK_FR_CANON, rs + 1),
        seg_of(g[R1_BETA], 0, 1, 0, SK_FR_CANON, rs + 0),
        seg_of(g[R1_DELTA], 0, 1, 0, SK_FR_CANON, rs + 2),
    };
  }
  const Region* g2 = pk->lay.g2;
  P->g2.outs = {{ZKVC_C2, 1, 0, 0}};
  P->g2.segs = {
      seg_of(g2[R2_LK], 0, n, 0, SK_FR_MONT, bk),
      seg_of(g2[R2_BETA], 0, 1, 0, SK_ONE, nullptr),
      seg_of(g2[R2_DELTA], 0, 1, 0, SK_FR_CANON, rs + 1),
  };
  P->small.tune.chunk = pk->prove_tune[0];
  P->rest.tune.chunk = pk->prove_tune[1];
  P->h.tune.chunk = pk->prove_tune[2];
  P->g2.tune.chunk = pk->prove_tune[3];
  P->h.tune.lanes = pk->prove_tune[8] ? 4 : 1;
  P->small.tune.lanes = pk->prove_tune[9] ? 4 : 1;
  P->rest.tune.lanes = 1;
  P->g2.tune.lanes = 4;  // a proof's G2 run is latency-bound
  if (!chain) msm_plan_finalize(P->rest);
  msm_plan_finalize(P->small);
  msm_plan_finalize(P->h);
  msm_plan_finalize(P->g2);
}

static size_t carve(const zkvc_pk* pk, int mode, void* base, size_t cap, ProveBufs* B, bool measuring) {
  const Shape& sh = pk->shape;
  const bool chain = mode == ZKVC_PROVE_CHAIN;
  Arena a;
  a.base = reinterpret_cast<uint8_t*>(base);
  a.cap = cap;
  a.measuring = measuring;
  B->ak = a.take<Fr>(sh.n);
  B->bk = a.take<Fr>(sh.n);
  B->yz = a.take<Fr>(sh.a);
  B->S = a.take<Fr>(sh.n);
  B->ev = a.take<Fr>(4 * sh.N);
  B->rs = a.take<Fr>(4);
  B->sw = chain ? nullptr : a.take<Fr>(sh.l + 1);
  B->sa = chain ? nullptr : a.take<Fr>(sh.n);
  B->rb = chain ? nullptr : a.take<Fr>(sh.n);
  B->flags = a.take<int>(4);
  B->res_small = a.take<G1J>(3);
  B->res_rest = a.take<G1J>(1);
  B->res_h = a.take<G1J>(1);
  B->res_chain = a.take<G1J>(2);
  B->cpart = a.take<G1J>(1);
  B->glv = a.take<GlvScalar>(2);
  B->res2 = a.take<G2J>(1);
  B->proof = a.take<uint8_t>(256);
  Plans P;
  plans(pk, mode, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, &P);
  B->ws_small_bytes = msm_workspace_bytes<Fp>(P.small);
  B->ws_rest_bytes = chain ? 0 : msm_workspace_bytes<Fp>(P.rest);
  B->ws_h_bytes = msm_workspace_bytes<Fp>(P.h);
  B->ws2_bytes = msm_workspace_bytes<Fp2>(P.g2);
  B->ws_small = a.take<uint8_t>(B->ws_small_bytes);
  B->ws_rest = chain ? nullptr : a.take<uint8_t>(B->ws_rest_bytes);
  B->ws_h = a.take<uint8_t>(B->ws_h_bytes);
  B->ws2 = a.take<uint8_t>(B->ws2_bytes);
  return a.off;
}

// Per-thread side streams and fork/join events (created on first use on each device).
static constexpr int NSIDE = 4;
struct SideStreams {
  int dev = -1;
  cudaStream_t st[NSIDE] = {};
  cudaEvent_t fork[NSIDE] = {}, join[NSIDE] = {};
  cudaEvent_t ntt_done = nullptr, h_accum = nullptr;  // points where the rest MSM may start
  cudaEvent_t wit_y = nullptr, wit_psq = nullptr;     // Y = X W done; PSQ chain done
};
static thread_local SideStreams t_side;

static int side_streams(SideStreams** out) {
  int dev = 0;
  ZK_CUDA(cudaGetDevice(&dev));
  if (t_side.st[0] == nullptr || t_side.dev != dev) {
    t_side.dev = dev;
    int lo = 0, hi = 0;
    ZK_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    for (int i = 0; i < NSIDE; i++) {
      // Stream 3 carries the critical chain NTT -> H MSM: its blocks go first.  Streams 0
      // and 1 (the latency-bound G2 and small-digit MSMs) come next; stream 2 carries the
      // throughput-bound "rest" MSM at the default priority and fills the gaps.
      const int next = hi < lo ? hi + 1 : hi;
      ZK_CUDA(cudaStreamCreateWithPriority(&t_side.st[i], cudaStreamNonBlocking, i == 3 ? hi : i == 2 ? lo : next));
      ZK_CUDA(cudaEventCreateWithFlags(&t_side.fork[i], cudaEventDisableTiming));
      ZK_CUDA(cudaEventCreateWithFlags(&t_side.join[i], cudaEventDisableTiming));
    }
    ZK_CUDA(cudaEventCreateWithFlags(&t_side.ntt_done, cudaEventDisableTiming));
    ZK_CUDA(cudaEventCreateWithFlags(&t_side.h_accum, cudaEventDisableTiming));
    ZK_CUDA(cudaEventCreateWithFlags(&t_side.wit_y, cudaEventDisableTiming));
    ZK_CUDA(cudaEventCreateWithFlags(&t_side.wit_psq, cudaEventDisableTiming));
  }
  *out = &t_side;
  return ZKVC_OK;
}

size_t prove_workspace_bytes(const zkvc_pk* pk, int mode) {
  ProveBufs B;
  return carve(pk, mode, nullptr, 0, &B, true);
}

static int fork_to(SideStreams* side, int i, cudaStream_t st) {
  ZK_CUDA(cudaEventRecord(side->fork[i], st));
  ZK_CUDA(cudaStreamWaitEvent(side->st[i], side->fork[i], 0));
  return ZKVC_OK;
}

// Enqueues one proof on st (and the calling thread's side streams, joined back into st).
// rs_host is read before the call returns; the proof lands in proof_out and the device
// flags in flags_out (host pointers, written when st reaches them: pinned memory lets the
// copies run asynchronously).  glv_host, when given (pinned, chain mode), supplies the
// GLV halves of s and r as a copy source instead of a split made now: a captured graph
// then reads whatever the host wrote there before each replay.
// y_given: dY holds a claimed Y (the caller's) instead of receiving X W; the witness
// takes it as is and the PSQ check and the quotient check decide whether it is X W.
static int prove_enqueue_impl(const zkvc_pk* pk, int mode, const int8_t* dX, const int8_t* dW, const uint8_t* rs_host,
                              const GlvScalar* glv_host, int32_t* dY, void* ws, size_t ws_bytes, uint8_t* proof_out,
                              int* flags_out, cudaStream_t st, bool y_given = false) {
  ZK_CHECK(pk && dX && dW && rs_host && dY && ws && proof_out && flags_out, ZKVC_EINVAL, "prove: null argument");
  ZK_CHECK(mode == ZKVC_PROVE_FOLD || mode == ZKVC_PROVE_CHAIN, ZKVC_EINVAL, "prove: mode %d", mode);
  size_t need = prove_workspace_bytes(pk, mode);
  ZK_CHECK(ws_bytes >= need, ZKVC_EINVAL, "prove: workspace %zu < %zu bytes", ws_bytes, need);
  const bool chain = mode == ZKVC_PROVE_CHAIN;
  const Shape& sh = pk->shape;
  ProveBufs B;
  carve(pk, mode, ws, ws_bytes, &B, false);
  const size_t N = sh.N;
  Fr* Aev = B.ev;
  Fr* Bev = B.ev + N;
  Fr* Cev = B.ev + 2 * N;
  Fr* Hev = B.ev + 3 * N;

  NvtxRange nv_prove("zkvc/prove");
  std::optional<NvtxRange> nv_stage;
  nv_stage.emplace("zkvc/prove/witness");
  prof_mark(PS_WITNESS, true, st);
  ZK_CUDA(cudaMemsetAsync(B.flags, 0, 4 * sizeof(int), st));
  ZK_CUDA(cudaMemcpyAsync(B.rs, rs_host, 64, cudaMemcpyHostToDevice, st));
  if (chain && glv_host) {
    ZK_CUDA(cudaMemcpyAsync(B.glv, glv_host, 2 * sizeof(GlvScalar), cudaMemcpyHostToDevice, st));
  } else if (chain) {
    // s and r split by the GLV endomorphism for the two scalar multiplications
    const GlvScalar g[2] = {glv_split(rs_host + 32), glv_split(rs_host)};
    ZK_CUDA(cudaMemcpyAsync(B.glv, g, sizeof(g), cudaMemcpyHostToDevice, st));
  }
  k_randomness<<<1, 1, 0, st>>>(B.rs, B.flags); ZK_COUNT_LAUNCH();
  SideStreams* side = nullptr;
  ZK_TRY(side_streams(&side));
  Plans P;
  plans(pk, mode, dX, dY, B.ak, B.bk, B.S, Hev, B.rs, B.sw, B.sa, B.rb, &P);
  // The witness runs on two streams: the CRPC sums a_k, b_k (X, W only) and the domain
  // evaluations past row n (X, Y) on side stream 3, which then carries the critical
  // NTT -> H chain; Y = X W, Y(z) and the PSQ chain on the main stream.  The side streams
  // may start at the points recorded below; their work is enqueued after the critical
  // chain's, so that the host reaches that chain's launches as early as possible.
  ZK_TRY(fork_to(side, 3, st));
  cudaStream_t s3 = side->st[3];
  // 1. the CRPC sums a_k, b_k (side stream 3);  2. Y = X W (tensor cores), unless a
  // claimed Y is given
  k_crpc_ab<<<sh.n, 256, 0, s3>>>(dX, dW, pk->zA, pk->zB, sh.a, sh.n, sh.b, B.ak, B.bk); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  ZK_CUDA(cudaEventRecord(side->fork[0], s3));  // G2 MSM: needs b_k and s
  if (!y_given) ZK_TRY(matmul_i8(dX, dW, dY, sh.a, sh.n, sh.b, B.flags, st));
  ZK_CUDA(cudaEventRecord(side->wit_y, st));
  // 3. Y(z) and the PSQ prefix sums; in fold mode the scalars s w_v, s a_k, r b_k
  k_crpc_y<<<sh.a, 256, 0, st>>>(dY, pk->zA, pk->zB, sh.b, B.yz); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaStreamWaitEvent(st, side->fork[0], 0));  // a_k, b_k
  k_psq<<<1, 1024, 0, st>>>(B.ak, B.bk, B.yz, sh.a, sh.n, B.S, Aev, Bev, Cev, B.flags); ZK_COUNT_LAUNCH();
  if (!chain) {
    uint32_t nsc = sh.l + 1 + 2 * uint32_t(sh.n);
    k_scaled_witness<<<(nsc + 255) / 256, 256, 0, st>>>(dX, dY, B.ak, B.bk, B.rs, sh.a * sh.n, sh.l, sh.n, B.sw, B.sa,
                                                        B.rb); ZK_COUNT_LAUNCH();
  }
  ZK_CUDA(cudaGetLastError());
  ZK_CUDA(cudaEventRecord(side->fork[1], st));  // small-digit G1 MSM
  ZK_CUDA(cudaEventRecord(side->fork[2], st));  // rest MSM
  prof_mark(PS_WITNESS, false, st);
  ZK_CUDA(cudaEventRecord(side->wit_psq, st));
  // 4. remaining domain evaluations (side stream 3, once Y exists)
  size_t rest = N - sh.n;
  ZK_CUDA(cudaStreamWaitEvent(s3, side->wit_y, 0));
  k_domain_rest<<<(unsigned)((rest + 255) / 256), 256, 0, s3>>>(dX, dY, sh.n, sh.a * sh.n, sh.l, N, Aev, Bev, Cev); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  // 5-6. quotient and the H part of C on side stream 3 (the critical chain), after the
  // PSQ chain's first n evaluations
  ZK_CUDA(cudaStreamWaitEvent(s3, side->wit_psq, 0));
  nv_stage.reset();
  nv_stage.emplace("zkvc/prove/ntt");
  prof_mark(PS_NTT, true, s3);
  const NttDomain* d = pk->dom;
  const int elog = pk->prove_tune[4] ? (int)pk->prove_tune[4] : 10;
  ZK_TRY(ntt_quotient_chain(Aev, 1, N, d, s3, elog));
  k_check_h<<<1, 32, 0, s3>>>(Hev, N, B.flags); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  prof_mark(PS_NTT, false, s3);
  ZK_CUDA(cudaEventRecord(side->ntt_done, s3));
  // the H MSM is the largest G1 run (N 16-bit digits): its stage and accumulation timers
  nv_stage.reset();
  nv_stage.emplace("zkvc/prove/msm_h");
  prof_mark(PS_MSM_G1, true, s3);
  ZK_TRY(msm_run<Fp>(P.h, pk->g1, B.ws_h, B.ws_h_bytes, B.res_h, s3, PS_ACCUM_G1, side->h_accum));
  prof_mark(PS_MSM_G1, false, s3);
  ZK_CUDA(cudaEventRecord(side->join[3], s3));
  // the G2 MSM on side stream 0 (at once or after the NTTs, a tuned choice), then the
  // encoding of B
  ZK_CUDA(cudaStreamWaitEvent(side->st[0], side->fork[0], 0));
  if (pk->prove_tune[7] == 1) ZK_CUDA(cudaStreamWaitEvent(side->st[0], side->ntt_done, 0));
  nv_stage.reset();
  nv_stage.emplace("zkvc/prove/msm_g2");
  prof_mark(PS_MSM_G2, true, side->st[0]);
  ZK_TRY(msm_run<Fp2>(P.g2, pk->g2, B.ws2, B.ws2_bytes, B.res2, side->st[0], PS_ACCUM_G2));
  k_encode_b<<<1, 32, 0, side->st[0]>>>(B.res2, B.proof); ZK_COUNT_LAUNCH();
  prof_mark(PS_MSM_G2, false, side->st[0]);
  ZK_CUDA(cudaEventRecord(side->join[0], side->st[0]));
  // the small-digit G1 MSM on side stream 1, then in chain mode the two variable-base
  // multiplications, then the encoding of A and the H-free part of C.  In chain mode it
  // is the side MSM whose start is tuned (at once, after the NTTs, after the H
  // accumulation); in fold mode the rest MSM is.
  ZK_CUDA(cudaStreamWaitEvent(side->st[1], side->fork[1], 0));
  if (chain && pk->prove_tune[5] == 1) ZK_CUDA(cudaStreamWaitEvent(side->st[1], side->ntt_done, 0));
  if (chain && pk->prove_tune[5] == 2) ZK_CUDA(cudaStreamWaitEvent(side->st[1], side->h_accum, 0));
  nv_stage.reset();
  nv_stage.emplace("zkvc/prove/msm_small");
  prof_mark(PS_MSM_SMALL, true, side->st[1]);
  ZK_TRY(msm_run<Fp>(P.small, pk->g1, B.ws_small, B.ws_small_bytes, B.res_small, side->st[1]));
  if (chain) {
    k_chains<<<1, 160, 0, side->st[1]>>>(B.glv, B.res_small, B.res_chain, B.cpart, B.proof); ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaGetLastError());
  } else {
    k_encode_a<<<1, 32, 0, side->st[1]>>>(B.res_small, nullptr, B.cpart, B.proof); ZK_COUNT_LAUNCH();
  }
  prof_mark(PS_MSM_SMALL, false, side->st[1]);
  ZK_CUDA(cudaEventRecord(side->join[1], side->st[1]));
  if (!chain) {
    // the full-scalar G1 terms that need no h, on side stream 2, then their term of C.
    // It starts at once, after the NTTs or after the H accumulation (a tuned choice: its
    // accumulation competes with the critical chain's for the SMs)
    ZK_CUDA(cudaStreamWaitEvent(side->st[2], side->fork[2], 0));
    if (pk->prove_tune[5] == 1) ZK_CUDA(cudaStreamWaitEvent(side->st[2], side->ntt_done, 0));
    if (pk->prove_tune[5] == 2) ZK_CUDA(cudaStreamWaitEvent(side->st[2], side->h_accum, 0));
    ZK_TRY(msm_run<Fp>(P.rest, pk->g1, B.ws_rest, B.ws_rest_bytes, B.res_rest, side->st[2]));
    ZK_CUDA(cudaStreamWaitEvent(side->st[2], side->join[1], 0));
    k_add_into<<<1, 4, 0, side->st[2]>>>(B.cpart, B.res_rest); ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaEventRecord(side->join[2], side->st[2]));
  }
  for (int i = 0; i < NSIDE; i++) {
    if (chain && i == 2) continue;
    ZK_CUDA(cudaStreamWaitEvent(st, side->join[i], 0));
  }
  // 7. encode
  nv_stage.reset();
  nv_stage.emplace("zkvc/prove/encode");
  prof_mark(PS_COMBINE, true, st);
  k_encode_c<<<1, 32, 0, st>>>(B.cpart, B.res_h, B.proof); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  prof_mark(PS_COMBINE, false, st);
  ZK_CUDA(cudaMemcpyAsync(proof_out, B.proof, 256, cudaMemcpyDeviceToHost, st));
  ZK_CUDA(cudaMemcpyAsync(flags_out, B.flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  return ZKVC_OK;
}

int prove_enqueue(const zkvc_pk* pk, int mode, const int8_t* dX, const int8_t* dW, const uint8_t* rs_host,
                  int32_t* dY, void* ws, size_t ws_bytes, uint8_t* proof_out, int* flags_out, cudaStream_t st) {
  return prove_enqueue_impl(pk, mode, dX, dW, rs_host, nullptr, dY, ws, ws_bytes, proof_out, flags_out, st);
}

// Status of a finished proof from its device flags.
int prove_status(int flags) {
  ZK_CHECK(!(flags & 4), ZKVC_EINVAL, "prove: r or s is not a canonical Fr element");
  ZK_CHECK(!(flags & 8), ZKVC_ETIMEOUT, "prove: a tensor-core wait of the witness matmul timed out");
  ZK_CHECK(!(flags & 1), ZKVC_EUNSAT, "prove: the PSQ chain does not close against Y(z)");
  ZK_CHECK(!(flags & 2), ZKVC_EUNSAT, "prove: the quotient has degree N - 1 (QAP not satisfied)");
  return ZKVC_OK;
}

// A proof for a claimed Y (device memory, read only): direct enqueue, no graph.
int prove_claimed(const zkvc_pk* pk, int mode, const int8_t* dX, const int8_t* dW, const uint8_t* rs_host,
                  const int32_t* dY, void* ws, size_t ws_bytes, uint8_t* proof_host, cudaStream_t st) {
  int flags = 0;
  ZK_TRY(prove_enqueue_impl(pk, mode, dX, dW, rs_host, nullptr, const_cast<int32_t*>(dY), ws, ws_bytes, proof_host,
                            &flags, st, true));
  ZK_CUDA(cudaStreamSynchronize(st));
  prof_collect();
  return prove_status(flags);
}

int prove_impl(const zkvc_pk* pk, int mode, const int8_t* dX, const int8_t* dW, const uint8_t* rs_host, int32_t* dY,
               void* ws, size_t ws_bytes, uint8_t* proof_host, cudaStream_t st) {
  int flags = 0;
  ZK_TRY(prove_enqueue(pk, mode, dX, dW, rs_host, dY, ws, ws_bytes, proof_host, &flags, st));
  ZK_CUDA(cudaStreamSynchronize(st));
  prof_collect();
  return prove_status(flags);
}

// ------------------------------------------------------------------ one-proof graph
// zkvc_prove and zkvc_prove_mode replay a CUDA graph of the whole proof (its kernels,
// memsets, copies and the fork/join events of its five streams) once a key is proven
// with the same buffers, mode and tuning on two calls in a row: the first of the two
// runs directly and records the buffers, the second captures the enqueue on a capture
// stream and instantiates it with the streams' priorities kept per node.  A captured copy
// reads its host source again on every replay, so every host source is pinned memory of
// this cache: r, s and their GLV halves (filled by the host before each replay) and the
// MSM runs' table images (constant for the buffers: the tables hold their pointers); the
// proof and the device flags land in pinned memory too.  A change of buffers, mode or
// tuning re-arms the capture; profiling, or another thread proving with the same key at
// the same time, takes the direct path.
struct ProveGraphKey {
  const void* ws;
  size_t ws_bytes;
  const int8_t* dX;
  const int8_t* dW;
  int32_t* dY;
  int mode, dev;
  uint32_t tune[ZKVC_PK_TUNING_LEN];
};

struct ProveGraph {
  std::mutex mu;
  ProveGraphKey key, cand, bad;  // captured; seen on the last call; failed to capture
  bool has_key = false, has_cand = false, has_bad = false;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  unsigned long long launches = 0;  // kernels per replay
  uint8_t* host = nullptr;          // pinned: rs (64 B) | GLV halves | proof (256 B) | flags
  uint8_t* tables = nullptr;        // pinned: the MSM runs' table images (msm_table_stage)
  static constexpr size_t GLV = 64, PROOF = 256, FLAGS = 512, BYTES = 1024, TABLE_BYTES = 256 << 10;
};
static_assert(ProveGraph::GLV + 2 * sizeof(GlvScalar) <= ProveGraph::PROOF, "staging layout");

static ProveGraphKey graph_key(const zkvc_pk* pk, int mode, const int8_t* dX, const int8_t* dW, int32_t* dY,
                               const void* ws, size_t ws_bytes, int dev) {
  ProveGraphKey k;
  std::memset(&k, 0, sizeof k);  // padding included: keys compare bytewise
  k.ws = ws;
  k.ws_bytes = ws_bytes;
  k.dX = dX;
  k.dW = dW;
  k.dY = dY;
  k.mode = mode;
  k.dev = dev;
  std::memcpy(k.tune, pk->prove_tune, sizeof k.tune);
  return k;
}

static bool same_key(const ProveGraphKey& a, const ProveGraphKey& b) { return std::memcmp(&a, &b, sizeof a) == 0; }

static std::mutex g_graph_create;

static ProveGraph* graph_of(const zkvc_pk* pk) {
  std::lock_guard<std::mutex> lock(g_graph_create);
  if (!pk->graph) {
    ProveGraph* g = new (std::nothrow) ProveGraph;
    if (!g) return nullptr;
    if (cudaMallocHost(&g->host, ProveGraph::BYTES) != cudaSuccess ||
        cudaMallocHost(&g->tables, ProveGraph::TABLE_BYTES) != cudaSuccess) {
      cudaGetLastError();
      if (g->host) cudaFreeHost(g->host);
      delete g;
      return nullptr;
    }
    pk->graph = g;
  }
  return pk->graph;
}

// Forgets the captured graph and the candidate buffers (the autotuner's, freed after it).
static void prove_graph_reset(const zkvc_pk* pk) {
  ProveGraph* g = pk->graph;
  if (!g) return;
  std::lock_guard<std::mutex> lock(g->mu);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  g->exec = nullptr;
  g->has_key = g->has_cand = g->has_bad = false;
}

void prove_graph_free(ProveGraph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->cap) cudaStreamDestroy(g->cap);
  if (g->host) cudaFreeHost(g->host);
  if (g->tables) cudaFreeHost(g->tables);
  delete g;
}

static int capture_proof(ProveGraph* g, const zkvc_pk* pk, int mode, const int8_t* dX, const int8_t* dW,
                         int32_t* dY, void* ws, size_t ws_bytes) {
  if (g->exec) {
    ZK_CUDA(cudaGraphExecDestroy(g->exec));
    g->exec = nullptr;
    g->has_key = false;
  }
  if (!g->cap) ZK_CUDA(cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking));
  const unsigned long long before = launches_so_far();
  ZK_CUDA(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
  // every host source of the captured copies is pinned memory of this cache: r and s,
  // their GLV halves, and the MSM tables (constant for the key: their pointers are the
  // key's buffers)
  msm_table_stage(g->tables, ProveGraph::TABLE_BYTES);
  int rc = prove_enqueue_impl(pk, mode, dX, dW, g->host, reinterpret_cast<const GlvScalar*>(g->host + ProveGraph::GLV),
                              dY, ws, ws_bytes, g->host + ProveGraph::PROOF,
                              reinterpret_cast<int*>(g->host + ProveGraph::FLAGS), g->cap);
  msm_table_stage(nullptr, 0);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(g->cap, &graph);
  // the kernels counted while capturing run on every replay, not now
  const unsigned long long n = launches_so_far() - before;
  uncount_launches(n);
  if (rc != ZKVC_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    ZK_TRY(rc);
    ZK_CUDA(e);
  }
  const cudaError_t ie = cudaGraphInstantiateWithFlags(&g->exec, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) g->exec = nullptr;
  ZK_CUDA(ie);
  g->launches = n;
  return ZKVC_OK;
}

int prove_graph(const zkvc_pk* pk, int mode, const int8_t* dX, const int8_t* dW, const uint8_t* rs, int32_t* dY,
                void* ws, size_t ws_bytes, uint8_t* proof, cudaStream_t st) {
  ProveGraph* g = prof_enabled() ? nullptr : graph_of(pk);
  if (!g) return prove_impl(pk, mode, dX, dW, rs, dY, ws, ws_bytes, proof, st);
  std::unique_lock<std::mutex> lock(g->mu, std::try_to_lock);
  if (!lock.owns_lock()) return prove_impl(pk, mode, dX, dW, rs, dY, ws, ws_bytes, proof, st);
  ZK_CHECK(mode == ZKVC_PROVE_FOLD || mode == ZKVC_PROVE_CHAIN, ZKVC_EINVAL, "prove: mode %d", mode);
  int dev = 0;
  ZK_CUDA(cudaGetDevice(&dev));
  const ProveGraphKey k = graph_key(pk, mode, dX, dW, dY, ws, ws_bytes, dev);
  if (!(g->exec && g->has_key && same_key(g->key, k))) {
    if (g->has_bad && same_key(g->bad, k)) return prove_impl(pk, mode, dX, dW, rs, dY, ws, ws_bytes, proof, st);
    if (!(g->has_cand && same_key(g->cand, k))) {
      // a direct proof; its buffers become the candidate if it went through (so that a
      // capture only ever repeats a sequence that has just run)
      const int rc = prove_impl(pk, mode, dX, dW, rs, dY, ws, ws_bytes, proof, st);
      g->cand = k;
      g->has_cand = rc == ZKVC_OK || rc == ZKVC_EUNSAT;
      return rc;
    }
    if (capture_proof(g, pk, mode, dX, dW, dY, ws, ws_bytes) != ZKVC_OK) {
      // not capturable here (the direct path reports any real error): stay direct for
      // these buffers until another key comes along
      cudaGetLastError();
      set_error("%s", "");
      g->bad = k;
      g->has_bad = true;
      return prove_impl(pk, mode, dX, dW, rs, dY, ws, ws_bytes, proof, st);
    }
    g->key = k;
    g->has_key = true;
  }
  std::memcpy(g->host, rs, 64);
  if (mode == ZKVC_PROVE_CHAIN) {
    GlvScalar* h = reinterpret_cast<GlvScalar*>(g->host + ProveGraph::GLV);
    h[0] = glv_split(rs + 32);
    h[1] = glv_split(rs);
  }
  ZK_CUDA(cudaGraphLaunch(g->exec, st));
  count_launches(g->launches);
  ZK_CUDA(cudaStreamSynchronize(st));
  std::memcpy(proof, g->host + ProveGraph::PROOF, 256);
  int flags = 0;
  std::memcpy(&flags, g->host + ProveGraph::FLAGS, sizeof flags);
  return prove_status(flags);
}

// Latency tuning of the one-proof prover (timing replays of the captured proof, as
// zkvc_prove runs it): coordinate descent over the level-0 chunk of
// each MSM run (the G2 and small-scalar runs first: their bucket sums are the longest
// dependent chains), the NTT block and, in fold mode, the start of the rest MSM, timing
// whole proofs with CUDA events on st.  With ZKVC_PROVE_AUTO both modes are tuned and the
// faster one is kept as the key's mode for zkvc_prove.  Proof bytes do not depend on any
// of it.  Allocates its own Y and workspace; the key must not be in use.
int prove_autotune(zkvc_pk* pk, int mode, const int8_t* dX, const int8_t* dW, const uint8_t* rs, cudaStream_t st,
                   uint32_t* chosen) {
  static const uint32_t kCand[] = {2, 4, 8, 16, 32, 64};
  static const uint32_t kElog[] = {8, 9, 10, 11};
  static const uint32_t kRest[] = {0, 1, 2};
  static const uint32_t kBin[] = {0, 1};
  uint32_t saved[ZKVC_PK_TUNING_LEN];
  for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) saved[i] = pk->prove_tune[i];
  for (int i = 0; i < 4; i++) pk->prove_tune[i] = 2;  // the largest workspace of all candidates
  size_t need = std::max(prove_workspace_bytes(pk, ZKVC_PROVE_FOLD), prove_workspace_bytes(pk, ZKVC_PROVE_CHAIN));
  for (int i = 0; i < 4; i++) pk->prove_tune[i] = saved[i];
  void* ws = nullptr;
  int32_t* dY = nullptr;
  void* flush = nullptr;  // written between timed proofs: each starts with a cold L2, as
                          // a served proof's fresh inputs do (and as the bench times it)
  const size_t flush_bytes = size_t(256) << 20;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    cudaFree(ws);
    cudaFree(dY);
    cudaFree(flush);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(&ws, need) != cudaSuccess || cudaMalloc(&dY, size_t(pk->shape.a) * pk->shape.b * 4) != cudaSuccess ||
      cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    set_error("autotune: cannot allocate %zu bytes of workspace", need);
    return ZKVC_ENOMEM;
  }
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cleanup();
    set_error("autotune: event creation failed");
    return ZKVC_ECUDA;
  }
  uint8_t proof[256];
  // median of nine timed proofs after two untimed, as zkvc_prove runs them: the first
  // direct, the second captured, the timed ones replays of the captured graph, each after
  // a write larger than L2
  auto measure = [&](int m, float* ms) -> int {
    float t[9];
    for (int rep = 0; rep < 11; rep++) {
      ZK_CUDA(cudaMemsetAsync(flush, rep & 0xff, flush_bytes, st));
      ZK_CUDA(cudaEventRecord(e0, st));
      ZK_TRY(prove_graph(pk, m, dX, dW, rs, dY, ws, need, proof, st));
      ZK_CUDA(cudaEventRecord(e1, st));
      ZK_CUDA(cudaEventSynchronize(e1));
      if (rep > 1) ZK_CUDA(cudaEventElapsedTime(&t[rep - 2], e0, e1));
    }
    std::sort(t, t + 9);
    *ms = t[4];
    return ZKVC_OK;
  };
  // for one mode, from the key's current setting: first a joint grid over the chunks of
  // the small-digit and G2 runs (side streams that share the SMs with the H path, so the
  // best size of each depends on the other; one knob at a time missed the joint optimum
  // by about 5 %), then coordinate descent over every knob: two sweeps, the incumbent
  // re-timed at the start of each (timings on a shared GPU drift)
  // every timed setting of the current mode, for the confirmation round
  struct Seen {
    float ms;
    std::array<uint32_t, ZKVC_PK_TUNING_LEN> t;
  };
  std::vector<Seen> seen;
  auto timed = [&](int m, float* ms) -> int {
    ZK_TRY(measure(m, ms));
    Seen e;
    e.ms = *ms;
    for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) e.t[i] = pk->prove_tune[i];
    seen.push_back(e);
    return ZKVC_OK;
  };
  auto tune = [&](int m, float* best_ms) -> int {
    seen.clear();
    {
      ZK_TRY(timed(m, best_ms));
      uint32_t bs = pk->prove_tune[0], bg = pk->prove_tune[3];
      for (int i = -1; i < 6; i++) {
        for (int j = -1; j < 6; j++) {
          const uint32_t cs = i < 0 ? 0u : kCand[i], cg = j < 0 ? 0u : kCand[j];
          if (cs == bs && cg == bg) continue;
          pk->prove_tune[0] = cs;
          pk->prove_tune[3] = cg;
          float ms = 0;
          ZK_TRY(timed(m, &ms));
          if (ms < 0.99f * *best_ms) {
            *best_ms = ms;
            bs = cs;
            bg = cg;
          }
        }
      }
      pk->prove_tune[0] = bs;
      pk->prove_tune[3] = bg;
    }
    const int order[4] = {3, 0, 2, 1};  // g2, small, h, rest
    for (int sweep = 0; sweep < 2; sweep++) {
    ZK_TRY(timed(m, best_ms));
    for (int oi = 0; oi < 9; oi++) {
      // then the NTT block, the side MSM's start, the G2 MSM's start, quads for the H and
      // small-digit accumulations (index 6 is the mode)
      const int r = oi < 4 ? order[oi] : oi < 6 ? oi : oi + 1;
      const uint32_t* cand = r < 4 ? kCand : r == 4 ? kElog : r == 5 ? kRest : kBin;
      const int ncand = r < 4 ? 6 : r == 4 ? 4 : r == 5 ? 3 : 2;
      uint32_t best = pk->prove_tune[r];
      for (int ci = 0; ci < ncand; ci++) {
        const uint32_t c = cand[ci];
        if (c == best || (r == 4 && best == 0 && c == 10)) continue;
        pk->prove_tune[r] = c;
        float ms = 0;
        ZK_TRY(timed(m, &ms));
        if (ms < 0.99f * *best_ms) {  // a gain within timing noise does not move the setting
          *best_ms = ms;
          best = c;
        }
      }
      pk->prove_tune[r] = best;
    }
    }
    // confirmation: the four fastest distinct settings seen, each timed twice more; the
    // lowest mean of three medians wins (one median of nine proofs drifts by a few per
    // cent between calls, which is as much as the knobs' differences near the optimum)
    std::sort(seen.begin(), seen.end(), [](const Seen& x, const Seen& y) { return x.ms < y.ms; });
    std::vector<Seen> top;
    for (const Seen& e : seen) {
      bool dup = false;
      for (const Seen& t : top) dup = dup || t.t == e.t;
      if (!dup) top.push_back(e);
      if (top.size() == 4) break;
    }
    float best_mean = 1e30f;
    std::array<uint32_t, ZKVC_PK_TUNING_LEN> pick = top.empty() ? std::array<uint32_t, ZKVC_PK_TUNING_LEN>{} : top[0].t;
    for (const Seen& e : top) {
      for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) pk->prove_tune[i] = e.t[i];
      float a = 0, b = 0;
      ZK_TRY(measure(m, &a));
      ZK_TRY(measure(m, &b));
      const float mean = (e.ms + a + b) / 3;
      if (mean < best_mean) {
        best_mean = mean;
        pick = e.t;
      }
    }
    if (!top.empty()) {
      for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) pk->prove_tune[i] = pick[i];
      *best_ms = best_mean;
    }
    return ZKVC_OK;
  };
  int rc = ZKVC_OK;
  if (mode == ZKVC_PROVE_AUTO) {
    float fold_ms = 0, chain_ms = 0;
    uint32_t fold_tune[ZKVC_PK_TUNING_LEN];
    rc = tune(ZKVC_PROVE_FOLD, &fold_ms);
    for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) fold_tune[i] = pk->prove_tune[i];
    if (rc == ZKVC_OK) {
      for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) pk->prove_tune[i] = saved[i];
      rc = tune(ZKVC_PROVE_CHAIN, &chain_ms);
    }
    if (rc == ZKVC_OK) {
      if (fold_ms <= chain_ms)
        for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) pk->prove_tune[i] = fold_tune[i];
      pk->prove_tune[6] = fold_ms <= chain_ms ? ZKVC_PROVE_FOLD : ZKVC_PROVE_CHAIN;
    }
  } else {
    float ms = 0;
    rc = tune(mode, &ms);
    if (rc == ZKVC_OK) pk->prove_tune[6] = (uint32_t)mode;
  }
  prove_graph_reset(pk);
  cleanup();
  if (rc != ZKVC_OK) {
    for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) pk->prove_tune[i] = saved[i];
    return rc;
  }
  if (chosen)
    for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) chosen[i] = pk->prove_tune[i];
  return ZKVC_OK;
}

}  // namespace zkvc
