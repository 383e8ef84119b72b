// Batched Groth16 proving: many CRPC + PSQ matmul proofs of uneven shapes (zkVC Sec. III,
// the [tokens, dim1] x [dim1, dim2] layers of Sec. V) in one persistent launch sequence
// that is captured once as a CUDA graph and replayed.
//
// Per call the sequence runs, for all instances at once:
//   witness   one launch per step over every instance (blockIdx.y/z = instance): Y = X W,
//             the CRPC sums a_k, b_k, Y(z), the PSQ chain and the domain evaluations;
//   NTTs      instances are grouped by domain size N; each group's 3m INTTs, 3m coset
//             NTTs, quotient and m coset INTTs are single batched launches;
//   MSMs      three merged multi-instance runs, keyed (instance, bucket) with each
//             output reading its own proving key's bases:
//               small (G1, 8-bit digits): per instance A, the L-query part over W
//                 (sum_k b_k [alpha L_k / delta]1) and B1 = [beta]1 + sum_k b_k [L_k]1 +
//                 s [delta]1 -- the W side through the CRPC sums over n per-row points;
//               main  (G1, 16-bit digits over the stored 2^(16 w) multiples): L over the
//                 prefix sums, the H query (h_j), and -r s [delta]1;
//               g2    (8-bit digits): B = [beta]2 + sum_k b_k [L_k]2 + s [delta]2;
//   C         = L_W + main + s A + r B1 (Groth16's C = ... + s A + r B - r s delta);
// (The G2 run starts once the CRPC sums b_k exist.)
//             s A and r B1 are 254-bit variable-base multiplications, one thread each,
//             overlapping the main run.  (The one-proof prover folds them into
//             fixed-base terms instead, which is shorter in latency but moves 16 extra
//             digits per witness entry into the MSM; batched, throughput decides.)
//   encode    affine conversion and the 256-byte encodings.
// The G2 run and the small run (+ the two multiplications) sit on two side streams that
// fork from and join the capture stream.
//
// An optional autotuner (first call) times candidate chunk sizes and block sizes of each
// MSM run and the NTT block size on the batch's own data, keeps the fastest, and only
// then captures the graph.
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "groth16.h"
#include "matmul_tc.cuh"
#include "msm.h"
#include "witness.cuh"

namespace zkvc {

struct BInst {
  const int8_t* X;
  const int8_t* W;
  int32_t* Y;
  const Fr* zA;
  const Fr* zB;
  Fr *ak, *bk, *yz, *S;
  Fr *Aev, *Bev, *Cev, *Hev;
  Fr* rs;    // r, s (canonical, from the caller)
  Fr* nrs;   // -r s (canonical)
  int* flags;
  int a, n, b;
  uint32_t l;
  uint32_t N;
};

// ------------------------------------------------------------------ batched kernels
__global__ void k_b_randomness(const BInst* __restrict__ I, int count) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const BInst in = I[t];
  Fr r = ld_field(in.rs), s = ld_field(in.rs + 1);
  if (!canonical_fr(r) || !canonical_fr(s)) atomicOr(in.flags, 4);
  st_field(in.nrs, f_neg(f_mul(f_to_mont(r), s)));  // (r R) s / R = r s, negated mod r
}

// the witness matmul of every instance on the tensor cores (matmul_tc.cuh)
__global__ void __launch_bounds__(MM_THREADS) k_b_matmul(const BInst* __restrict__ I) {
  extern __shared__ __align__(128) uint8_t mm_dyn[];
  MatmulSmem& sm = *reinterpret_cast<MatmulSmem*>(mm_dyn);
  const BInst& in = I[blockIdx.z];
  const int a = in.a, b = in.b;
  if ((int)blockIdx.x * MM_M >= b || (int)blockIdx.y * MM_N >= a) return;  // uniform per block
  matmul_tc_tile(in.X, in.W, in.Y, a, in.n, b, blockIdx.x * MM_M, blockIdx.y * MM_N, 0, in.n, false, sm, in.flags);
}

static std::once_flag g_bmm_once;
static void b_matmul_init() {
  std::call_once(g_bmm_once, [] {
    cudaFuncSetAttribute(k_b_matmul, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MatmulSmem));
  });
}

__global__ void __launch_bounds__(256) k_b_crpc_ab(const BInst* __restrict__ I) {
  __shared__ Fr sh[256];
  const BInst& in = I[blockIdx.y];
  if ((int)blockIdx.x >= in.n) return;
  crpc_ab_row(in.X, in.W, in.zA, in.zB, in.a, in.n, in.b, blockIdx.x, in.ak, in.bk, sh);
}

__global__ void __launch_bounds__(256) k_b_crpc_y(const BInst* __restrict__ I) {
  __shared__ Fr sh[256];
  const BInst& in = I[blockIdx.y];
  if ((int)blockIdx.x >= in.a) return;
  crpc_y_row(in.Y, in.zA, in.zB, in.b, blockIdx.x, in.yz, sh);
}

__global__ void __launch_bounds__(1024) k_b_psq(const BInst* __restrict__ I) {
  __shared__ Fr sh[1024];
  const BInst& in = I[blockIdx.x];
  psq_chain(in.ak, in.bk, in.yz, in.a, in.n, in.S, in.Aev, in.Bev, in.Cev, in.flags, sh);
}

__global__ void k_b_domain_rest(const BInst* __restrict__ I) {
  const BInst& in = I[blockIdx.y];
  size_t k = in.n + size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= in.N) return;
  domain_rest_row(in.X, in.Y, in.n, uint32_t(in.a) * in.n, in.l, k, in.Aev, in.Bev, in.Cev);
}

__global__ void k_b_check_h(const BInst* __restrict__ I, int count) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const BInst& in = I[t];
  if (!ld_field(in.Hev + (in.N - 1)).is_zero()) atomicOr(in.flags, 2);
}

// thread 2i: s A_i; thread 2i + 1: r B1_i (small-run outputs 3i and 3i + 2)
__global__ void __launch_bounds__(64) k_b_chains(const BInst* __restrict__ I, int count, const G1J* __restrict__ small,
                                                 G1J* chain) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * count) return;
  const int i = t >> 1, which = t & 1;
  const G1J P = ld_field(small + 3 * i + (which ? 2 : 0));
  const Fr k = ld_field(I[i].rs + (which ? 0 : 1));
  uint32_t kk[8];
#pragma unroll
  for (int l = 0; l < 8; l++) kk[l] = k.v[l];
  st_field(chain + t, p_mul_scalar_w4(P, kk));
}

// block i: A = small[3i]; C = small[3i + 1] + main[i] + s A + r B1; B = g2[i]
__global__ void k_b_encode(const G1J* __restrict__ small, const G1J* __restrict__ mainr, const G1J* __restrict__ chain,
                           const G2J* __restrict__ g2, uint8_t* proofs) {
  const int i = blockIdx.x;
  if (threadIdx.x == 0) {
    G1J A = ld_field(small + 3 * i);
    G1J C = p_add(p_add(ld_field(small + 3 * i + 1), ld_field(mainr + i)),
                  p_add(ld_field(chain + 2 * i), ld_field(chain + 2 * i + 1)));
    encode_a_c(A, C, proofs + size_t(i) * 256);
  } else if (threadIdx.x == 32) {
    encode_b(ld_field(g2 + i), proofs + size_t(i) * 256);
  }
}

// ------------------------------------------------------------------ the batch object
struct BatchTune {
  MsmTune small, main, g2;
  int elog = 10;
};

struct NttGroup {
  const NttDomain* d = nullptr;
  size_t N = 0;
  int m = 0;
  Fr* ev = nullptr;  // [A_0..A_(m-1) | B_.. | C_.. | H_..], N each
};

}  // namespace zkvc

using namespace zkvc;

struct zkvc_batch {
  int device = 0;
  int count = 0;
  int flags = 0;
  std::vector<const zkvc_pk*> pks;
  // device memory (one allocation)
  uint8_t* mem = nullptr;
  size_t mem_bytes = 0;
  int8_t *X = nullptr, *W = nullptr;
  int32_t* Y = nullptr;
  std::vector<size_t> xo, wo, yo;  // per-instance offsets (elements)
  BInst* dinst = nullptr;
  std::vector<BInst> hinst;
  Fr* rs = nullptr;                // count x 2
  Fr* nrs = nullptr;               // count
  int* dflags = nullptr;           // count
  G1J *res_small = nullptr, *res_main = nullptr, *chain = nullptr;
  G2J* res_g2 = nullptr;
  uint8_t* dproofs = nullptr;
  std::vector<NttGroup> groups;
  MsmPlan p_small, p_main, p_g2;
  MsmExec x_small, x_main, x_g2;
  void *ws_small = nullptr, *ws_main = nullptr, *ws_g2 = nullptr;
  size_t ws_small_bytes = 0, ws_main_bytes = 0, ws_g2_bytes = 0;
  BatchTune tune;
  bool tuned = false;
  // pinned host staging
  uint8_t* h_rs = nullptr;      // count x 64
  int* h_flags = nullptr;       // count
  uint8_t* h_proofs = nullptr;  // count x 256
  // streams and events
  cudaStream_t cap = nullptr, side[2] = {nullptr, nullptr};
  cudaEvent_t fork[2] = {nullptr, nullptr}, join[2] = {nullptr, nullptr}, ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t graph = nullptr;
  unsigned long long graph_launches = 0;
  bool busy = false;  // a previous call timed out with work in flight
  bool owns_mem = true;  // false for the proof server's transient batches
  int cap_count = 0;     // instances the pinned staging holds
  ~zkvc_batch();
};

zkvc_batch::~zkvc_batch() {
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(device);
  if (cap) cudaStreamSynchronize(cap);
  if (graph) cudaGraphExecDestroy(graph);
  for (int i = 0; i < 2; i++) {
    if (side[i]) cudaStreamDestroy(side[i]);
    if (fork[i]) cudaEventDestroy(fork[i]);
    if (join[i]) cudaEventDestroy(join[i]);
  }
  if (ev_in) cudaEventDestroy(ev_in);
  if (ev_out) cudaEventDestroy(ev_out);
  if (cap) cudaStreamDestroy(cap);
  if (mem && owns_mem) cudaFree(mem);
  if (h_rs) cudaFreeHost(h_rs);
  if (h_flags) cudaFreeHost(h_flags);
  if (h_proofs) cudaFreeHost(h_proofs);
  if (cur >= 0) cudaSetDevice(cur);
}

namespace zkvc {

// The candidates the autotuner tries; workspaces are sized for the smallest chunk.
static const uint32_t kChunkG1[] = {8, 16, 32, 64, 128, 256};
static const uint32_t kChunkG2[] = {8, 16, 32};
static const uint32_t kAccumG1[] = {64, 128, 256};
static const uint32_t kAccumG2[] = {64, 128};
static const int kElog[] = {9, 10, 11};

static MsmSeg bseg(const Region& r, uint32_t first, uint32_t count, uint32_t out, int kind, const void* sc,
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

static void batch_plans(zkvc_batch* B) {
  B->p_small = MsmPlan();
  B->p_main = MsmPlan();
  B->p_g2 = MsmPlan();
  for (int i = 0; i < B->count; i++) {
    const zkvc_pk* pk = B->pks[i];
    const Shape& sh = pk->shape;
    const Region* g = pk->lay.g1;
    const Region* g2 = pk->lay.g2;
    const BInst& in = B->hinst[i];
    const uint32_t an = sh.a * sh.n, ab = sh.a * sh.b;
    const uint32_t o = 3 * i;
    for (int q = 0; q < 3; q++) B->p_small.outs.push_back({8, 1, 0, 0, pk->g1});
    auto& s = B->p_small.segs;
    s.push_back(bseg(g[R1_AIN], 0, 1, o, SK_ONE, nullptr));
    s.push_back(bseg(g[R1_AIN], 1, an, o, SK_I8, in.X));
    s.push_back(bseg(g[R1_AY8], 0, ab, o, SK_I32, in.Y));
    s.push_back(bseg(g[R1_ALPHA], 0, 1, o, SK_ONE, nullptr));
    s.push_back(bseg(g[R1_DELTA8], 0, 1, o, SK_FR_CANON, in.rs + 0));
    s.push_back(bseg(g[R1_LK], 0, (uint32_t)sh.n, o, SK_FR_MONT, in.ak));
    s.push_back(bseg(g[R1_ALK], 0, (uint32_t)sh.n, o + 1, SK_FR_MONT, in.bk));
    s.push_back(bseg(g[R1_LK], 0, (uint32_t)sh.n, o + 2, SK_FR_MONT, in.bk));
    s.push_back(bseg(g[R1_BETA], 0, 1, o + 2, SK_ONE, nullptr));
    s.push_back(bseg(g[R1_DELTA8], 0, 1, o + 2, SK_FR_CANON, in.rs + 1));

    B->p_main.outs.push_back({ZKVC_C1, 1, 0, 0, pk->g1});
    auto& m = B->p_main.segs;
    m.push_back(bseg(g[R1_LS], 0, (uint32_t)(sh.n - 1), i, SK_FR_MONT, in.S));
    m.push_back(bseg(g[R1_H], 0, (uint32_t)sh.N, i, SK_FR_MONT, in.Hev, (uint32_t)sh.N - 1));
    m.push_back(bseg(g[R1_DELTA], 0, 1, i, SK_FR_CANON, in.nrs));

    B->p_g2.outs.push_back({ZKVC_C2, 1, 0, 0, pk->g2});
    auto& t = B->p_g2.segs;
    t.push_back(bseg(g2[R2_LK], 0, (uint32_t)sh.n, i, SK_FR_MONT, in.bk));
    t.push_back(bseg(g2[R2_BETA], 0, 1, i, SK_ONE, nullptr));
    t.push_back(bseg(g2[R2_DELTA], 0, 1, i, SK_FR_CANON, in.rs + 1));
  }
}

// Carves (or measures) every device buffer of the batch.  Workspaces of the MSM runs are
// sized for the smallest candidate chunk, so any tuning fits.
static size_t carve(zkvc_batch* B, bool measuring) {
  Arena a;
  a.base = B->mem;
  a.cap = B->mem_bytes;
  a.measuring = measuring;
  const int n = B->count;
  size_t xs = 0, ws = 0, ys = 0;
  B->xo.assign(n, 0);
  B->wo.assign(n, 0);
  B->yo.assign(n, 0);
  for (int i = 0; i < n; i++) {
    const Shape& sh = B->pks[i]->shape;
    B->xo[i] = xs;
    B->wo[i] = ws;
    B->yo[i] = ys;
    xs += (size_t(sh.a) * sh.n + 15) & ~size_t(15);
    ws += (size_t(sh.n) * sh.b + 15) & ~size_t(15);
    ys += (size_t(sh.a) * sh.b + 3) & ~size_t(3);
  }
  B->X = a.take<int8_t>(xs);
  B->W = a.take<int8_t>(ws);
  B->Y = a.take<int32_t>(ys);
  B->dinst = a.take<BInst>(n);
  B->rs = a.take<Fr>(2 * size_t(n));
  B->nrs = a.take<Fr>(n);
  B->dflags = a.take<int>(n);
  B->res_small = a.take<G1J>(3 * size_t(n));
  B->res_main = a.take<G1J>(n);
  B->chain = a.take<G1J>(2 * size_t(n));
  B->res_g2 = a.take<G2J>(n);
  B->dproofs = a.take<uint8_t>(256 * size_t(n));
  // NTT groups by domain size
  std::map<uint32_t, std::vector<int>> by_log;
  for (int i = 0; i < n; i++) by_log[B->pks[i]->shape.logN].push_back(i);
  B->groups.clear();
  B->hinst.assign(n, BInst{});
  for (auto& kv : by_log) {
    NttGroup gr;
    gr.N = size_t(1) << kv.first;
    gr.m = (int)kv.second.size();
    gr.d = B->pks[kv.second[0]]->dom;
    gr.ev = a.take<Fr>(4 * gr.N * gr.m);
    for (int j = 0; j < gr.m; j++) {
      BInst& in = B->hinst[kv.second[j]];
      in.Aev = gr.ev ? gr.ev + size_t(j) * gr.N : nullptr;
      in.Bev = gr.ev ? gr.ev + size_t(gr.m + j) * gr.N : nullptr;
      in.Cev = gr.ev ? gr.ev + size_t(2 * gr.m + j) * gr.N : nullptr;
      in.Hev = gr.ev ? gr.ev + size_t(3 * gr.m + j) * gr.N : nullptr;
    }
    B->groups.push_back(gr);
  }
  for (int i = 0; i < n; i++) {
    const zkvc_pk* pk = B->pks[i];
    const Shape& sh = pk->shape;
    BInst& in = B->hinst[i];
    in.X = B->X ? B->X + B->xo[i] : nullptr;
    in.W = B->W ? B->W + B->wo[i] : nullptr;
    in.Y = B->Y ? B->Y + B->yo[i] : nullptr;
    in.zA = pk->zA;
    in.zB = pk->zB;
    in.ak = a.take<Fr>(sh.n);
    in.bk = a.take<Fr>(sh.n);
    in.yz = a.take<Fr>(sh.a);
    in.S = a.take<Fr>(sh.n);
    in.rs = B->rs ? B->rs + 2 * i : nullptr;
    in.nrs = B->nrs ? B->nrs + i : nullptr;
    in.flags = B->dflags ? B->dflags + i : nullptr;
    in.a = sh.a;
    in.n = sh.n;
    in.b = sh.b;
    in.l = sh.l;
    in.N = (uint32_t)sh.N;
  }
  batch_plans(B);
  MsmPlan ps = B->p_small, pm = B->p_main, pg = B->p_g2;
  ps.tune.chunk = kChunkG1[0];
  pm.tune.chunk = kChunkG1[0];
  pg.tune.chunk = kChunkG2[0];
  msm_plan_finalize(ps);
  msm_plan_finalize(pm);
  msm_plan_finalize(pg);
  B->ws_small_bytes = msm_workspace_bytes<Fp>(ps);
  B->ws_main_bytes = msm_workspace_bytes<Fp>(pm);
  B->ws_g2_bytes = msm_workspace_bytes<Fp2>(pg);
  B->ws_small = a.take<uint8_t>(B->ws_small_bytes);
  B->ws_main = a.take<uint8_t>(B->ws_main_bytes);
  B->ws_g2 = a.take<uint8_t>(B->ws_g2_bytes);
  return a.off;
}

static int prepare_execs(zkvc_batch* B, cudaStream_t st) {
  B->p_small.tune = B->tune.small;
  B->p_main.tune = B->tune.main;
  B->p_g2.tune = B->tune.g2;
  ZK_TRY(msm_plan_finalize(B->p_small));
  ZK_TRY(msm_plan_finalize(B->p_main));
  ZK_TRY(msm_plan_finalize(B->p_g2));
  ZK_TRY(msm_prepare<Fp>(B->p_small, B->ws_small, B->ws_small_bytes, &B->x_small));
  ZK_TRY(msm_prepare<Fp>(B->p_main, B->ws_main, B->ws_main_bytes, &B->x_main));
  ZK_TRY(msm_prepare<Fp2>(B->p_g2, B->ws_g2, B->ws_g2_bytes, &B->x_g2));
  ZK_TRY(msm_upload(&B->x_small, st));
  ZK_TRY(msm_upload(&B->x_main, st));
  ZK_TRY(msm_upload(&B->x_g2, st));
  return ZKVC_OK;
}

static int run_ntts(zkvc_batch* B, cudaStream_t st) {
  for (const NttGroup& gr : B->groups) {
    const size_t N = gr.N;
    const int m = gr.m;
    ZK_TRY(ntt_quotient_chain(gr.ev, m, N, gr.d, st, B->tune.elog));
  }
  return ZKVC_OK;
}

// The whole launch sequence on B->cap (captured, or run eagerly while tuning).
static int enqueue(zkvc_batch* B) {
  cudaStream_t st = B->cap;
  const int n = B->count;
  int maxa = 0, maxn = 0, maxb = 0;
  size_t maxrest = 0;
  for (const BInst& in : B->hinst) {
    maxa = std::max(maxa, in.a);
    maxn = std::max(maxn, in.n);
    maxb = std::max(maxb, in.b);
    maxrest = std::max(maxrest, size_t(in.N) - in.n);
  }
  ZK_CUDA(cudaMemsetAsync(B->dflags, 0, n * sizeof(int), st));
  ZK_CUDA(cudaMemcpyAsync(B->rs, B->h_rs, size_t(n) * 64, cudaMemcpyHostToDevice, st));
  k_b_randomness<<<(n + 63) / 64, 64, 0, st>>>(B->dinst, n); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  // witness
  b_matmul_init();
  k_b_matmul<<<dim3((maxb + MM_M - 1) / MM_M, (maxa + MM_N - 1) / MM_N, n), MM_THREADS, sizeof(MatmulSmem), st>>>(
      B->dinst);
  ZK_COUNT_LAUNCH();
  k_b_crpc_ab<<<dim3(maxn, n), 256, 0, st>>>(B->dinst); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  // G2 run on side stream 0 (needs b_k and s)
  ZK_CUDA(cudaEventRecord(B->fork[0], st));
  ZK_CUDA(cudaStreamWaitEvent(B->side[0], B->fork[0], 0));
  ZK_TRY(msm_launch<Fp2>(&B->x_g2, nullptr, B->res_g2, B->side[0]));
  ZK_CUDA(cudaEventRecord(B->join[0], B->side[0]));
  k_b_crpc_y<<<dim3(maxa, n), 256, 0, st>>>(B->dinst); ZK_COUNT_LAUNCH();
  k_b_psq<<<n, 1024, 0, st>>>(B->dinst); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  // small run and the two variable-base multiplications on side stream 1
  ZK_CUDA(cudaEventRecord(B->fork[1], st));
  ZK_CUDA(cudaStreamWaitEvent(B->side[1], B->fork[1], 0));
  ZK_TRY(msm_launch<Fp>(&B->x_small, nullptr, B->res_small, B->side[1]));
  k_b_chains<<<(2 * n + 63) / 64, 64, 0, B->side[1]>>>(B->dinst, n, B->res_small, B->chain); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  ZK_CUDA(cudaEventRecord(B->join[1], B->side[1]));
  // domain evaluations, NTTs, main run
  k_b_domain_rest<<<dim3((unsigned)((maxrest + 255) / 256), n), 256, 0, st>>>(B->dinst); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  ZK_TRY(run_ntts(B, st));
  k_b_check_h<<<(n + 63) / 64, 64, 0, st>>>(B->dinst, n); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  ZK_TRY(msm_launch<Fp>(&B->x_main, nullptr, B->res_main, st));
  ZK_CUDA(cudaStreamWaitEvent(st, B->join[0], 0));
  ZK_CUDA(cudaStreamWaitEvent(st, B->join[1], 0));
  k_b_encode<<<n, 64, 0, st>>>(B->res_small, B->res_main, B->chain, B->res_g2, B->dproofs); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  ZK_CUDA(cudaMemcpyAsync(B->h_proofs, B->dproofs, size_t(n) * 256, cudaMemcpyDeviceToHost, st));
  ZK_CUDA(cudaMemcpyAsync(B->h_flags, B->dflags, size_t(n) * sizeof(int), cudaMemcpyDeviceToHost, st));
  return ZKVC_OK;
}

static int capture(zkvc_batch* B) {
  if (B->graph) {
    ZK_CUDA(cudaGraphExecDestroy(B->graph));
    B->graph = nullptr;
  }
  const unsigned long long before = launches_so_far();
  ZK_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue(B);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(B->cap, &g);
  if (rc != ZKVC_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  ZK_CUDA(e);
  // the kernels counted while capturing run on every replay, not now
  B->graph_launches = launches_so_far() - before;
  uncount_launches(B->graph_launches);
  cudaError_t ie = cudaGraphInstantiate(&B->graph, g, 0);
  cudaGraphDestroy(g);
  ZK_CUDA(ie);
  return ZKVC_OK;
}

// Times one stage (median of three after one warm-up) on the capture stream.
template <class Fn>
static int time_stage(zkvc_batch* B, Fn fn, float* ms_out) {
  cudaEvent_t e0, e1;
  ZK_CUDA(cudaEventCreate(&e0));
  ZK_CUDA(cudaEventCreate(&e1));
  float best[3];
  int rc = ZKVC_OK;
  for (int rep = 0; rep < 4 && rc == ZKVC_OK; rep++) {
    cudaEventRecord(e0, B->cap);
    rc = fn();
    cudaEventRecord(e1, B->cap);
    if (rc == ZKVC_OK) rc = wait_stream(B->cap, "batch autotune");
    float ms = 0;
    if (rc == ZKVC_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = ZKVC_ECUDA;
    if (rep > 0) best[rep - 1] = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ZK_TRY(rc);
  std::sort(best, best + 3);
  *ms_out = best[1];
  return ZKVC_OK;
}

// Coordinate descent over the launch-shape knobs, each timed on the batch's own inputs
// (already staged by one eager run of the whole sequence).  The results do not depend on
// these knobs, only the time does.
static int autotune(zkvc_batch* B) {
  ZK_TRY(prepare_execs(B, B->cap));
  ZK_TRY(enqueue(B));
  ZK_TRY(wait_stream(B->cap, "batch autotune"));
  struct Knob {
    MsmPlan* plan;
    MsmExec* ex;
    MsmTune* tune;
    bool g2;
    void* ws;
    size_t ws_bytes;
    void* res;
  };
  Knob knobs[3] = {{&B->p_main, &B->x_main, &B->tune.main, false, B->ws_main, B->ws_main_bytes, B->res_main},
                   {&B->p_small, &B->x_small, &B->tune.small, false, B->ws_small, B->ws_small_bytes, B->res_small},
                   {&B->p_g2, &B->x_g2, &B->tune.g2, true, B->ws_g2, B->ws_g2_bytes, B->res_g2}};
  for (Knob& k : knobs) {
    auto trial = [&](const MsmTune& t, float* ms) -> int {
      k.plan->tune = t;
      ZK_TRY(msm_plan_finalize(*k.plan));
      if (k.g2)
        ZK_TRY(msm_prepare<Fp2>(*k.plan, k.ws, k.ws_bytes, k.ex));
      else
        ZK_TRY(msm_prepare<Fp>(*k.plan, k.ws, k.ws_bytes, k.ex));
      ZK_TRY(msm_upload(k.ex, B->cap));
      return time_stage(B, [&]() -> int {
        if (k.g2) return msm_launch<Fp2>(k.ex, nullptr, (G2J*)k.res, B->cap);
        return msm_launch<Fp>(k.ex, nullptr, (G1J*)k.res, B->cap);
      }, ms);
    };
    MsmTune best = *k.tune;
    float best_ms = 1e30f;
    const uint32_t* chunks = k.g2 ? kChunkG2 : kChunkG1;
    const int nchunks = k.g2 ? (int)(sizeof(kChunkG2) / sizeof(kChunkG2[0]))
                             : (int)(sizeof(kChunkG1) / sizeof(kChunkG1[0]));
    for (int c = 0; c < nchunks; c++) {
      MsmTune t = best;
      t.chunk = chunks[c];
      float ms;
      ZK_TRY(trial(t, &ms));
      if (ms < best_ms) { best_ms = ms; best = t; }
    }
    const uint32_t* accs = k.g2 ? kAccumG2 : kAccumG1;
    const int naccs = k.g2 ? 2 : 3;
    for (int c = 0; c < naccs; c++) {
      if (accs[c] == best.accum_threads) continue;
      MsmTune t = best;
      t.accum_threads = accs[c];
      float ms;
      ZK_TRY(trial(t, &ms));
      if (ms < best_ms) { best_ms = ms; best = t; }
    }
    *k.tune = best;
  }
  // NTT block size (the sequence transforms the evaluation buffers in place; the graph
  // recomputes them from the inputs afterwards)
  int best_elog = B->tune.elog;
  float best_ms = 1e30f;
  for (int e : kElog) {
    B->tune.elog = e;
    float ms;
    ZK_TRY(time_stage(B, [&]() -> int { return run_ntts(B, B->cap); }, &ms));
    if (ms < best_ms) { best_ms = ms; best_elog = e; }
  }
  B->tune.elog = best_elog;
  ZK_TRY(prepare_execs(B, B->cap));
  ZK_TRY(wait_stream(B->cap, "batch autotune"));
  B->tuned = true;
  return ZKVC_OK;
}

// Streams, events and pinned staging for up to cap instances.
static int batch_resources(zkvc_batch* B, int cap) {
  ZK_CUDA(cudaMallocHost(&B->h_rs, size_t(cap) * 64));
  ZK_CUDA(cudaMallocHost(&B->h_flags, size_t(cap) * sizeof(int)));
  ZK_CUDA(cudaMallocHost(&B->h_proofs, size_t(cap) * 256));
  std::memset(B->h_rs, 0, size_t(cap) * 64);
  B->cap_count = cap;
  ZK_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
  int lo = 0, hi = 0;
  ZK_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  for (int i = 0; i < 2; i++) {
    ZK_CUDA(cudaStreamCreateWithPriority(&B->side[i], cudaStreamNonBlocking, hi));
    ZK_CUDA(cudaEventCreateWithFlags(&B->fork[i], cudaEventDisableTiming));
    ZK_CUDA(cudaEventCreateWithFlags(&B->join[i], cudaEventDisableTiming));
  }
  ZK_CUDA(cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming));
  ZK_CUDA(cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming));
  return ZKVC_OK;
}

// Per-instance status codes from the device flags (bit 2: r or s not canonical; bit 3: a
// tensor-core wait timed out; bits 0-1: unsatisfied constraints); returns the first
// failing instance (-1: none) and its flags.
static int decode_flags(const int* flags, int n, int* status, int* first_flag) {
  int first_bad = -1;
  *first_flag = 0;
  for (int i = 0; i < n; i++) {
    const int f = flags[i];
    const int code = (f & 4) ? ZKVC_EINVAL : (f & 8) ? ZKVC_ETIMEOUT : (f & 3) ? ZKVC_EUNSAT : ZKVC_OK;
    if (status) status[i] = code;
    if (code != ZKVC_OK && first_bad < 0) {
      first_bad = i;
      *first_flag = f;
    }
  }
  return first_bad;
}

static int batch_create(const zkvc_pk* const* pks, int count, int flags, zkvc_batch** out) {
  ZK_CHECK(pks && out, ZKVC_EINVAL, "batch: null argument");
  b_matmul_init();  // before any capture
  ZK_CHECK(count >= 1 && count <= 4096, ZKVC_EINVAL, "batch: %d instances outside [1, 4096]", count);
  ZK_CHECK((flags & ~(ZKVC_BATCH_AUTOTUNE | ZKVC_BATCH_EAGER)) == 0, ZKVC_EINVAL, "batch: unknown flags 0x%x", flags);
  int dev = 0;
  ZK_CUDA(cudaGetDevice(&dev));
  for (int i = 0; i < count; i++) {
    ZK_CHECK(pks[i], ZKVC_EINVAL, "batch: key %d is null", i);
    ZK_CHECK(!pks[i]->gen, ZKVC_EINVAL, "batch: key %d is a zkvc_setup_circuit key (only CRPC + PSQ keys batch)", i);
    ZK_CHECK(pks[i]->device == dev, ZKVC_EINVAL, "batch: key %d lives on device %d, current is %d", i,
             pks[i]->device, dev);
  }
  zkvc_batch* B = new zkvc_batch();
  B->device = dev;
  B->count = count;
  B->flags = flags;
  B->pks.assign(pks, pks + count);
  int rc = [&]() -> int {
    B->mem_bytes = carve(B, true);
    cudaError_t e = cudaMalloc(&B->mem, B->mem_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      B->mem = nullptr;
      set_error("batch: cannot allocate %zu bytes of device memory", B->mem_bytes);
      return ZKVC_ENOMEM;
    }
    carve(B, false);
    ZK_TRY(batch_resources(B, count));
    ZK_CUDA(cudaMemcpyAsync(B->dinst, B->hinst.data(), size_t(count) * sizeof(BInst), cudaMemcpyHostToDevice, B->cap));
    ZK_TRY(ntt_init());
    ZK_TRY(prepare_execs(B, B->cap));
    return wait_stream(B->cap, "batch create");
  }();
  if (rc != ZKVC_OK) {
    delete B;
    return rc;
  }
  *out = B;
  return ZKVC_OK;
}

static int batch_prove(zkvc_batch* B, const int8_t* const* dX, const int8_t* const* dW, const uint8_t* rs,
                       int32_t* const* dY, uint8_t* proofs, int* status, cudaStream_t st) {
  ZK_CHECK(dX && dW && rs && dY && proofs, ZKVC_EINVAL, "batch prove: null argument");
  const int n = B->count;
  for (int i = 0; i < n; i++)
    ZK_CHECK(dX[i] && dW[i] && dY[i], ZKVC_EINVAL, "batch prove: null matrix pointer for instance %d", i);
  if (B->busy) {
    ZK_TRY(wait_stream(B->cap, "batch prove (previous call)"));
    B->busy = false;
  }
  // inputs into the batch's own buffers (ordered after the caller's earlier work on st)
  for (int i = 0; i < n; i++) {
    const Shape& sh = B->pks[i]->shape;
    ZK_CUDA(cudaMemcpyAsync(B->X + B->xo[i], dX[i], size_t(sh.a) * sh.n, cudaMemcpyDeviceToDevice, st));
    ZK_CUDA(cudaMemcpyAsync(B->W + B->wo[i], dW[i], size_t(sh.n) * sh.b, cudaMemcpyDeviceToDevice, st));
  }
  std::memcpy(B->h_rs, rs, size_t(n) * 64);
  ZK_CUDA(cudaEventRecord(B->ev_in, st));
  ZK_CUDA(cudaStreamWaitEvent(B->cap, B->ev_in, 0));
  if ((B->flags & ZKVC_BATCH_AUTOTUNE) && !B->tuned) {
    ZK_TRY(autotune(B));
  }
  if (B->flags & ZKVC_BATCH_EAGER) {
    ZK_TRY(enqueue(B));
  } else {
    if (!B->graph) ZK_TRY(capture(B));
    ZK_CUDA(cudaGraphLaunch(B->graph, B->cap));
    count_launches(B->graph_launches);
  }
  ZK_CUDA(cudaEventRecord(B->ev_out, B->cap));
  ZK_CUDA(cudaStreamWaitEvent(st, B->ev_out, 0));
  for (int i = 0; i < n; i++) {
    const Shape& sh = B->pks[i]->shape;
    ZK_CUDA(cudaMemcpyAsync(dY[i], B->Y + B->yo[i], size_t(sh.a) * sh.b * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                            st));
  }
  int rc = wait_stream(st, "batch prove");
  if (rc == ZKVC_ETIMEOUT) B->busy = true;
  ZK_TRY(rc);
  std::memcpy(proofs, B->h_proofs, size_t(n) * 256);
  int first_flag = 0;
  const int first_bad = decode_flags(B->h_flags, n, status, &first_flag);
  ZK_CHECK(first_bad < 0 || !(first_flag & 4), ZKVC_EINVAL, "batch prove: instance %d: r or s is not a canonical Fr element",
           first_bad);
  ZK_CHECK(first_bad < 0 || !(first_flag & 8), ZKVC_ETIMEOUT, "batch prove: instance %d: a tensor-core wait timed out",
           first_bad);
  ZK_CHECK(first_bad < 0, ZKVC_EUNSAT, "batch prove: instance %d does not satisfy its constraints (flags %d)", first_bad,
           first_flag);
  return ZKVC_OK;
}

// ------------------------------------------------------------------ server batches
// The proof server merges the requests waiting in its queue into one batch: the same
// launch sequence as above, run eagerly (no capture: every dispatch has a new mix of
// keys), laid over device memory the server owns (no allocation per dispatch), with the
// default launch shapes (no autotuning).  One transient batch object per server worker
// holds the streams, events and pinned staging, for up to `cap` instances.
int batch_serve_open(int cap, zkvc_batch** out) {
  ZK_CHECK(out && cap >= 1 && cap <= 4096, ZKVC_EINVAL, "server batch: capacity %d", cap);
  *out = nullptr;
  b_matmul_init();
  ZK_TRY(ntt_init());
  std::unique_ptr<zkvc_batch> B(new zkvc_batch());
  ZK_CUDA(cudaGetDevice(&B->device));
  B->flags = ZKVC_BATCH_EAGER;
  B->owns_mem = false;
  ZK_TRY(batch_resources(B.get(), cap));
  *out = B.release();
  return ZKVC_OK;
}

// Device bytes of a batch of these keys (host computation only).
size_t batch_serve_bytes(const zkvc_pk* const* pks, int count) {
  zkvc_batch B;
  B.owns_mem = false;
  cudaGetDevice(&B.device);
  B.pks.assign(pks, pks + count);
  B.count = count;
  return carve(&B, true);
}

// Proves count requests of the given keys as one batch over [mem, mem + mem_bytes): host
// X (a x n), W (n x b) and r || s in, host Y (a x b) and proofs (256 bytes each) out,
// status[i] per instance.  Returns ZKVC_ETIMEOUT with work possibly still in flight (the
// memory must not be reused until the object's next call has drained it).
int batch_serve_run(zkvc_batch* B, const zkvc_pk* const* pks, int count, uint8_t* mem, size_t mem_bytes,
                    const int8_t* const* hX, const int8_t* const* hW, const uint8_t* rs, int32_t* const* hY,
                    uint8_t* proofs, int* status) {
  ZK_CHECK(count >= 1 && count <= B->cap_count, ZKVC_EINVAL, "server batch: %d instances, capacity %d", count,
           B->cap_count);
  if (B->busy) {
    ZK_TRY(wait_stream(B->cap, "server batch (previous call)"));
    B->busy = false;
  }
  B->pks.assign(pks, pks + count);
  B->count = count;
  B->mem = nullptr;
  const size_t need = carve(B, true);
  ZK_CHECK(need <= mem_bytes, ZKVC_ENOMEM, "server batch: %zu bytes needed, %zu given", need, mem_bytes);
  B->mem = mem;
  B->mem_bytes = mem_bytes;
  carve(B, false);
  B->tune = BatchTune();
  B->tuned = true;
  cudaStream_t st = B->cap;
  ZK_CUDA(cudaMemcpyAsync(B->dinst, B->hinst.data(), size_t(count) * sizeof(BInst), cudaMemcpyHostToDevice, st));
  ZK_TRY(prepare_execs(B, st));
  for (int i = 0; i < count; i++) {
    const Shape& sh = pks[i]->shape;
    ZK_CUDA(cudaMemcpyAsync(B->X + B->xo[i], hX[i], size_t(sh.a) * sh.n, cudaMemcpyHostToDevice, st));
    ZK_CUDA(cudaMemcpyAsync(B->W + B->wo[i], hW[i], size_t(sh.n) * sh.b, cudaMemcpyHostToDevice, st));
  }
  std::memcpy(B->h_rs, rs, size_t(count) * 64);
  ZK_TRY(enqueue(B));
  for (int i = 0; i < count; i++) {
    const Shape& sh = pks[i]->shape;
    ZK_CUDA(cudaMemcpyAsync(hY[i], B->Y + B->yo[i], size_t(sh.a) * sh.b * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            st));
  }
  const int rc = wait_stream(st, "server batch");
  if (rc == ZKVC_ETIMEOUT) B->busy = true;
  ZK_TRY(rc);
  std::memcpy(proofs, B->h_proofs, size_t(count) * 256);
  int first_flag = 0;
  decode_flags(B->h_flags, count, status, &first_flag);
  return ZKVC_OK;
}

void batch_serve_drain(zkvc_batch* B) {
  if (B && B->cap) cudaStreamSynchronize(B->cap);
  if (B) B->busy = false;
}

static int device_guard_batch(int dev) {
  int cur = -1;
  ZK_CUDA(cudaGetDevice(&cur));
  ZK_CHECK(cur == dev, ZKVC_EINVAL, "batch was built on device %d but device %d is current", dev, cur);
  return ZKVC_OK;
}

static void tune_to_array(const BatchTune& t, int32_t* v) {
  const MsmTune* m[3] = {&t.small, &t.main, &t.g2};
  for (int i = 0; i < 3; i++) {
    v[2 * i] = (int32_t)m[i]->chunk;
    v[2 * i + 1] = (int32_t)m[i]->accum_threads;
  }
  v[6] = t.elog;
}

}  // namespace zkvc

extern "C" {

int zkvc_batch_create(const zkvc_pk* const* pks, int count, int flags, zkvc_batch** out) {
  set_error("%s", "");
  if (out) *out = nullptr;
  return batch_create(pks, count, flags, out);
}

void zkvc_batch_free(zkvc_batch* b) { delete b; }

int zkvc_batch_info(const zkvc_batch* b, int* count, size_t* device_bytes, uint64_t* graph_launches) {
  set_error("%s", "");
  ZK_CHECK(b, ZKVC_EINVAL, "batch: null handle");
  if (count) *count = b->count;
  if (device_bytes) *device_bytes = b->mem_bytes;
  if (graph_launches) *graph_launches = b->graph_launches;
  return ZKVC_OK;
}

int zkvc_batch_terms(const zkvc_batch* b, uint64_t terms[3]) {
  set_error("%s", "");
  ZK_CHECK(b && terms, ZKVC_EINVAL, "batch terms: null argument");
  ZK_TRY(device_guard_batch(b->device));
  ZK_TRY(wait_stream(b->cap, "batch terms"));
  const MsmExec* ex[3] = {&b->x_small, &b->x_main, &b->x_g2};
  for (int i = 0; i < 3; i++) {
    uint32_t v = 0;
    ZK_CUDA(cudaMemcpy(&v, msm_term_count(ex[i]), sizeof(v), cudaMemcpyDeviceToHost));
    terms[i] = v;
  }
  return ZKVC_OK;
}

int zkvc_batch_get_tuning(const zkvc_batch* b, int32_t* params, int n) {
  set_error("%s", "");
  ZK_CHECK(b && params && n >= ZKVC_BATCH_TUNING_LEN, ZKVC_EINVAL, "batch tuning: need %d slots",
           ZKVC_BATCH_TUNING_LEN);
  int32_t v[ZKVC_BATCH_TUNING_LEN];
  tune_to_array(b->tune, v);
  // chunk 0 means "automatic": report the chunk the finalized plans use
  v[0] = (int32_t)b->p_small.chunk;
  v[2] = (int32_t)b->p_main.chunk;
  v[4] = (int32_t)b->p_g2.chunk;
  std::memcpy(params, v, sizeof(v));
  return ZKVC_OK;
}

int zkvc_batch_set_tuning(zkvc_batch* b, const int32_t* params, int n) {
  set_error("%s", "");
  ZK_CHECK(b && params && n >= ZKVC_BATCH_TUNING_LEN, ZKVC_EINVAL, "batch tuning: need %d slots",
           ZKVC_BATCH_TUNING_LEN);
  ZK_TRY(device_guard_batch(b->device));
  BatchTune t;
  MsmTune* m[3] = {&t.small, &t.main, &t.g2};
  const uint32_t min_chunk[3] = {kChunkG1[0], kChunkG1[0], kChunkG2[0]};
  for (int i = 0; i < 3; i++) {
    ZK_CHECK(params[2 * i] >= (int32_t)min_chunk[i] && params[2 * i] <= 1024, ZKVC_EINVAL,
             "batch tuning: chunk %d outside [%u, 1024]", params[2 * i], min_chunk[i]);
    m[i]->chunk = (uint32_t)params[2 * i];
    m[i]->accum_threads = (uint32_t)params[2 * i + 1];
  }
  t.elog = params[6];
  ZK_CHECK(t.elog >= 8 && t.elog <= 11, ZKVC_EINVAL, "batch tuning: NTT block of 2^%d elements", t.elog);
  ZK_TRY(wait_stream(b->cap, "batch set tuning"));
  BatchTune old = b->tune;
  b->tune = t;
  int rc = prepare_execs(b, b->cap);
  if (rc != ZKVC_OK) {
    b->tune = old;
    prepare_execs(b, b->cap);
    return rc;
  }
  ZK_TRY(wait_stream(b->cap, "batch set tuning"));
  b->tuned = true;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return ZKVC_OK;
}

int zkvc_batch_prove(zkvc_batch* b, const int8_t* const* dX, const int8_t* const* dW, const uint8_t* rs,
                     int32_t* const* dY, uint8_t* proofs, int* status, void* stream) {
  set_error("%s", "");
  ZK_CHECK(b, ZKVC_EINVAL, "batch: null handle");
  ZK_TRY(device_guard_batch(b->device));
  return batch_prove(b, dX, dW, rs, dY, proofs, status, (cudaStream_t)stream);
}

int zkvc_prove_batch(const zkvc_pk* const* pks, const int8_t* const* dX, const int8_t* const* dW, const uint8_t* rs,
                     int count, int32_t* const* dY, uint8_t* proofs, int* status, void* stream) {
  zkvc_batch* b = nullptr;
  int rc = zkvc_batch_create(pks, count, ZKVC_BATCH_EAGER, &b);
  if (rc != ZKVC_OK) return rc;
  rc = batch_prove(b, dX, dW, rs, dY, proofs, status, (cudaStream_t)stream);
  zkvc_batch_free(b);
  return rc;
}

}  // extern "C"
