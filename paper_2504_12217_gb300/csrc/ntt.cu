// Radix-2 NTT over Fr for the QAP quotient h(x) (zkVC Sec. II: the R1CS is encoded as a
// QAP by interpolation over the domain H = <omega_N>; the prover divides A B - C by
// t(x) = x^N - 1 through evaluations on the coset gH).
//
// GB300 design: every pass takes k <= 10 consecutive radix-2 stages of one group of 2^k
// elements, staged through shared memory in a limb-major (structure-of-arrays) layout
// so that the 8 words of neighbouring elements fall in different banks.  A block holds
// G groups whose global indices differ in the low bits, so each global load or store of
// the block touches G consecutive elements (G * 32 contiguous bytes).  N = 2^16 takes
// two passes (two HBM round trips), N = 2^24 three.  Decimation in frequency maps
// natural order to bit-reversed order and decimation in time maps it back, so the prove
// path (INTT -> coset NTT -> pointwise -> coset INTT) never runs a bit-reversal pass:
// the coset shift g^i and 1/N are applied at the bit-reversed store of the inverse
// transforms.  Twiddles are read from a table omega^e (e < N/2), L2-resident for the
// proof domains.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "ntt.h"

namespace zkvc {

struct ScaleTabs {
  const Fr* g_lo;
  const Fr* gi_lo;
  const Fr* g_hi;
  const Fr* g_hi_n;
  const Fr* gi_hi_n;
  const Fr* consts;
};

__device__ __forceinline__ uint32_t brev_bits(uint32_t x, uint32_t logN) {
  return logN ? (__brev(x) >> (32 - logN)) : 0u;
}

__device__ __forceinline__ Fr scale_factor(const ScaleTabs& t, int mode, uint32_t i) {
  switch (mode) {
    case SC_G: return f_mul(ld_field(t.g_lo + (i & 1023u)), ld_field(t.g_hi + (i >> 10)));
    case SC_NG: return f_mul(ld_field(t.g_lo + (i & 1023u)), ld_field(t.g_hi_n + (i >> 10)));
    case SC_NGI: return f_mul(ld_field(t.gi_lo + (i & 1023u)), ld_field(t.gi_hi_n + (i >> 10)));
    case SC_N: return ld_field(t.consts + 0);
    default: return Fr::one();
  }
}

__device__ __forceinline__ Fr f_pow_u32(Fr base, uint32_t e) {
  Fr r = Fr::one();
  while (e) {
    if (e & 1u) r = f_mul(r, base);
    base = f_sqr(base);
    e >>= 1;
  }
  return r;
}

// consts: [0] N^-1 [1] 1/(g^N - 1) [2] omega [3] omega^-1 [4] g [5] g^-1 [6] g^1024
//         [7] g^-1024 [8] one
__global__ void k_domain_consts(Fr* consts, uint32_t logN) {
  // omega_(2^28) = g^((r - 1) / 2^28), g = 5 (a quadratic non-residue of Fr)
  uint32_t e[8];
  {
    uint32_t m[8];
#pragma unroll
    for (int i = 0; i < 8; i++) m[i] = mod_limb<FrCfg>(i);
    m[0] -= 1;  // r - 1 (r is odd, no borrow)
#pragma unroll
    for (int i = 0; i < 8; i++) e[i] = (m[i] >> 28) | (i < 7 ? (m[i + 1] << 4) : 0u);
  }
  Fr g = f_from_int<FrCfg>(5);
  Fr w = f_pow(g, e);
  for (uint32_t i = logN; i < 28; i++) w = f_sqr(w);
  Fr gN = g;
  for (uint32_t i = 0; i < logN; i++) gN = f_sqr(gN);
  Fr nm = f_from_int<FrCfg>((int32_t)(1u << logN));
  Fr gi = f_inv(g);
  consts[0] = f_inv(nm);
  consts[1] = f_inv(f_sub(gN, Fr::one()));
  consts[2] = w;
  consts[3] = f_inv(w);
  consts[4] = g;
  consts[5] = gi;
  consts[6] = f_pow_u32(g, 1024);
  consts[7] = f_pow_u32(gi, 1024);
  consts[8] = Fr::one();
}

// out[e] = mult * base^e for e < count; each thread fills a run of 16.
__global__ void k_fill_pows(Fr* out, size_t count, const Fr* base_p, const Fr* mult_p) {
  size_t e0 = (size_t(blockIdx.x) * blockDim.x + threadIdx.x) * 16;
  if (e0 >= count) return;
  Fr base = *base_p;
  Fr x = f_mul(*mult_p, f_pow_u32(base, (uint32_t)e0));
  for (size_t e = e0; e < e0 + 16 && e < count; e++) {
    st_field(out + e, x);
    x = f_mul(x, base);
  }
}

static int fill_pows(Fr* out, size_t count, const Fr* base, const Fr* mult, cudaStream_t st) {
  size_t runs = (count + 15) / 16;
  unsigned blocks = (unsigned)((runs + 127) / 128);
  k_fill_pows<<<blocks, 128, 0, st>>>(out, count, base, mult); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

static std::mutex g_dom_mu;
static std::map<std::pair<int, uint32_t>, NttDomain*> g_domains;

int ntt_domain(uint32_t logN, const NttDomain** out) {
  ZK_CHECK(logN >= 1 && logN <= 28, ZKVC_EINVAL, "ntt: log N = %u outside [1, 28]", logN);
  int dev = 0;
  ZK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_dom_mu);
  auto it = g_domains.find({dev, logN});
  if (it != g_domains.end()) {
    *out = it->second;
    return ZKVC_OK;
  }
  NttDomain* d = new NttDomain();
  d->logN = logN;
  d->N = size_t(1) << logN;
  size_t half = d->N / 2;
  size_t hi = d->N >= 1024 ? d->N / 1024 : 1;
  cudaStream_t st;
  ZK_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  ZK_CUDA(cudaMalloc(&d->consts, 16 * sizeof(Fr)));
  ZK_CUDA(cudaMalloc(&d->tw_fwd, half * sizeof(Fr)));
  ZK_CUDA(cudaMalloc(&d->tw_inv, half * sizeof(Fr)));
  ZK_CUDA(cudaMalloc(&d->g_lo, 1024 * sizeof(Fr)));
  ZK_CUDA(cudaMalloc(&d->gi_lo, 1024 * sizeof(Fr)));
  ZK_CUDA(cudaMalloc(&d->g_hi, hi * sizeof(Fr)));
  ZK_CUDA(cudaMalloc(&d->g_hi_n, hi * sizeof(Fr)));
  ZK_CUDA(cudaMalloc(&d->gi_hi_n, hi * sizeof(Fr)));
  k_domain_consts<<<1, 1, 0, st>>>(d->consts, logN); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  const Fr* c = d->consts;
  ZK_TRY(fill_pows(d->tw_fwd, half, c + 2, c + 8, st));
  ZK_TRY(fill_pows(d->tw_inv, half, c + 3, c + 8, st));
  ZK_TRY(fill_pows(d->g_lo, 1024, c + 4, c + 8, st));
  ZK_TRY(fill_pows(d->gi_lo, 1024, c + 5, c + 8, st));
  ZK_TRY(fill_pows(d->g_hi, hi, c + 6, c + 8, st));
  ZK_TRY(fill_pows(d->g_hi_n, hi, c + 6, c + 0, st));
  ZK_TRY(fill_pows(d->gi_hi_n, hi, c + 7, c + 0, st));
  ZK_CUDA(cudaStreamSynchronize(st));
  ZK_CUDA(cudaStreamDestroy(st));
  g_domains[{dev, logN}] = d;
  *out = d;
  return ZKVC_OK;
}

static ScaleTabs tabs_of(const NttDomain* d) {
  return {d->g_lo, d->gi_lo, d->g_hi, d->g_hi_n, d->gi_hi_n, d->consts};
}

// One pass: k consecutive radix-2 stages from stage s0, over G = 2^logG groups of 2^k
// elements per block (E = G 2^k elements, staged limb-major in shared memory).
struct PassGeo {
  uint32_t L, s0, k, logG;
};

// global index of the block's e-th staged element
template <bool DIT>
__device__ __forceinline__ size_t pass_index(const PassGeo& g, size_t gid0, uint32_t e) {
  const uint32_t G = 1u << g.logG;
  const uint32_t gg = e & (G - 1), j = e >> g.logG;
  const size_t gid = gid0 + gg;
  const uint32_t sbits = DIT ? g.s0 : (g.L - g.s0 - g.k);
  const size_t lo = gid & ((size_t(1) << sbits) - 1), hi = gid >> sbits;
  const size_t base = DIT ? ((hi << (g.s0 + g.k)) | lo) : ((hi << (g.L - g.s0)) | lo);
  return base + (size_t(j) << sbits);
}

__device__ __forceinline__ Fr sm_get(const uint32_t* sm, uint32_t E, uint32_t e) {
  Fr x;
#pragma unroll
  for (int l = 0; l < 8; l++) x.v[l] = sm[l * E + e];
  return x;
}
__device__ __forceinline__ void sm_put(uint32_t* sm, uint32_t E, uint32_t e, const Fr& x) {
#pragma unroll
  for (int l = 0; l < 8; l++) sm[l * E + e] = x.v[l];
}

template <bool DIT>
__device__ __forceinline__ void pass_load(const Fr* arr, const PassGeo& g, size_t gid0, uint32_t* sm, int load_scale,
                                          int to_mont, const ScaleTabs& tabs) {
  const uint32_t E = 1u << (g.logG + g.k);
  for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) {
    const size_t idx = pass_index<DIT>(g, gid0, e);
    Fr x = ld_field(arr + idx);
    if (to_mont) x = f_to_mont(x);
    if (load_scale) x = f_mul(x, scale_factor(tabs, load_scale, (uint32_t)idx));
    sm_put(sm, E, e, x);
  }
}

template <bool DIT>
__device__ __forceinline__ void pass_store(Fr* arr, const PassGeo& g, size_t gid0, const uint32_t* sm, int store_scale,
                                           const ScaleTabs& tabs) {
  const uint32_t E = 1u << (g.logG + g.k);
  for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) {
    const size_t idx = pass_index<DIT>(g, gid0, e);
    Fr x = sm_get(sm, E, e);
    if (store_scale) x = f_mul(x, scale_factor(tabs, store_scale, brev_bits((uint32_t)idx, g.L)));
    st_field(arr + idx, x);
  }
}

// The pass's k stages on NPOLY staged arrays (8 E words apart).  Radix 2 (R4 false):
// one stage per shared-memory round trip, one butterfly per element pair.  R4: two stages
// at a time: a radix-4 unit reads four elements, runs their four butterflies of stages t
// and t + 1 in registers (two independent products per stage) and writes them back, so a
// pair of stages costs one round trip and one barrier instead of two; an odd last stage
// runs as radix 2.  R4 holds more registers (112 against 64: two blocks of 256 per SM
// instead of four), which pays where the grid is too small to fill the GPU (the latency of
// a thread's serial stages decides) and costs a few per cent where it is large.  Barriers
// between rounds (the first one orders the loads before it).
//   DIF, stage t of half h (block 2h), then h/2: a unit is j0 = blk 2h + off (off < h/2)
//     and j0 + h/2, j0 + h, j0 + 3h/2; twiddles w_t(off), w_t(off + h/2), w_(t+1)(off).
//   DIT, stage t of half h (block 2h), then 2h: a unit is j0 = blk 4h + off (off < h) and
//     j0 + h, j0 + 2h, j0 + 3h; twiddles w_t(off), w_(t+1)(off), w_(t+1)(off + h).
// w_t(q) is the table entry of the radix-2 form: DIF ((q << sbits) + lo) << s, DIT
// ((q << s0) + lo) << (L - 1 - s), lo the group's low index bits, s = s0 + t.
template <bool DIT, int NPOLY, bool R4>
__device__ __forceinline__ void pass_stages(uint32_t* sm, const PassGeo& g, size_t gid0, const Fr* tw) {
  const uint32_t G = 1u << g.logG, E = G << g.k, L = g.L, logG = g.logG;
  const uint32_t sbits = DIT ? g.s0 : (L - g.s0 - g.k);
  const size_t smask = (size_t(1) << sbits) - 1;
  auto twi = [&](uint32_t s, uint32_t q, size_t lo) -> size_t {
    return DIT ? ((((size_t)q << g.s0) + lo) << (L - 1 - s)) : ((((size_t)q << sbits) + lo) << s);
  };
  __syncthreads();
  uint32_t t = 0;
  const uint32_t nq = E >> 2;
  for (; R4 && t + 1 < g.k; t += 2) {
    const uint32_t s = g.s0 + t;
    for (uint32_t ua = threadIdx.x; ua < nq * (uint32_t)NPOLY; ua += blockDim.x) {
      const uint32_t poly = NPOLY == 1 ? 0u : ua / nq, u = ua - poly * nq;
      uint32_t* smp = sm + size_t(poly) * 8 * E;
      const uint32_t gg = u & (G - 1), q = u >> logG;
      const size_t lo = (gid0 + gg) & smask;
      if (DIT) {
        const uint32_t lh = t, h = 1u << lh;  // stage t: half h; stage t + 1: half 2h
        const uint32_t off = q & (h - 1), j0 = ((q >> lh) << (lh + 2)) + off;
        const uint32_t p0 = (j0 << logG) + gg, p1 = ((j0 + h) << logG) + gg, p2 = ((j0 + 2 * h) << logG) + gg,
                       p3 = ((j0 + 3 * h) << logG) + gg;
        const Fr w0 = ld_field(tw + twi(s, off, lo));
        Fr x0 = sm_get(smp, E, p0), x1 = sm_get(smp, E, p1), x2 = sm_get(smp, E, p2), x3 = sm_get(smp, E, p3);
        x1 = f_mul(x1, w0);
        x3 = f_mul(x3, w0);
        const Fr a = f_add(x0, x1), b = f_sub(x0, x1), c = f_add(x2, x3), d = f_sub(x2, x3);
        const Fr w1 = ld_field(tw + twi(s + 1, off, lo)), w2 = ld_field(tw + twi(s + 1, off + h, lo));
        const Fr vc = f_mul(c, w1), vd = f_mul(d, w2);
        sm_put(smp, E, p0, f_add(a, vc));
        sm_put(smp, E, p2, f_sub(a, vc));
        sm_put(smp, E, p1, f_add(b, vd));
        sm_put(smp, E, p3, f_sub(b, vd));
      } else {
        const uint32_t lh = g.k - 1 - t, h = 1u << lh, hq = h >> 1;  // stage t: half h; t + 1: h/2
        const uint32_t off = q & (hq - 1), j0 = ((q >> (lh - 1)) << (lh + 1)) + off;
        const uint32_t p0 = (j0 << logG) + gg, p1 = ((j0 + hq) << logG) + gg, p2 = ((j0 + h) << logG) + gg,
                       p3 = ((j0 + h + hq) << logG) + gg;
        const Fr w0 = ld_field(tw + twi(s, off, lo)), w1 = ld_field(tw + twi(s, off + hq, lo));
        const Fr x0 = sm_get(smp, E, p0), x1 = sm_get(smp, E, p1), x2 = sm_get(smp, E, p2), x3 = sm_get(smp, E, p3);
        const Fr a = f_add(x0, x2), b = f_mul(f_sub(x0, x2), w0);
        const Fr c = f_add(x1, x3), d = f_mul(f_sub(x1, x3), w1);
        const Fr w2 = ld_field(tw + twi(s + 1, off, lo));
        sm_put(smp, E, p0, f_add(a, c));
        sm_put(smp, E, p1, f_mul(f_sub(a, c), w2));
        sm_put(smp, E, p2, f_add(b, d));
        sm_put(smp, E, p3, f_mul(f_sub(b, d), w2));
      }
    }
    __syncthreads();
  }
  for (; t < g.k; t++) {  // radix 2: every stage, or the last of an odd count
    const uint32_t s = g.s0 + t, nbf = E >> 1;
    const uint32_t logh = DIT ? t : (g.k - 1 - t), h = 1u << logh;
    for (uint32_t bfa = threadIdx.x; bfa < nbf * (uint32_t)NPOLY; bfa += blockDim.x) {
      const uint32_t poly = NPOLY == 1 ? 0u : bfa / nbf, bf = bfa - poly * nbf;
      uint32_t* smp = sm + size_t(poly) * 8 * E;
      const uint32_t gg = bf & (G - 1), q = bf >> logG;
      const uint32_t qh = q & (h - 1);
      const uint32_t ju = ((q >> logh) << (logh + 1)) + qh;
      const uint32_t pu = (ju << logG) + gg, pv = ((ju + h) << logG) + gg;
      const size_t lo = (gid0 + gg) & smask;
      const Fr w = ld_field(tw + twi(s, qh, lo));
      Fr u = sm_get(smp, E, pu), v = sm_get(smp, E, pv);
      Fr a, b;
      if (DIT) {
        v = f_mul(v, w);
        a = f_add(u, v);
        b = f_sub(u, v);
      } else {
        a = f_add(u, v);
        b = f_mul(f_sub(u, v), w);
      }
      sm_put(smp, E, pu, a);
      sm_put(smp, E, pv, b);
    }
    __syncthreads();
  }
}

// One pass of k stages over G groups per block; see the file comment.
template <bool DIT, bool R4>
__global__ void __launch_bounds__(256) k_ntt_pass(Fr* data, size_t bstride, const Fr* __restrict__ tw,
                                                  uint32_t logN, uint32_t s0, uint32_t k, uint32_t logG,
                                                  int load_scale, int store_scale, int to_mont, ScaleTabs tabs) {
  extern __shared__ uint32_t sm[];
  const PassGeo g{logN, s0, k, logG};
  Fr* arr = data + size_t(blockIdx.y) * bstride;
  const size_t gid0 = size_t(blockIdx.x) << logG;
  pass_load<DIT>(arr, g, gid0, sm, load_scale, to_mont, tabs);
  pass_stages<DIT, 1, R4>(sm, g, gid0, tw);
  pass_store<DIT>(arr, g, gid0, sm, store_scale, tabs);
}

// The turn of an inverse DIF transform into a forward DIT transform, in one pass: the
// DIF's last pass (its k stages end at stage L - 1, groups of 2^k consecutive elements),
// the inverse's scaling by the factor of each element's natural index, and the DIT's
// first pass over the same groups.  Saves a global round trip and a launch.
template <bool R4>
__global__ void __launch_bounds__(256) k_ntt_turn(Fr* data, size_t bstride, const Fr* __restrict__ tw_inv,
                                                  const Fr* __restrict__ tw_fwd, uint32_t L, uint32_t k,
                                                  uint32_t logG, int mid_scale, ScaleTabs tabs) {
  extern __shared__ uint32_t sm[];
  const PassGeo gdif{L, L - k, k, logG}, gdit{L, 0, k, logG};
  Fr* arr = data + size_t(blockIdx.y) * bstride;
  const size_t gid0 = size_t(blockIdx.x) << logG;
  const uint32_t E = 1u << (logG + k);
  pass_load<false>(arr, gdif, gid0, sm, SC_NONE, 0, tabs);
  pass_stages<false, 1, R4>(sm, gdif, gid0, tw_inv);
  for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) {
    const size_t idx = pass_index<false>(gdif, gid0, e);
    sm_put(sm, E, e, f_mul(sm_get(sm, E, e), scale_factor(tabs, mid_scale, brev_bits((uint32_t)idx, L))));
  }
  pass_stages<true, 1, R4>(sm, gdit, gid0, tw_fwd);
  pass_store<true>(arr, gdit, gid0, sm, SC_NONE, tabs);
}

// The quotient turn, one instance per blockIdx.y (arrays A_i, B_i, C_i, H_i of N
// elements at i, m + i, 2m + i, 3m + i): the last DIT pass of A, B and C (strided groups),
// h_ev = (A B - C) / (g^N - 1) on the staged elements, and the first DIF pass of the
// inverse transform of h over the same groups; only H is written.  Small grids get up
// to three times the threads of a single-array pass (the three forward passes side by
// side), large ones one array's worth.
template <bool R4>
__global__ void __launch_bounds__(768) k_ntt_quotient_turn(Fr* ev, uint32_t m, size_t N, const Fr* __restrict__ tw_fwd,
                                                           const Fr* __restrict__ tw_inv, uint32_t L, uint32_t k,
                                                           uint32_t logG, ScaleTabs tabs) {
  extern __shared__ uint32_t sm[];
  const PassGeo gdit{L, L - k, k, logG}, gdif{L, 0, k, logG};
  const size_t gid0 = size_t(blockIdx.x) << logG;
  const uint32_t E = 1u << (logG + k);
  const size_t i = blockIdx.y;
  for (int p = 0; p < 3; p++)
    pass_load<true>(ev + (size_t(p) * m + i) * N, gdit, gid0, sm + size_t(p) * 8 * E, SC_NONE, 0, tabs);
  pass_stages<true, 3, R4>(sm, gdit, gid0, tw_fwd);
  const Fr zinv = ld_field(tabs.consts + 1);
  for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) {
    const Fr a = sm_get(sm, E, e), b = sm_get(sm + 8 * E, E, e), c = sm_get(sm + 16 * E, E, e);
    sm_put(sm, E, e, f_mul(f_sub(f_mul(a, b), c), zinv));
  }
  pass_stages<false, 1, R4>(sm, gdif, gid0, tw_inv);
  pass_store<false>(ev + (size_t(3) * m + i) * N, gdif, gid0, sm, SC_NONE, tabs);
}

static std::once_flag g_smem_once;

static void ntt_smem_attrs() {
  std::call_once(g_smem_once, [] {
    cudaFuncSetAttribute(k_ntt_pass<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 << 10);
    cudaFuncSetAttribute(k_ntt_pass<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 << 10);
    cudaFuncSetAttribute(k_ntt_pass<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 << 10);
    cudaFuncSetAttribute(k_ntt_pass<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 << 10);
    cudaFuncSetAttribute(k_ntt_turn<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 << 10);
    cudaFuncSetAttribute(k_ntt_turn<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 << 10);
    cudaFuncSetAttribute(k_ntt_quotient_turn<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 192 << 10);
    cudaFuncSetAttribute(k_ntt_quotient_turn<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 192 << 10);
  });
}

int ntt_init() {
  ntt_smem_attrs();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

// Stage split of an N = 2^L transform into passes of at most min(elog, 10) stages, the
// first passes one stage longer.
static std::vector<uint32_t> pass_split(uint32_t L, int elog) {
  const uint32_t kmax = (uint32_t)elog < 10 ? (uint32_t)elog : 10;
  const uint32_t P = (L + kmax - 1) / kmax;
  const uint32_t kb = L / P, rem = L % P;
  std::vector<uint32_t> ks(P);
  for (uint32_t p = 0; p < P; p++) ks[p] = kb + (p < rem ? 1 : 0);
  return ks;
}

// groups per block (log2) and the block shape of a pass of k stages
struct PassShape {
  uint32_t logG, E, threads;
  dim3 grid;
};
static PassShape pass_shape(uint32_t L, uint32_t k, int elog, int batch) {
  PassShape sh;
  const uint32_t groups_log = L - k;
  sh.logG = (uint32_t)elog - k;
  if (sh.logG > groups_log) sh.logG = groups_log;
  sh.E = 1u << (sh.logG + k);
  sh.threads = sh.E / 2 < 256 ? sh.E / 2 : 256;
  sh.grid = dim3((unsigned)(size_t(1) << (groups_log - sh.logG)), (unsigned)batch);
  return sh;
}

// Radix 4 for grids below four blocks per SM (latency-bound: fewer, longer-lived threads
// with two independent products per stage finish sooner), radix 2 above (throughput:
// twice the resident warps).
static bool radix4(dim3 grid) { return uint64_t(grid.x) * grid.y < 4ull * (uint64_t)device_sm_count(); }

static int launch_pass(bool dit, Fr* data, int batch, size_t bstride, const NttDomain* d, const Fr* tw, uint32_t s0,
                       uint32_t k, int elog, int ls, int ss, int tm, cudaStream_t st) {
  const uint32_t L = d->logN;
  const PassShape sh = pass_shape(L, k, elog, batch);
  const size_t smem = size_t(sh.E) * 32;
  const ScaleTabs tabs = tabs_of(d);
  const bool r4 = radix4(sh.grid);
  if (dit && r4)
    k_ntt_pass<true, true><<<sh.grid, sh.threads, smem, st>>>(data, bstride, tw, L, s0, k, sh.logG, ls, ss, tm, tabs);
  else if (dit)
    k_ntt_pass<true, false><<<sh.grid, sh.threads, smem, st>>>(data, bstride, tw, L, s0, k, sh.logG, ls, ss, tm, tabs);
  else if (r4)
    k_ntt_pass<false, true><<<sh.grid, sh.threads, smem, st>>>(data, bstride, tw, L, s0, k, sh.logG, ls, ss, tm, tabs);
  else
    k_ntt_pass<false, false><<<sh.grid, sh.threads, smem, st>>>(data, bstride, tw, L, s0, k, sh.logG, ls, ss, tm, tabs);
  ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

static int run_passes(bool dit, Fr* data, int batch, size_t bstride, const NttDomain* d, bool inverse,
                      int load_scale, int store_scale, bool to_mont, int elog, cudaStream_t st) {
  ZK_CHECK(elog >= 8 && elog <= 11, ZKVC_EINVAL, "ntt: 2^%d elements per block outside [2^8, 2^11]", elog);
  ZK_CHECK(batch >= 1 && batch <= 65535, ZKVC_EINVAL, "ntt: batch of %d arrays", batch);
  ntt_smem_attrs();
  const std::vector<uint32_t> ks = pass_split(d->logN, elog);
  const uint32_t P = (uint32_t)ks.size();
  const Fr* tw = inverse ? d->tw_inv : d->tw_fwd;
  uint32_t s0 = 0;
  for (uint32_t p = 0; p < P; p++) {
    const bool first = p == 0, last = p + 1 == P;
    ZK_TRY(launch_pass(dit, data, batch, bstride, d, tw, s0, ks[p], elog, first ? load_scale : 0,
                       last ? store_scale : 0, (first && to_mont) ? 1 : 0, st));
    s0 += ks[p];
  }
  return ZKVC_OK;
}

int ntt_quotient_chain(Fr* ev, int m, size_t N, const NttDomain* d, cudaStream_t st, int elog) {
  ZK_CHECK(elog >= 8 && elog <= 11, ZKVC_EINVAL, "ntt: 2^%d elements per block outside [2^8, 2^11]", elog);
  ZK_CHECK(m >= 1 && 3 * m <= 65535, ZKVC_EINVAL, "ntt: %d instances", m);
  ZK_CHECK(N == d->N, ZKVC_EINVAL, "ntt: array stride %zu is not N", N);
  ntt_smem_attrs();
  const uint32_t L = d->logN;
  const std::vector<uint32_t> ks = pass_split(L, elog);
  const uint32_t P = (uint32_t)ks.size();
  Fr* H = ev + size_t(3) * m * N;
  if (P < 2 || L < 2) {  // one pass: no turn to fuse
    ZK_TRY(run_passes(false, ev, 3 * m, N, d, true, SC_NONE, SC_NG, false, elog, st));
    ZK_TRY(run_passes(true, ev, 3 * m, N, d, false, SC_NONE, SC_NONE, false, elog, st));
    ZK_TRY(ntt_quotient(ev, ev + size_t(m) * N, ev + size_t(2) * m * N, H, d, st, size_t(m) * N));
    return run_passes(false, H, m, N, d, true, SC_NONE, SC_NGI, false, elog, st);
  }
  const ScaleTabs tabs = tabs_of(d);
  // inverse DIF transforms of A, B, C up to their last pass
  uint32_t s0 = 0;
  for (uint32_t p = 0; p + 1 < P; p++) {
    ZK_TRY(launch_pass(false, ev, 3 * m, N, d, d->tw_inv, s0, ks[p], elog, 0, 0, 0, st));
    s0 += ks[p];
  }
  // turn: the inverse's last pass, x N^-1 g^i, the forward DIT's first pass
  {
    const uint32_t k = ks[P - 1];
    const PassShape sh = pass_shape(L, k, elog, 3 * m);
    if (radix4(sh.grid))
      k_ntt_turn<true><<<sh.grid, sh.threads, size_t(sh.E) * 32, st>>>(ev, N, d->tw_inv, d->tw_fwd, L, k, sh.logG,
                                                                      SC_NG, tabs);
    else
      k_ntt_turn<false><<<sh.grid, sh.threads, size_t(sh.E) * 32, st>>>(ev, N, d->tw_inv, d->tw_fwd, L, k, sh.logG,
                                                                       SC_NG, tabs);
    ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaGetLastError());
  }
  // the forward DIT's middle passes: the mirror of the DIF split (its pass q covers the
  // groups of the DIF's pass P - 1 - q)
  uint32_t s0d = ks[P - 1];
  for (uint32_t q = 1; q + 1 < P; q++) {
    ZK_TRY(launch_pass(true, ev, 3 * m, N, d, d->tw_fwd, s0d, ks[P - 1 - q], elog, 0, 0, 0, st));
    s0d += ks[P - 1 - q];
  }
  // quotient turn: the forward's last pass of A, B, C, the quotient, the first inverse
  // DIF pass of h
  {
    const uint32_t k = ks[0];
    const PassShape sh = pass_shape(L, k, elog, m);
    // three times the threads where the grid is too small to fill the GPU (latency-bound),
    // one array's worth where it is large (more blocks per SM)
    const uint64_t blocks = uint64_t(sh.grid.x) * sh.grid.y;
    const uint32_t threads =
        blocks < 2 * uint64_t(device_sm_count()) ? std::min<uint32_t>(3 * sh.threads, 768) : sh.threads;
    if (radix4(sh.grid))
      k_ntt_quotient_turn<true><<<sh.grid, threads, size_t(3) * sh.E * 32, st>>>(ev, (uint32_t)m, N, d->tw_fwd,
                                                                                 d->tw_inv, L, k, sh.logG, tabs);
    else
      k_ntt_quotient_turn<false><<<sh.grid, threads, size_t(3) * sh.E * 32, st>>>(ev, (uint32_t)m, N, d->tw_fwd,
                                                                                  d->tw_inv, L, k, sh.logG, tabs);
    ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaGetLastError());
  }
  // the rest of h's inverse DIF transform, x N^-1 g^-i at the last store
  s0 = ks[0];
  for (uint32_t p = 1; p < P; p++) {
    ZK_TRY(launch_pass(false, H, m, N, d, d->tw_inv, s0, ks[p], elog, 0, p + 1 == P ? SC_NGI : 0, 0, st));
    s0 += ks[p];
  }
  return ZKVC_OK;
}

int ntt_dif(Fr* data, int batch, size_t bstride, const NttDomain* d, bool inverse, int load_scale,
            int store_scale, bool to_mont, cudaStream_t st, int elog) {
  return run_passes(false, data, batch, bstride, d, inverse, load_scale, store_scale, to_mont, elog, st);
}

int ntt_dit(Fr* data, int batch, size_t bstride, const NttDomain* d, bool inverse, cudaStream_t st, int elog) {
  return run_passes(true, data, batch, bstride, d, inverse, 0, 0, false, elog, st);
}

__global__ void k_bitrev(Fr* a, uint32_t logN, int scale, int from_mont, ScaleTabs tabs) {
  size_t N = size_t(1) << logN;
  size_t p = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= N) return;
  size_t q = brev_bits((uint32_t)p, logN);
  if (p > q) return;
  Fr x = ld_field(a + p), y = ld_field(a + q);
  // natural index p receives the element at bit-reversed position q, and vice versa
  if (scale) {
    y = f_mul(y, scale_factor(tabs, scale, (uint32_t)p));
    if (p != q) x = f_mul(x, scale_factor(tabs, scale, (uint32_t)q));
  }
  if (from_mont) {
    x = f_from_mont(x);
    y = f_from_mont(y);
  }
  st_field(a + p, y);
  if (p != q) st_field(a + q, x);
}

int ntt_bitrev(Fr* data, const NttDomain* d, int scale, bool from_mont, cudaStream_t st) {
  unsigned blocks = (unsigned)((d->N + 255) / 256);
  k_bitrev<<<blocks, 256, 0, st>>>(data, d->logN, scale, from_mont ? 1 : 0, tabs_of(d)); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

__global__ void k_quotient(const Fr* __restrict__ A, const Fr* __restrict__ B, const Fr* __restrict__ C, Fr* H,
                           size_t N, const Fr* consts) {
  size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  Fr zinv = ld_field(consts + 1);
  Fr v = f_sub(f_mul(ld_field(A + i), ld_field(B + i)), ld_field(C + i));
  st_field(H + i, f_mul(v, zinv));
}

int ntt_quotient(const Fr* A, const Fr* B, const Fr* C, Fr* H, const NttDomain* d, cudaStream_t st, size_t count) {
  size_t n = count ? count : d->N;
  unsigned blocks = (unsigned)((n + 255) / 256);
  k_quotient<<<blocks, 256, 0, st>>>(A, B, C, H, n, d->consts); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

}  // namespace zkvc
