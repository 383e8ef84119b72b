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
#include <map>
#include <mutex>
#include <utility>

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

// One pass of k stages over G groups per block; see the file comment.
template <bool DIT>
__global__ void __launch_bounds__(256) k_ntt_pass(Fr* data, size_t bstride, const Fr* __restrict__ tw,
                                                  uint32_t logN, uint32_t s0, uint32_t k, uint32_t logG,
                                                  int load_scale, int store_scale, int to_mont, ScaleTabs tabs) {
  extern __shared__ uint32_t sm[];
  const uint32_t G = 1u << logG;
  const uint32_t E = G << k;
  Fr* arr = data + size_t(blockIdx.y) * bstride;
  const uint32_t L = logN;
  const uint32_t sbits = DIT ? s0 : (L - s0 - k);
  const size_t smask = (size_t(1) << sbits) - 1;
  const size_t gid0 = size_t(blockIdx.x) << logG;

  for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) {
    uint32_t g = e & (G - 1), j = e >> logG;
    size_t gid = gid0 + g;
    size_t lo = gid & smask, hi = gid >> sbits;
    size_t base = DIT ? ((hi << (s0 + k)) | lo) : ((hi << (L - s0)) | lo);
    size_t idx = base + (size_t(j) << sbits);
    Fr x = ld_field(arr + idx);
    if (to_mont) x = f_to_mont(x);
    if (load_scale) x = f_mul(x, scale_factor(tabs, load_scale, (uint32_t)idx));
#pragma unroll
    for (int l = 0; l < 8; l++) sm[l * E + e] = x.v[l];
  }
  __syncthreads();

  const uint32_t nbf = E >> 1;
  for (uint32_t t = 0; t < k; t++) {
    const uint32_t s = s0 + t;
    const uint32_t logh = DIT ? t : (k - 1 - t);
    const uint32_t h = 1u << logh;
    for (uint32_t bf = threadIdx.x; bf < nbf; bf += blockDim.x) {
      uint32_t g = bf & (G - 1), q = bf >> logG;
      uint32_t qh = q & (h - 1);
      uint32_t ju = ((q >> logh) << (logh + 1)) + qh;
      uint32_t pu = (ju << logG) + g, pv = ((ju + h) << logG) + g;
      size_t lo = (gid0 + g) & smask;
      size_t etw = DIT ? ((((size_t)qh << s0) + lo) << (L - 1 - s)) : ((((size_t)qh << sbits) + lo) << s);
      Fr w = ld_field(tw + etw);
      Fr u, v;
#pragma unroll
      for (int l = 0; l < 8; l++) {
        u.v[l] = sm[l * E + pu];
        v.v[l] = sm[l * E + pv];
      }
      Fr a, b;
      if (DIT) {
        v = f_mul(v, w);
        a = f_add(u, v);
        b = f_sub(u, v);
      } else {
        a = f_add(u, v);
        b = f_mul(f_sub(u, v), w);
      }
#pragma unroll
      for (int l = 0; l < 8; l++) {
        sm[l * E + pu] = a.v[l];
        sm[l * E + pv] = b.v[l];
      }
    }
    __syncthreads();
  }

  for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) {
    uint32_t g = e & (G - 1), j = e >> logG;
    size_t gid = gid0 + g;
    size_t lo = gid & smask, hi = gid >> sbits;
    size_t base = DIT ? ((hi << (s0 + k)) | lo) : ((hi << (L - s0)) | lo);
    size_t idx = base + (size_t(j) << sbits);
    Fr x;
#pragma unroll
    for (int l = 0; l < 8; l++) x.v[l] = sm[l * E + e];
    if (store_scale) x = f_mul(x, scale_factor(tabs, store_scale, brev_bits((uint32_t)idx, L)));
    st_field(arr + idx, x);
  }
}

static std::once_flag g_smem_once;

static void ntt_smem_attrs() {
  std::call_once(g_smem_once, [] {
    cudaFuncSetAttribute(k_ntt_pass<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 << 10);
    cudaFuncSetAttribute(k_ntt_pass<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 << 10);
  });
}

int ntt_init() {
  ntt_smem_attrs();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

static int run_passes(bool dit, Fr* data, int batch, size_t bstride, const NttDomain* d, bool inverse,
                      int load_scale, int store_scale, bool to_mont, int elog, cudaStream_t st) {
  ZK_CHECK(elog >= 8 && elog <= 11, ZKVC_EINVAL, "ntt: 2^%d elements per block outside [2^8, 2^11]", elog);
  ZK_CHECK(batch >= 1 && batch <= 65535, ZKVC_EINVAL, "ntt: batch of %d arrays", batch);
  ntt_smem_attrs();
  const uint32_t L = d->logN;
  const uint32_t kmax = (uint32_t)elog < 10 ? (uint32_t)elog : 10;
  const uint32_t P = (L + kmax - 1) / kmax;
  const uint32_t kb = L / P, rem = L % P;
  uint32_t s0 = 0;
  const Fr* tw = inverse ? d->tw_inv : d->tw_fwd;
  ScaleTabs tabs = tabs_of(d);
  for (uint32_t p = 0; p < P; p++) {
    uint32_t k = kb + (p < rem ? 1 : 0);
    uint32_t groups_log = L - k;
    uint32_t logG = (uint32_t)elog - k;
    if (logG > groups_log) logG = groups_log;
    uint32_t E = 1u << (logG + k);
    uint32_t threads = E / 2 < 256 ? E / 2 : 256;
    dim3 grid((unsigned)(size_t(1) << (groups_log - logG)), (unsigned)batch);
    size_t smem = size_t(E) * 32;
    bool first = p == 0, last = p + 1 == P;
    int ls = first ? load_scale : 0, ss = last ? store_scale : 0, tm = (first && to_mont) ? 1 : 0;
    if (dit)
      k_ntt_pass<true><<<grid, threads, smem, st>>>(data, bstride, tw, L, s0, k, logG, ls, ss, tm, tabs);
    else
      k_ntt_pass<false><<<grid, threads, smem, st>>>(data, bstride, tw, L, s0, k, logG, ls, ss, tm, tabs);
    ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaGetLastError());
    s0 += k;
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
