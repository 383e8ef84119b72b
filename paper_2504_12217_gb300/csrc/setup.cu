// Groth16 Gen for the CRPC + PSQ matmul circuit (zkVC Sec. II: Gen; Sec. III-A/B: the
// circuit), on the GPU.
//
// The QAP polynomials of the circuit are sparse and structured, so every proving-key
// scalar has a closed form in the Lagrange values L_k(tau) of the domain H = <omega_N>:
//   row k < n:   A_k = sum_i z^(ib) [X_ik],  B_k = sum_j z^j [W_kj],
//                C_k = [S_k] - [S_(k-1)] (k < n-1),  C_(n-1) = sum_ij z^(ib+j) [Y_ij] - [S_(n-2)]
//   row n + v:   A = [variable v] for v = 0 .. l (public-input binding rows)
// so   A_one = L_n,  A_Xik = z^(ib) L_k + L_(n+v),  A_Yij = L_(n+v),  C_Yij = z^(ib+j) L_(n-1),
//      B_Wkj = z^j L_k,  C_Sk = L_k - L_(k+1).
// L_k(tau) = (tau^N - 1) omega^k / (N (tau - omega^k)) is evaluated with one batched
// inversion per chunk of 32 rows.  Each proving-key base P = [s]G is then produced by a
// fixed-base comb over 32 byte-windows of the generator (32 mixed additions per point)
// and normalised to affine with Montgomery's batch-inversion trick; bases that the
// prover's MSMs read at several windows are stored as [s 2^(c w)]G for each window.
#include <cstring>
#include <mutex>
#include <map>

#include "groth16.h"
#include "setup_common.h"

namespace zkvc {

int make_shape(int a, int n, int b, Shape* s) {
  ZK_CHECK(a >= 1 && n >= 1 && b >= 1, ZKVC_EINVAL, "shape (%d, %d, %d): every dimension must be >= 1", a, n, b);
  uint64_t l = uint64_t(a) * n + uint64_t(a) * b;
  uint64_t vars = 1 + l + uint64_t(n) * b + (n - 1);
  uint64_t rows = uint64_t(n) + l + 1;
  ZK_CHECK(rows <= (1ull << 26) && vars < (1ull << 30), ZKVC_EINVAL, "shape (%d, %d, %d) too large", a, n, b);
  s->a = a;
  s->n = n;
  s->b = b;
  s->l = (uint32_t)l;
  s->n_vars = (uint32_t)vars;
  s->rows = (uint32_t)rows;
  s->logN = ceil_log2(rows);
  if (s->logN < 1) s->logN = 1;
  s->N = size_t(1) << s->logN;
  return ZKVC_OK;
}

Layout make_layout(const Shape& s) {
  Layout L{};
  const uint32_t nb = s.n * s.b, ab = s.a * s.b;
  const uint32_t n = (uint32_t)s.n;
  const uint32_t cnt1[R1_COUNT] = {s.l + 1, 1, 1, 1, nb, nb, n - 1, (uint32_t)s.N, ab, 1, s.l + 1, n, n};
  const uint32_t win1[R1_COUNT] = {1, ZKVC_W1, ZKVC_W1, ZKVC_W1, 1, 1, ZKVC_W1, ZKVC_W1, 4, 32, ZKVC_W1, 32, 32};
  const uint32_t c1[R1_COUNT] = {ZKVC_C1, ZKVC_C1, ZKVC_C1, ZKVC_C1, ZKVC_C1, ZKVC_C1, ZKVC_C1, ZKVC_C1, 8, 8, ZKVC_C1, 8, 8};
  uint64_t off = 0;
  for (int r = 0; r < R1_COUNT; r++) {
    L.g1[r] = {off, cnt1[r], win1[r], c1[r], r};
    off += uint64_t(cnt1[r]) * win1[r];
  }
  L.n_g1 = off;
  const uint32_t cnt2[R2_COUNT] = {nb, 1, 1, 1, n};
  const uint32_t win2[R2_COUNT] = {1, 1, ZKVC_W2_FULL, 1, ZKVC_W2_FULL};
  off = 0;
  for (int r = 0; r < R2_COUNT; r++) {
    L.g2[r] = {off, cnt2[r], win2[r], ZKVC_C2, r};
    off += uint64_t(cnt2[r]) * win2[r];
  }
  L.n_g2 = off;
  return L;
}

// ------------------------------------------------------------------ setup constants
__device__ __forceinline__ bool lt_modulus_fr(const Fr& x) {
  for (int i = 7; i >= 0; i--) {
    uint32_t m = mod_limb<FrCfg>(i);
    if (x.v[i] != m) return x.v[i] < m;
  }
  return false;
}

__global__ void k_setup_consts(const Fr* toxic, SetupConsts* sc, uint32_t logN, const Fr* dom_consts) {
  int bad = 0;
  Fr v[6];
  for (int i = 0; i < 6; i++) {
    Fr x = ld_field(toxic + i);
    if (!lt_modulus_fr(x)) bad |= 1;
    v[i] = f_to_mont(x);
  }
  Fr tN = v[0];
  for (uint32_t i = 0; i < logN; i++) tN = f_sqr(tN);
  Fr tN1 = f_sub(tN, Fr::one());
  if (tN1.is_zero()) bad |= 2;
  for (int i = 1; i <= 4; i++)
    if (v[i].is_zero()) bad |= 4;
  if (v[5].is_zero() || v[5] == Fr::one()) bad |= 8;
  SetupConsts s;
  s.tau = v[0];
  s.alpha = v[1];
  s.beta = v[2];
  s.gamma = v[3];
  s.delta = v[4];
  s.z = v[5];
  s.tN1 = tN1;
  s.c = f_mul(tN1, ld_field(dom_consts + 0));
  s.dinv = v[4].is_zero() ? Fr::zero() : f_inv(v[4]);
  s.ginv = v[3].is_zero() ? Fr::zero() : f_inv(v[3]);
  s.bad = bad;
  *sc = s;
}

__global__ void k_zpows(const SetupConsts* sc, Fr* zA, int a, Fr* zB, int b) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a + b) return;
  Fr z = sc->z;
  if (t < a)
    st_field(zA + t, pow_u32(z, (uint32_t)t * (uint32_t)b));
  else
    st_field(zB + (t - a), pow_u32(z, (uint32_t)(t - a)));
}

// omega^k from the half table omega^e (e < N/2): omega^(k + N/2) = -omega^k
__device__ __forceinline__ Fr omega_pow(const Fr* tw, size_t N, size_t k) {
  size_t h = N / 2;
  return k < h ? ld_field(tw + k) : f_neg(ld_field(tw + (k - h)));
}

__global__ void k_lagrange(const SetupConsts* sc, const Fr* tw, size_t N, uint32_t rows, Fr* L) {
  size_t k0 = (size_t(blockIdx.x) * blockDim.x + threadIdx.x) * LAG_CHUNK;
  if (k0 >= rows) return;
  size_t k1 = k0 + LAG_CHUNK < rows ? k0 + LAG_CHUNK : rows;
  Fr tau = sc->tau, c = sc->c;
  Fr pre[LAG_CHUNK];
  Fr acc = Fr::one();
  for (size_t k = k0; k < k1; k++) {
    acc = f_mul(acc, f_sub(tau, omega_pow(tw, N, k)));
    pre[k - k0] = acc;
  }
  Fr inv = f_inv(acc);
  for (size_t k = k1; k-- > k0;) {
    Fr d = f_sub(tau, omega_pow(tw, N, k));
    Fr ik = (k > k0) ? f_mul(inv, pre[k - k0 - 1]) : inv;   // 1 / (tau - omega^k)
    inv = f_mul(inv, d);
    st_field(L + k, f_mul(f_mul(c, omega_pow(tw, N, k)), ik));
  }
}

// ------------------------------------------------------------------ query scalars
enum : int { GRP_G1 = 1, GRP_G2 = 2, GRP_IC = 3 };

struct RegionTab {
  Region r[R1_COUNT];
  uint32_t entry_off[R1_COUNT + 1];
  int n;
};

__global__ void k_query_scalars(RegionTab tab, int group, const SetupConsts* __restrict__ scp, const Fr* __restrict__ L,
                                const Fr* __restrict__ zA, const Fr* __restrict__ zB, Shape sh, Fr* out) {
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tab.entry_off[tab.n]) return;
  int ri = 0;
  while (ri + 1 < tab.n && tab.entry_off[ri + 1] <= t) ri++;
  const Region rg = tab.r[ri];
  const uint32_t e = t - tab.entry_off[ri];
  const SetupConsts& sc = *scp;
  const uint32_t n = sh.n, b = sh.b, an = sh.a * sh.n;
  Fr s = Fr::zero();
  if (group == GRP_G1) {
    switch (rg.kind) {
      case R1_A: {
        uint32_t v = e;
        if (v == 0) {
          s = ld_field(L + n);
        } else if (v <= an) {
          uint32_t i = (v - 1) / n, k = (v - 1) % n;
          s = f_add(f_mul(ld_field(zA + i), ld_field(L + k)), ld_field(L + n + v));
        } else {
          s = ld_field(L + n + v);
        }
        break;
      }
      case R1_ALPHA: s = sc.alpha; break;
      case R1_BETA: s = sc.beta; break;
      case R1_DELTA: s = sc.delta; break;
      case R1_B: s = f_mul(ld_field(zB + e % b), ld_field(L + e / b)); break;
      case R1_LW: s = f_mul(f_mul(sc.alpha, sc.dinv), f_mul(ld_field(zB + e % b), ld_field(L + e / b))); break;
      case R1_LS: s = f_mul(f_sub(ld_field(L + e), ld_field(L + e + 1)), sc.dinv); break;
      case R1_H: {
        uint32_t j = bitrev_n(e, sh.logN);
        if (j + 1 < (uint32_t)sh.N) s = f_mul(pow_u32(sc.tau, j), f_mul(sc.tN1, sc.dinv));
        break;
      }
      case R1_AY8: s = ld_field(L + n + 1 + an + e); break;
      case R1_DELTA8: s = sc.delta; break;
      case R1_AIN: s = ld_field(L + n + e); break;
      case R1_LK: s = ld_field(L + e); break;
      case R1_ALK: s = f_mul(f_mul(sc.alpha, sc.dinv), ld_field(L + e)); break;
    }
  } else if (group == GRP_G2) {
    switch (rg.kind) {
      case R2_B: s = f_mul(ld_field(zB + e % b), ld_field(L + e / b)); break;
      case R2_BETA: s = sc.beta; break;
      case R2_DELTA: s = sc.delta; break;
      case R2_GAMMA: s = sc.gamma; break;
      case R2_LK: s = ld_field(L + e); break;
    }
  } else {  // verifying-key IC_v = (beta A_v + alpha B_v + C_v) / gamma, v = 0 .. l
    uint32_t v = e;
    Fr av, cv = Fr::zero();
    if (v == 0) {
      av = ld_field(L + n);
    } else if (v <= an) {
      uint32_t i = (v - 1) / n, k = (v - 1) % n;
      av = f_add(f_mul(ld_field(zA + i), ld_field(L + k)), ld_field(L + n + v));
    } else {
      uint32_t q = v - 1 - an, i = q / b, j = q % b;
      av = ld_field(L + n + v);
      cv = f_mul(f_mul(ld_field(zA + i), ld_field(zB + j)), ld_field(L + n - 1));
    }
    s = f_mul(f_add(f_mul(sc.beta, av), cv), sc.ginv);
  }
  Fr step = f_from_int<FrCfg>((int32_t)(1u << rg.c));  // 2^c
  uint64_t base = rg.off + uint64_t(e) * rg.nwin;
  for (uint32_t w = 0; w < rg.nwin; w++) {
    st_field(out + base + w, s);
    s = f_mul(s, step);
  }
}

// ------------------------------------------------------------------ fixed-base comb
template <class F>
__global__ void k_fb_seed(XYZZ<F>* tmp) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  XYZZ<F> P;
  if constexpr (sizeof(F) == sizeof(Fp))
    P = XYZZ<F>::from_affine(g1_generator());
  else
    P = XYZZ<F>::from_affine(g2_generator());
  for (int w = 0; w < 32; w++) {
    st_field(tmp + w * 256, XYZZ<F>::inf());
    st_field(tmp + w * 256 + 1, P);
    for (int i = 0; i < 8; i++) P = p_dbl(P);
  }
}

template <class F>
__global__ void k_fb_fill(XYZZ<F>* tmp) {
  int w = threadIdx.x;
  if (w >= 32) return;
  XYZZ<F> base = ld_field(tmp + w * 256 + 1), acc = base;
  for (int d = 2; d < 256; d++) {
    acc = p_add(acc, base);
    st_field(tmp + w * 256 + d, acc);
  }
}

static constexpr int NORM_CHUNK = 16;

// XYZZ -> affine (Montgomery) with one inversion per chunk of NORM_CHUNK points.
template <class F>
__global__ void k_normalize(const XYZZ<F>* __restrict__ in, Affine<F>* out, size_t n) {
  size_t i0 = (size_t(blockIdx.x) * blockDim.x + threadIdx.x) * NORM_CHUNK;
  if (i0 >= n) return;
  size_t i1 = i0 + NORM_CHUNK < n ? i0 + NORM_CHUNK : n;
  F pre[NORM_CHUNK];
  F acc = F::one();
  for (size_t i = i0; i < i1; i++) {
    XYZZ<F> p = ld_field(in + i);
    if (!p.is_inf()) acc = f_mul(acc, f_mul(p.ZZ, p.ZZZ));
    pre[i - i0] = acc;
  }
  F inv = f_inv(acc);
  for (size_t i = i1; i-- > i0;) {
    XYZZ<F> p = ld_field(in + i);
    if (p.is_inf()) {
      st_field(out + i, Affine<F>::inf());
      continue;
    }
    F ik = (i > i0) ? f_mul(inv, pre[i - i0 - 1]) : inv;  // 1 / (ZZ ZZZ)
    inv = f_mul(inv, f_mul(p.ZZ, p.ZZZ));
    Affine<F> a;
    a.x = f_mul(p.X, f_mul(ik, p.ZZZ));
    a.y = f_mul(p.Y, f_mul(ik, p.ZZ));
    st_field(out + i, a);
  }
}

template <class F>
__global__ void __launch_bounds__(256) k_fixed_base(const Fr* __restrict__ scal, size_t n, const Affine<F>* __restrict__ T,
                                                    XYZZ<F>* out, int canonical = 0) {
  size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Fr k = ld_field(scal + i);
  if (!canonical) k = f_from_mont(k);
  XYZZ<F> acc = XYZZ<F>::inf();
#pragma unroll 1
  for (int w = 0; w < 32; w++) {
    uint32_t byte = (k.v[w >> 2] >> (8 * (w & 3))) & 255u;
    if (byte) acc = p_add_affine(acc, ld_field(T + w * 256 + byte));
  }
  st_field(out + i, acc);
}

template <class F>
static int normalize(const XYZZ<F>* in, Affine<F>* out, size_t n, cudaStream_t st) {
  size_t chunks = (n + NORM_CHUNK - 1) / NORM_CHUNK;
  k_normalize<F><<<(unsigned)((chunks + 127) / 128), 128, 0, st>>>(in, out, n); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

static std::mutex g_tab_mu;
static std::map<int, std::pair<G1A*, G2A*>> g_tables;

template <class F>
static int build_table(Affine<F>** out, cudaStream_t st) {
  XYZZ<F>* tmp = nullptr;
  ZK_CUDA(cudaMalloc(&tmp, 32 * 256 * sizeof(XYZZ<F>)));
  ZK_CUDA(cudaMalloc(out, 32 * 256 * sizeof(Affine<F>)));
  k_fb_seed<F><<<1, 1, 0, st>>>(tmp); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  k_fb_fill<F><<<1, 32, 0, st>>>(tmp); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  ZK_TRY(normalize<F>(tmp, *out, 32 * 256, st));
  ZK_CUDA(cudaStreamSynchronize(st));
  ZK_CUDA(cudaFree(tmp));
  return ZKVC_OK;
}

int fb_tables(G1A** t1, G2A** t2, cudaStream_t st) {
  int dev = 0;
  ZK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_tab_mu);
  auto it = g_tables.find(dev);
  if (it == g_tables.end()) {
    G1A* a = nullptr;
    G2A* b = nullptr;
    ZK_TRY(build_table<Fp>(&a, st));
    ZK_TRY(build_table<Fp2>(&b, st));
    it = g_tables.emplace(dev, std::make_pair(a, b)).first;
  }
  *t1 = it->second.first;
  *t2 = it->second.second;
  return ZKVC_OK;
}

// scalars (Montgomery) -> affine bases, in chunks to bound the XYZZ temporary
template <class F>
int points_from_scalars(const Fr* scal, size_t n, const Affine<F>* T, Affine<F>* out, XYZZ<F>* tmp,
                               size_t chunk, cudaStream_t st) {
  for (size_t s = 0; s < n; s += chunk) {
    size_t m = n - s < chunk ? n - s : chunk;
    k_fixed_base<F><<<(unsigned)((m + 255) / 256), 256, 0, st>>>(scal + s, m, T, tmp); ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaGetLastError());
    ZK_TRY(normalize<F>(tmp, out + s, m, st));
  }
  return ZKVC_OK;
}

static RegionTab region_tab(const Region* r, int n) {
  RegionTab t{};
  t.n = n;
  uint32_t e = 0;
  for (int i = 0; i < n; i++) {
    t.r[i] = r[i];
    t.entry_off[i] = e;
    e += r[i].count;
  }
  t.entry_off[n] = e;
  return t;
}

template <class F>
__global__ void k_export(const Affine<F>* src, const uint64_t* idx, size_t count, Affine<F>* dst) {
  size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= count) return;
  Affine<F> a = ld_field(src + idx[i]);
  a.x = f_from_mont(a.x);
  a.y = f_from_mont(a.y);
  st_field(dst + i, a);
}

template <class F>
int export_points(const Affine<F>* src, const std::vector<uint64_t>& idx, uint8_t* host_out, cudaStream_t st) {
  if (idx.empty()) return ZKVC_OK;
  uint64_t* d_idx = nullptr;
  Affine<F>* d_out = nullptr;
  ZK_CUDA(cudaMalloc(&d_idx, idx.size() * sizeof(uint64_t)));
  ZK_CUDA(cudaMalloc(&d_out, idx.size() * sizeof(Affine<F>)));
  ZK_CUDA(cudaMemcpyAsync(d_idx, idx.data(), idx.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  k_export<F><<<(unsigned)((idx.size() + 255) / 256), 256, 0, st>>>(src, d_idx, idx.size(), d_out); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  ZK_CUDA(cudaMemcpyAsync(host_out, d_out, idx.size() * sizeof(Affine<F>), cudaMemcpyDeviceToHost, st));
  ZK_CUDA(cudaStreamSynchronize(st));
  ZK_CUDA(cudaFree(d_idx));
  ZK_CUDA(cudaFree(d_out));
  return ZKVC_OK;
}

template int export_points<Fp>(const G1A*, const std::vector<uint64_t>&, uint8_t*, cudaStream_t);
template int points_from_scalars<Fp>(const Fr*, size_t, const G1A*, G1A*, XYZZ<Fp>*, size_t, cudaStream_t);
template int points_from_scalars<Fp2>(const Fr*, size_t, const G2A*, G2A*, XYZZ<Fp2>*, size_t, cudaStream_t);
template int export_points<Fp2>(const G2A*, const std::vector<uint64_t>&, uint8_t*, cudaStream_t);


template <class F>
__global__ void k_points_canonical(Affine<F>* p, size_t n) {
  size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Affine<F> a = ld_field(p + i);
  a.x = f_from_mont(a.x);
  a.y = f_from_mont(a.y);
  st_field(p + i, a);
}

static constexpr size_t GEN_CHUNK = size_t(1) << 20;

template <class F>
size_t generator_mul_ws(size_t n) {
  return (n < GEN_CHUNK ? n : GEN_CHUNK) * sizeof(XYZZ<F>) + 256;
}

// out[i] = [k_i] G (canonical affine) for canonical scalars k_i: the fixed-base comb of
// setup applied to caller data.
template <class F>
int generator_mul(const uint8_t* d_scalars, size_t n, uint8_t* d_out, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (n == 0) return ZKVC_OK;
  ZK_CHECK(d_scalars && d_out && ws, ZKVC_EINVAL, "generator_mul: null pointer");
  ZK_CHECK(ws_bytes >= generator_mul_ws<F>(n), ZKVC_EINVAL, "generator_mul: workspace too small");
  G1A* T1 = nullptr;
  G2A* T2 = nullptr;
  ZK_TRY(fb_tables(&T1, &T2, st));
  const Affine<F>* T;
  if constexpr (sizeof(F) == sizeof(Fp))
    T = T1;
  else
    T = T2;
  const Fr* sc = reinterpret_cast<const Fr*>(d_scalars);
  Affine<F>* out = reinterpret_cast<Affine<F>*>(d_out);
  XYZZ<F>* tmp = reinterpret_cast<XYZZ<F>*>(ws);
  for (size_t s = 0; s < n; s += GEN_CHUNK) {
    size_t m = n - s < GEN_CHUNK ? n - s : GEN_CHUNK;
    k_fixed_base<F><<<(unsigned)((m + 255) / 256), 256, 0, st>>>(sc + s, m, T, tmp, 1); ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaGetLastError());
    ZK_TRY(normalize<F>(tmp, out + s, m, st));
  }
  k_points_canonical<F><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

template size_t generator_mul_ws<Fp>(size_t);
template size_t generator_mul_ws<Fp2>(size_t);
template int generator_mul<Fp>(const uint8_t*, size_t, uint8_t*, void*, size_t, cudaStream_t);
template int generator_mul<Fp2>(const uint8_t*, size_t, uint8_t*, void*, size_t, cudaStream_t);

int setup_impl(int a, int n, int b, const uint8_t* toxic, cudaStream_t st, zkvc_pk** pk_out, zkvc_vk** vk_out) {
  Shape sh;
  ZK_TRY(make_shape(a, n, b, &sh));
  Layout lay = make_layout(sh);
  const NttDomain* dom = nullptr;
  ZK_TRY(ntt_domain(sh.logN, &dom));
  G1A* T1 = nullptr;
  G2A* T2 = nullptr;
  ZK_TRY(fb_tables(&T1, &T2, st));

  DevTemps tmp;
  Fr* d_toxic = nullptr;
  SetupConsts* d_sc = nullptr;
  Fr* d_L = nullptr;
  ZK_TRY(tmp.alloc(&d_toxic, 6));
  ZK_TRY(tmp.alloc(&d_sc, 1));
  ZK_TRY(tmp.alloc(&d_L, sh.rows));
  ZK_CUDA(cudaMemcpyAsync(d_toxic, toxic, 6 * 32, cudaMemcpyHostToDevice, st));
  k_setup_consts<<<1, 1, 0, st>>>(d_toxic, d_sc, sh.logN, dom->consts); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  int bad = 0;
  ZK_CUDA(cudaMemcpyAsync(&bad, &d_sc->bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  ZK_CUDA(cudaStreamSynchronize(st));
  ZK_CHECK(!(bad & 1), ZKVC_EINVAL, "setup: a toxic-waste value is not a canonical Fr element");
  ZK_CHECK(!(bad & 2), ZKVC_EINVAL, "setup: tau lies in the evaluation domain (tau^N = 1)");
  ZK_CHECK(!(bad & 4), ZKVC_EINVAL, "setup: alpha, beta, gamma and delta must be nonzero");
  ZK_CHECK(!(bad & 8), ZKVC_EINVAL, "setup: the CRPC point z must not be 0 or 1");

  zkvc_pk* pk = new zkvc_pk();
  pk->shape = sh;
  pk->lay = lay;
  pk->dom = dom;
  ZK_CUDA(cudaGetDevice(&pk->device));
  auto fail = [&](int rc) {
    cudaFree(pk->g1);
    cudaFree(pk->g2);
    cudaFree(pk->zA);
    cudaFree(pk->zB);
    delete pk;
    return rc;
  };
  if (cudaMalloc(&pk->g1, lay.n_g1 * sizeof(G1A)) != cudaSuccess ||
      cudaMalloc(&pk->g2, lay.n_g2 * sizeof(G2A)) != cudaSuccess ||
      cudaMalloc(&pk->zA, sh.a * sizeof(Fr)) != cudaSuccess || cudaMalloc(&pk->zB, sh.b * sizeof(Fr)) != cudaSuccess) {
    set_error("setup: proving key allocation failed (%zu G1 + %zu G2 bases)", (size_t)lay.n_g1, (size_t)lay.n_g2);
    return fail(ZKVC_ENOMEM);
  }
  int rc = ZKVC_OK;
  do {
    k_zpows<<<(sh.a + sh.b + 127) / 128, 128, 0, st>>>(d_sc, pk->zA, sh.a, pk->zB, sh.b); ZK_COUNT_LAUNCH();
    size_t lag_threads = (sh.rows + LAG_CHUNK - 1) / LAG_CHUNK;
    k_lagrange<<<(unsigned)((lag_threads + 127) / 128), 128, 0, st>>>(d_sc, dom->tw_fwd, sh.N, sh.rows, d_L); ZK_COUNT_LAUNCH();
    if (cudaGetLastError() != cudaSuccess) {
      rc = ZKVC_ECUDA;
      break;
    }
    const size_t chunk = size_t(1) << 20;
    // G1
    Fr* scal = nullptr;
    size_t max_n = lay.n_g1 > sh.l + 1 ? lay.n_g1 : sh.l + 1;
    if ((rc = tmp.alloc(&scal, max_n)) != ZKVC_OK) break;
    XYZZ<Fp2>* xtmp = nullptr;  // large enough for G1 or G2 chunks
    if ((rc = tmp.alloc(&xtmp, chunk)) != ZKVC_OK) break;
    RegionTab t1 = region_tab(lay.g1, R1_COUNT);
    k_query_scalars<<<(t1.entry_off[R1_COUNT] + 255) / 256, 256, 0, st>>>(t1, GRP_G1, d_sc, d_L, pk->zA, pk->zB, sh, scal); ZK_COUNT_LAUNCH();
    if ((rc = points_from_scalars<Fp>(scal, lay.n_g1, T1, pk->g1, reinterpret_cast<XYZZ<Fp>*>(xtmp), 2 * chunk, st)) != ZKVC_OK) break;
    // G2
    RegionTab t2 = region_tab(lay.g2, R2_COUNT);
    k_query_scalars<<<(t2.entry_off[R2_COUNT] + 255) / 256, 256, 0, st>>>(t2, GRP_G2, d_sc, d_L, pk->zA, pk->zB, sh, scal); ZK_COUNT_LAUNCH();
    if ((rc = points_from_scalars<Fp2>(scal, lay.n_g2, T2, pk->g2, xtmp, chunk, st)) != ZKVC_OK) break;
    // verifying key: IC_v for v = 0 .. l
    Region ric{0, sh.l + 1, 1, ZKVC_C2, 0};
    RegionTab t3 = region_tab(&ric, 1);
    G1A* ic = nullptr;
    if ((rc = tmp.alloc(&ic, sh.l + 1)) != ZKVC_OK) break;
    k_query_scalars<<<(sh.l + 1 + 255) / 256, 256, 0, st>>>(t3, GRP_IC, d_sc, d_L, pk->zA, pk->zB, sh, scal); ZK_COUNT_LAUNCH();
    if ((rc = points_from_scalars<Fp>(scal, sh.l + 1, T1, ic, reinterpret_cast<XYZZ<Fp>*>(xtmp), 2 * chunk, st)) != ZKVC_OK) break;
    if (cudaGetLastError() != cudaSuccess) {
      rc = ZKVC_ECUDA;
      break;
    }
    zkvc_vk* vk = new zkvc_vk();
    vk->shape = sh;
    vk->alpha1.resize(64);
    vk->beta2.resize(128);
    vk->gamma2.resize(128);
    vk->delta2.resize(128);
    vk->ic.resize(size_t(sh.l + 1) * 64);
    std::vector<uint64_t> idx(sh.l + 1);
    for (size_t i = 0; i <= sh.l; i++) idx[i] = i;
    if ((rc = export_points<Fp>(ic, idx, vk->ic.data(), st)) != ZKVC_OK ||
        (rc = export_points<Fp>(pk->g1, {lay.g1[R1_ALPHA].off}, vk->alpha1.data(), st)) != ZKVC_OK ||
        (rc = export_points<Fp2>(pk->g2, {lay.g2[R2_BETA].off}, vk->beta2.data(), st)) != ZKVC_OK ||
        (rc = export_points<Fp2>(pk->g2, {lay.g2[R2_GAMMA].off}, vk->gamma2.data(), st)) != ZKVC_OK ||
        (rc = export_points<Fp2>(pk->g2, {lay.g2[R2_DELTA].off}, vk->delta2.data(), st)) != ZKVC_OK) {
      delete vk;
      break;
    }
    *vk_out = vk;
  } while (0);
  if (rc == ZKVC_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error("setup: %s", cudaGetErrorString(e));
      rc = ZKVC_ECUDA;
    }
  }
  if (rc != ZKVC_OK) {
    if (zkvc_last_error()[0] == 0) set_error("setup: CUDA launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(rc);
  }
  *pk_out = pk;
  return ZKVC_OK;
}

}  // namespace zkvc
