// C-ABI entry points for the kernel layer: field products, NTT, variable-base MSM.
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <thread>

#include "glv.h"
#include "msm.h"
#include "ntt.h"

namespace zkvc {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

static void clear_error() { g_err.clear(); }

const char* last_error_text() { return g_err.c_str(); }

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void uncount_launches(unsigned long long n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

static std::atomic<int> g_sm_count[64];

int device_sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    cudaGetLastError();
    return 1;
  }
  if (dev < 64) {
    int c = g_sm_count[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int c = 0;
  if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0) {
    cudaGetLastError();
    return 1;
  }
  if (dev < 64) g_sm_count[dev].store(c, std::memory_order_relaxed);
  return c;
}

static std::atomic<int> g_wait_ms{60000};

int wait_stream(cudaStream_t st, const char* what) {
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  const long long limit = g_wait_ms.load(std::memory_order_relaxed);
  long long sleep_us = 0;
  for (;;) {
    cudaError_t e = cudaStreamQuery(st);
    if (e == cudaSuccess) return ZKVC_OK;
    if (e != cudaErrorNotReady) {
      set_error("%s: %s", what, cudaGetErrorString(e));
      return ZKVC_ECUDA;
    }
    long long el = std::chrono::duration_cast<std::chrono::milliseconds>(clk::now() - t0).count();
    if (el >= limit) {
      set_error("%s: device work not finished after %lld ms", what, el);
      return ZKVC_ETIMEOUT;
    }
    // poll tightly for the first ~100 us, then back off up to 1 ms
    if (sleep_us > 0) std::this_thread::sleep_for(std::chrono::microseconds(sleep_us));
    sleep_us = sleep_us == 0 ? 1 : (sleep_us * 2 > 1000 ? 1000 : sleep_us * 2);
  }
}

struct ProfSlot {
  const char* name;
  cudaEvent_t b = nullptr, e = nullptr;
  uint32_t* host_units = nullptr;
  bool pending = false;
  double ms = 0;
  double start_ms = 0, end_ms = 0;  // offsets of the begin and end events from the witness begin
  unsigned long long calls = 0, units = 0;
};
static ProfSlot g_prof_slots[PS_COUNT] = {{"witness"},   {"ntt"},    {"msm_g1"},  {"msm_g1_bucket_accum"},
                                          {"msm_g2"},    {"msm_g2_bucket_accum"}, {"combine"},
                                          {"msm_g1_small"}};
static std::atomic<bool> g_prof{false};

void prof_mark(int stage, bool begin, cudaStream_t st) {
  if (!g_prof.load(std::memory_order_relaxed)) return;
  ProfSlot& x = g_prof_slots[stage];
  if (!x.b) {
    cudaEventCreate(&x.b);
    cudaEventCreate(&x.e);
    cudaMallocHost(&x.host_units, sizeof(uint32_t));
    *x.host_units = 0;
  }
  cudaEventRecord(begin ? x.b : x.e, st);
  if (!begin) x.pending = true;
}

bool prof_enabled() { return g_prof.load(std::memory_order_relaxed); }

uint32_t* prof_units(int stage) {
  if (!g_prof.load(std::memory_order_relaxed)) return nullptr;
  return g_prof_slots[stage].host_units;
}

void prof_collect() {
  if (!g_prof.load(std::memory_order_relaxed)) return;
  const ProfSlot& ref = g_prof_slots[PS_WITNESS];
  const bool spans = ref.pending;
  for (auto& x : g_prof_slots) {
    if (!x.pending) continue;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, x.b, x.e) == cudaSuccess) x.ms += ms;
    if (spans && cudaEventElapsedTime(&ms, ref.b, x.b) == cudaSuccess) x.start_ms += ms;
    if (spans && cudaEventElapsedTime(&ms, ref.b, x.e) == cudaSuccess) x.end_ms += ms;
    x.calls++;
    x.units += *x.host_units;
    *x.host_units = 0;
    x.pending = false;
  }
}

// ------------------------------------------------------------------ field products
template <class C>
__global__ void k_field_mul(const Field<C>* a, const Field<C>* b, Field<C>* out, size_t n) {
  size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // (a R) b / R = a b: one conversion and one Montgomery product, canonical in and out
  st_field(out + i, f_mul(f_to_mont(ld_field(a + i)), ld_field(b + i)));
}

// a^-1 (0 -> 0): Montgomery form in, inversion (binary GCD), canonical out
template <class C>
__global__ void k_field_inv(const Field<C>* a, Field<C>* out, size_t n) {
  size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  st_field(out + i, f_from_mont(f_inv(f_to_mont(ld_field(a + i)))));
}

__global__ void k_fp2_mul(const Fp2* a, const Fp2* b, Fp2* out, size_t n) {
  size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Fp2 x = ld_field(a + i);
  x = f_to_mont(x);
  st_field(out + i, f_mul(x, ld_field(b + i)));
}

// ------------------------------------------------------------------ points
template <class F>
__global__ void k_points_to_mont(const Affine<F>* in, Affine<F>* out, size_t n) {
  size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Affine<F> p = ld_field(in + i);
  p.x = f_to_mont(p.x);
  p.y = f_to_mont(p.y);
  st_field(out + i, p);
}

template <class F>
__global__ void k_export_point(const XYZZ<F>* in, Affine<F>* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Affine<F> a = p_to_affine(ld_field(in));
  a.x = f_from_mont(a.x);
  a.y = f_from_mont(a.y);
  st_field(out, a);
}

static uint32_t window_bits(size_t n) {
  uint32_t lg = ceil_log2(n < 2 ? 2 : n);
  int c = (int)lg - 3;
  if (c < 4) c = 4;
  if (c > 16) c = 16;
  return (uint32_t)c;
}

// Both groups take a two-way endomorphism split of every scalar (glv.h): in G1
// s P = k1 P + k2 phi(P) (GLV, |k1|, |k2| < 2^127), in G2 s Q = k1 Q + k2 psi(Q)
// (k1, k2 in [0, 2^127)).  The run then has 2n points of 127-bit scalars: as many bucket
// terms as n points of 254-bit scalars, but half the windows, hence half the buckets to
// reduce and half of Horner's chain of doublings over the windows (the latency-bound
// tail of a variable-base MSM).
template <class F>
constexpr bool msm_api_glv() { return true; }

static int variable_base_plan(size_t n, const void* scalars, bool glv, MsmPlan* out) {
  MsmPlan& p = *out;
  const size_t pts = glv ? 2 * n : n;
  const uint32_t bits = glv ? 128 : 255;
  // the window rule's c, then the smallest c with the same window count, so that the top
  // window is not left with a bit or two (all of its terms in one or two huge buckets)
  const uint32_t nd = (bits + window_bits(pts) - 1) / window_bits(pts);
  const uint32_t c = (bits + nd - 1) / nd;
  MsmOut o{};
  o.c = c;
  o.win_keys = nd;
  p.outs.push_back(o);
  MsmSeg s{};
  s.base_off = 0;
  s.count = (uint32_t)pts;
  s.nwin = 1;
  s.out = 0;
  s.kind = glv ? SK_SIGNED127 : SK_FR_CANON;
  s.scalars = scalars;
  s.skip = 0xffffffffu;
  p.segs.push_back(s);
  return msm_plan_finalize(p);
}

template <class F>
size_t msm_api_ws(size_t n) {
  constexpr bool glv = msm_api_glv<F>();
  const size_t pts = glv ? 2 * n : n;
  MsmPlan p;
  if (n > ZKVC_MSM_MAX_POINTS || variable_base_plan(n, nullptr, glv, &p) != ZKVC_OK) return 0;
  return msm_workspace_bytes<F>(p) + round256(pts * sizeof(Affine<F>)) + (glv ? round256(pts * sizeof(uint4)) : 0) +
         2 * 256 + sizeof(XYZZ<F>) + sizeof(Affine<F>);
}

// bases[i] = P_i and bases[n + i] = phi(P_i) = (beta x_i, y_i) in Montgomery form;
// halves[i], halves[n + i] = the GLV halves k1, k2 of s_i (reduced mod r first)
__global__ void k_glv_prep(const Affine<Fp>* __restrict__ pts, const Fr* __restrict__ sc, size_t n,
                           Affine<Fp>* bases, uint4* halves) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Affine<Fp> p = ld_field(pts + i);
  p.x = f_to_mont(p.x);
  p.y = f_to_mont(p.y);
  Fp beta;
#pragma unroll
  for (int l = 0; l < 8; l++) beta.v[l] = glv_beta_limb(l);
  Affine<Fp> q;
  q.x = f_mul(p.x, f_to_mont(beta));
  q.y = p.y;
  st_field(bases + i, p);
  st_field(bases + n + i, q);
  Fr k = ld_field(sc + i);
  const Fr r = Fr::modulus();
  for (int t = 0; t < 6; t++) {  // 2^256 < 6 r
    uint32_t d[8];
    if (sub8(d, k.v, r.v)) break;
#pragma unroll
    for (int l = 0; l < 8; l++) k.v[l] = d[l];
  }
  uint4 h1, h2;
  glv_split_dev(k.v, &h1, &h2);
  halves[i] = h1;
  halves[n + i] = h2;
}

// bases[i] = Q_i and bases[n + i] = psi(Q_i) = (conj(x_i) gx, conj(y_i) gy) in Montgomery
// form; halves[i], halves[n + i] = k1, k2 of s_i = k1 + k2 lambda2 (reduced mod r first)
__global__ void k_psi_prep(const Affine<Fp2>* __restrict__ pts, const Fr* __restrict__ sc, size_t n,
                           Affine<Fp2>* bases, uint4* halves) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Affine<Fp2> p = ld_field(pts + i);
  p.x = f_to_mont(p.x);
  p.y = f_to_mont(p.y);
  Fp2 gx, gy;
#pragma unroll
  for (int l = 0; l < 8; l++) {
    gx.c0.v[l] = psi_gx_limb(0, l);
    gx.c1.v[l] = psi_gx_limb(1, l);
    gy.c0.v[l] = psi_gy_limb(0, l);
    gy.c1.v[l] = psi_gy_limb(1, l);
  }
  Affine<Fp2> q;
  Fp2 cx = p.x, cy = p.y;
  cx.c1 = f_neg(cx.c1);
  cy.c1 = f_neg(cy.c1);
  q.x = f_mul(cx, f_to_mont(gx));
  q.y = f_mul(cy, f_to_mont(gy));
  st_field(bases + i, p);
  st_field(bases + n + i, q);
  Fr k = ld_field(sc + i);
  const Fr r = Fr::modulus();
  for (int t = 0; t < 6; t++) {  // 2^256 < 6 r
    uint32_t d[8];
    if (sub8(d, k.v, r.v)) break;
#pragma unroll
    for (int l = 0; l < 8; l++) k.v[l] = d[l];
  }
  uint4 h1, h2;
  psi_split_dev(k.v, &h1, &h2);
  halves[i] = h1;
  halves[n + i] = h2;
}

template <class F>
int msm_api(const uint8_t* d_points, const uint8_t* d_scalars, size_t n, void* d_ws, size_t ws_bytes,
            uint8_t* out, cudaStream_t st) {
  constexpr bool glv = msm_api_glv<F>();
  ZK_CHECK(out != nullptr, ZKVC_EINVAL, "msm: null output");
  ZK_CHECK(n <= ZKVC_MSM_MAX_POINTS, ZKVC_EINVAL, "msm: n = %zu above %u", n, (unsigned)ZKVC_MSM_MAX_POINTS);
  if (n == 0) {
    memset(out, 0, sizeof(Affine<F>));
    return ZKVC_OK;
  }
  ZK_CHECK(d_points && d_scalars && d_ws, ZKVC_EINVAL, "msm: null device pointer");
  MsmPlan p;
  ZK_TRY(variable_base_plan(n, nullptr, glv, &p));
  size_t need = msm_api_ws<F>(n);
  ZK_CHECK(ws_bytes >= need, ZKVC_EINVAL, "msm: workspace %zu < %zu bytes", ws_bytes, need);
  Arena a;
  a.base = reinterpret_cast<uint8_t*>(d_ws);
  a.cap = ws_bytes;
  const size_t pts = glv ? 2 * n : n;
  Affine<F>* bases = a.take<Affine<F>>(pts);
  uint4* halves = glv ? a.take<uint4>(pts) : nullptr;
  XYZZ<F>* res = a.take<XYZZ<F>>(1);
  Affine<F>* aff = a.take<Affine<F>>(1);
  uint8_t* rest = a.base + a.off;
  size_t rest_bytes = ws_bytes - a.off;
  if constexpr (glv && sizeof(F) == sizeof(Fp)) {
    k_glv_prep<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const Affine<Fp>*>(d_points),
                                                             reinterpret_cast<const Fr*>(d_scalars), n, bases, halves);
  } else if constexpr (glv) {
    k_psi_prep<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const Affine<Fp2>*>(d_points),
                                                             reinterpret_cast<const Fr*>(d_scalars), n, bases, halves);
  } else {
    k_points_to_mont<F><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        reinterpret_cast<const Affine<F>*>(d_points), bases, n);
  }
  ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  p.segs[0].scalars = glv ? static_cast<const void*>(halves) : d_scalars;
  ZK_TRY(msm_run<F>(p, bases, rest, rest_bytes, res, st));
  k_export_point<F><<<1, 32, 0, st>>>(res, aff); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  ZK_CUDA(cudaMemcpyAsync(out, aff, sizeof(Affine<F>), cudaMemcpyDeviceToHost, st));
  ZK_CUDA(cudaStreamSynchronize(st));
  return ZKVC_OK;
}

template int msm_api<Fp>(const uint8_t*, const uint8_t*, size_t, void*, size_t, uint8_t*, cudaStream_t);
template size_t msm_api_ws<Fp>(size_t);

// ------------------------------------------------------------------ integer-pipe rate
// Throughput microbenchmark of the 32-bit multiply-adds that Montgomery products are made
// of, counted as the products' IMADs are (a 32 x 32 -> 64-bit product is two: its low
// and its high word).  Every form runs 16 such IMADs per thread and iteration:
//   0  sixteen independent mad.lo.u32 chains
//   1  the CIOS row of the field code: a carry chain of eight mad.lo.cc / madc.lo.cc,
//      then eight mad.hi.cc / madc.hi.cc
//   2  sixteen independent mad.hi.u32 chains
//   3  eight independent mad.wide.u32 chains (64-bit accumulators; two IMADs each)
//   4  two carry chains of eight mad.lo.cc / madc.lo.cc
//   5  whole Fp Montgomery products, the inlined carry-chain CIOS (f_mul): two independent
//      product chains per thread, 264 IMADs per product
//   6  the same with the out-of-line 64-bit-accumulator CIOS of the point formulas (f_mulc)
// A full-occupancy grid of 256-thread blocks covers all SMs.  The result xor goes to
// `sink` so that nothing is dead code.
template <int FORM>
__global__ void __launch_bounds__(256) k_imad_rate(uint32_t iters, uint32_t seed, uint32_t* sink) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t t[16];
#pragma unroll
  for (int j = 0; j < 16; j++) t[j] = g * 2654435761u + seed * (j + 1);
  const uint32_t x = seed | 1u, y = g ^ 0x9e3779b9u;
  uint64_t w[8];
#pragma unroll
  for (int j = 0; j < 8; j++) w[j] = (uint64_t(t[j]) << 32) | t[j + 8];
  for (uint32_t it = 0; it < iters; it++) {
    if constexpr (FORM == 0) {
#pragma unroll
      for (int j = 0; j < 16; j++) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(t[j]) : "r"(x), "r"(y));
    } else if constexpr (FORM == 2) {
#pragma unroll
      for (int j = 0; j < 16; j++) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(t[j]) : "r"(x), "r"(y));
    } else if constexpr (FORM == 3) {
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const uint32_t lo = (uint32_t)w[j];
        asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[j]) : "r"(lo), "r"(x));
      }
    } else if constexpr (FORM == 4) {
      const uint32_t b = (t[7] ^ t[15]) | 1u;  // changes every iteration: no product is invariant
#pragma unroll
      for (int h = 0; h < 2; h++)
        asm volatile(
            "mad.lo.cc.u32  %0, %8,  %16, %0;\n\t"
            "madc.lo.cc.u32 %1, %9,  %16, %1;\n\t"
            "madc.lo.cc.u32 %2, %10, %16, %2;\n\t"
            "madc.lo.cc.u32 %3, %11, %16, %3;\n\t"
            "madc.lo.cc.u32 %4, %12, %16, %4;\n\t"
            "madc.lo.cc.u32 %5, %13, %16, %5;\n\t"
            "madc.lo.cc.u32 %6, %14, %16, %6;\n\t"
            "madc.lo.u32    %7, %15, %16, %7;"
            : "+r"(t[8 * h + 0]), "+r"(t[8 * h + 1]), "+r"(t[8 * h + 2]), "+r"(t[8 * h + 3]), "+r"(t[8 * h + 4]),
              "+r"(t[8 * h + 5]), "+r"(t[8 * h + 6]), "+r"(t[8 * h + 7])
            : "r"(t[8 - 8 * h]), "r"(t[9 - 8 * h]), "r"(t[10 - 8 * h]), "r"(t[11 - 8 * h]), "r"(t[12 - 8 * h]),
              "r"(t[13 - 8 * h]), "r"(t[14 - 8 * h]), "r"(t[15 - 8 * h]), "r"(b));
    } else {
      const uint32_t b = t[15] | 1u;
      asm volatile(
          "mad.lo.cc.u32  %0, %9,  %17, %0;\n\t"
          "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"
          "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"
          "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"
          "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"
          "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"
          "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"
          "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"
          "addc.u32       %8, %8, 0;\n\t"
          "mad.hi.cc.u32  %1, %9,  %17, %1;\n\t"
          "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"
          "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"
          "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"
          "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"
          "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"
          "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"
          "madc.hi.u32    %8, %16, %17, %8;"
          : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]),
            "+r"(t[15])
          : "r"(t[8]), "r"(t[9]), "r"(t[10]), "r"(t[11]), "r"(t[12]), "r"(t[13]), "r"(t[14]), "r"(x), "r"(b));
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < 16; j++) acc ^= t[j];
#pragma unroll
  for (int j = 0; j < 8; j++) acc ^= (uint32_t)w[j] ^ (uint32_t)(w[j] >> 32);
  if (acc == 0x12345678u) sink[0] = acc;
}

// Product-scanning Montgomery multiplication (finely integrated: every column sums its
// a_j b_(i-j) and m_j p_(i-j) terms into a 96-bit accumulator, and the low word of column
// i < 8 yields m_i), written out for the throughput comparison of zkvc_imad_rate: WIDE = 0
// accumulates with mad.lo.cc / madc.hi.cc / addc (the field code's f_mul), WIDE = 1 (form
// 8) with one 64-bit product (mul.wide) and three additions.
template <int WIDE>
__device__ __forceinline__ void col_acc(uint32_t& t0, uint32_t& t1, uint32_t& t2, uint32_t x, uint32_t y) {
  if constexpr (WIDE) {
    const uint64_t p = (uint64_t)x * y;
    asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.u32 %2, %2, 0;"
        : "+r"(t0), "+r"(t1), "+r"(t2)
        : "r"((uint32_t)p), "r"((uint32_t)(p >> 32)));
  } else {
    asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\tmadc.hi.cc.u32 %1, %3, %4, %1;\n\taddc.u32 %2, %2, 0;"
        : "+r"(t0), "+r"(t1), "+r"(t2)
        : "r"(x), "r"(y));
  }
}

template <int WIDE>
__device__ __forceinline__ Fp f_mul_fips(const Fp& a, const Fp& b) {
  uint32_t m[8], r[8];
  uint32_t t0 = 0, t1 = 0, t2 = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
#pragma unroll
    for (int j = 0; j < i; j++) {
      col_acc<WIDE>(t0, t1, t2, a.v[j], b.v[i - j]);
      col_acc<WIDE>(t0, t1, t2, m[j], mod_limb<FpCfg>(i - j));
    }
    col_acc<WIDE>(t0, t1, t2, a.v[i], b.v[0]);
    m[i] = t0 * FpCfg::INV;
    col_acc<WIDE>(t0, t1, t2, m[i], mod_limb<FpCfg>(0));
    t0 = t1;
    t1 = t2;
    t2 = 0;
  }
#pragma unroll
  for (int i = 8; i < 15; i++) {
#pragma unroll
    for (int j = i - 7; j < 8; j++) {
      col_acc<WIDE>(t0, t1, t2, a.v[j], b.v[i - j]);
      col_acc<WIDE>(t0, t1, t2, m[j], mod_limb<FpCfg>(i - j));
    }
    r[i - 8] = t0;
    t0 = t1;
    t1 = t2;
    t2 = 0;
  }
  r[7] = t0;  // the value r < 2p < 2^255: no word beyond
  Fp x, d;
#pragma unroll
  for (int i = 0; i < 8; i++) x.v[i] = r[i];
  const Fp mm = Fp::modulus();
  const uint32_t br = sub8(d.v, x.v, mm.v);
  return br ? x : d;
}

template <int FORM>
__global__ void __launch_bounds__(256) k_mont_rate(uint32_t iters, uint32_t seed, uint32_t* sink) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  Fp a = Fp::one(), b = Fp::one(), m = Fp::one();
  a.v[0] ^= g;
  b.v[1] ^= g * 7u;
  m.v[2] ^= seed;
  for (uint32_t it = 0; it < iters; it++) {
    if constexpr (FORM == 5) {
      a = f_mul_cios(a, m);
      b = f_mul_cios(b, m);
    } else if constexpr (FORM == 6) {
      a = f_mulc_cios(a, m);
      b = f_mulc_cios(b, m);
    } else if constexpr (FORM == 7) {
      a = f_mul(a, m);
      b = f_mul(b, m);
    } else if constexpr (FORM == 8) {
      a = f_mul_fips<1>(a, m);
      b = f_mul_fips<1>(b, m);
    } else if constexpr (FORM == 9) {  // latency: one dependent chain
      a = f_mul(a, m);
    } else {
      a = f_mulc_cios(a, m);
    }
  }
  // every form against the CIOS reference product on this thread's values
  Fp got;
  if constexpr (FORM == 5) got = f_mul_cios(a, b);
  else if constexpr (FORM == 6 || FORM == 10) got = f_mulc_cios(a, b);
  else if constexpr (FORM == 7 || FORM == 9) got = f_mul(a, b);
  else got = f_mul_fips<1>(a, b);
  if (got != f_mul_cios(a, b)) atomicAdd(sink + 1, 1u);
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < 8; j++) acc ^= a.v[j] ^ b.v[j];
  if (acc == 0x12345678u) sink[0] = acc;
}

}  // namespace zkvc

using namespace zkvc;

extern "C" {

const char* zkvc_last_error(void) { return g_err.c_str(); }

int zkvc_version(void) { return 100; }

int zkvc_glv_split(const uint8_t k[32], uint8_t out[34]) {
  clear_error();
  ZK_CHECK(k && out, ZKVC_EINVAL, "glv_split: null pointer");
  const GlvScalar g = glv_split(k);
  for (int h = 0; h < 2; h++) {
    for (int i = 0; i < 4; i++)
      for (int b = 0; b < 4; b++) out[17 * h + 4 * i + b] = (uint8_t)(g.h[h].mag[i] >> (8 * b));
    out[17 * h + 16] = (uint8_t)g.h[h].neg;
  }
  return ZKVC_OK;
}

uint64_t zkvc_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int zkvc_set_device_wait_limit_ns(uint64_t ns) {
  clear_error();
  set_matmul_first_wait_ns(ns);
  return ZKVC_OK;
}

int zkvc_set_wait_timeout_ms(int ms) {
  clear_error();
  ZK_CHECK(ms > 0, ZKVC_EINVAL, "wait timeout of %d ms", ms);
  g_wait_ms.store(ms);
  return ZKVC_OK;
}

void zkvc_profile_enable(int on) {
  for (auto& x : g_prof_slots) {
    x.ms = x.start_ms = x.end_ms = 0;
    x.calls = x.units = 0;
    x.pending = false;
  }
  g_prof.store(on != 0);
}

int zkvc_profile_read(int stage, const char** name, double* ms, uint64_t* calls, uint64_t* units) {
  clear_error();
  ZK_CHECK(stage >= 0 && stage < PS_COUNT, ZKVC_EINVAL, "profile: stage %d outside [0, %d)", stage, (int)PS_COUNT);
  const ProfSlot& x = g_prof_slots[stage];
  if (name) *name = x.name;
  if (ms) *ms = x.ms;
  if (calls) *calls = x.calls;
  if (units) *units = x.units;
  return ZKVC_OK;
}

int zkvc_profile_span(int stage, double* start_ms, double* end_ms) {
  clear_error();
  ZK_CHECK(stage >= 0 && stage < PS_COUNT, ZKVC_EINVAL, "profile: stage %d outside [0, %d)", stage, (int)PS_COUNT);
  const ProfSlot& x = g_prof_slots[stage];
  const double n = x.calls ? (double)x.calls : 1.0;
  if (start_ms) *start_ms = x.start_ms / n;
  if (end_ms) *end_ms = x.end_ms / n;
  return ZKVC_OK;
}

int zkvc_fr_mul(const uint8_t* d_a, const uint8_t* d_b, uint8_t* d_out, size_t n, void* stream) {
  clear_error();
  if (n == 0) return ZKVC_OK;
  ZK_CHECK(d_a && d_b && d_out, ZKVC_EINVAL, "fr_mul: null pointer");
  k_field_mul<FrCfg><<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      (const Fr*)d_a, (const Fr*)d_b, (Fr*)d_out, n); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

int zkvc_fp_mul(const uint8_t* d_a, const uint8_t* d_b, uint8_t* d_out, size_t n, void* stream) {
  clear_error();
  if (n == 0) return ZKVC_OK;
  ZK_CHECK(d_a && d_b && d_out, ZKVC_EINVAL, "fp_mul: null pointer");
  k_field_mul<FpCfg><<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      (const Fp*)d_a, (const Fp*)d_b, (Fp*)d_out, n); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

int zkvc_fr_inv(const uint8_t* d_a, uint8_t* d_out, size_t n, void* stream) {
  clear_error();
  if (n == 0) return ZKVC_OK;
  ZK_CHECK(d_a && d_out, ZKVC_EINVAL, "fr_inv: null pointer");
  k_field_inv<FrCfg><<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>((const Fr*)d_a, (Fr*)d_out, n);
  ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

int zkvc_fp_inv(const uint8_t* d_a, uint8_t* d_out, size_t n, void* stream) {
  clear_error();
  if (n == 0) return ZKVC_OK;
  ZK_CHECK(d_a && d_out, ZKVC_EINVAL, "fp_inv: null pointer");
  k_field_inv<FpCfg><<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>((const Fp*)d_a, (Fp*)d_out, n);
  ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

int zkvc_fp2_mul(const uint8_t* d_a, const uint8_t* d_b, uint8_t* d_out, size_t n, void* stream) {
  clear_error();
  if (n == 0) return ZKVC_OK;
  ZK_CHECK(d_a && d_b && d_out, ZKVC_EINVAL, "fp2_mul: null pointer");
  k_fp2_mul<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>((const Fp2*)d_a, (const Fp2*)d_b,
                                                                            (Fp2*)d_out, n); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

int zkvc_ntt(uint8_t* d_data, uint32_t log_n, int kind, void* stream) {
  clear_error();
  ZK_CHECK(d_data != nullptr, ZKVC_EINVAL, "ntt: null pointer");
  ZK_CHECK(kind >= 0 && kind <= 3, ZKVC_EINVAL, "ntt: kind %d", kind);
  const NttDomain* d = nullptr;
  ZK_TRY(ntt_domain(log_n, &d));
  cudaStream_t st = (cudaStream_t)stream;
  Fr* x = reinterpret_cast<Fr*>(d_data);
  bool inverse = kind == ZKVC_NTT_INVERSE || kind == ZKVC_NTT_COSET_INVERSE;
  int load_scale = kind == ZKVC_NTT_COSET_FORWARD ? SC_G : SC_NONE;
  int out_scale = kind == ZKVC_NTT_INVERSE ? SC_N : (kind == ZKVC_NTT_COSET_INVERSE ? SC_NGI : SC_NONE);
  ZK_TRY(ntt_dif(x, 1, 0, d, inverse, load_scale, SC_NONE, true, st));
  ZK_TRY(ntt_bitrev(x, d, out_scale, true, st));
  return ZKVC_OK;
}

int zkvc_matmul_i8(const int8_t* d_X, const int8_t* d_W, int32_t* d_Y, int a, int n, int b, void* stream) {
  clear_error();
  ZK_CHECK(d_X && d_W && d_Y, ZKVC_EINVAL, "matmul: null pointer");
  static thread_local int* t_flag = nullptr;
  static thread_local int t_dev = -1;
  int dev = 0;
  ZK_CUDA(cudaGetDevice(&dev));
  if (!t_flag || t_dev != dev) {
    ZK_CUDA(cudaMalloc(&t_flag, sizeof(int)));
    t_dev = dev;
  }
  cudaStream_t st = (cudaStream_t)stream;
  ZK_CUDA(cudaMemsetAsync(t_flag, 0, sizeof(int), st));
  ZK_TRY(matmul_i8(d_X, d_W, d_Y, a, n, b, t_flag, st));
  int h = 0;
  ZK_CUDA(cudaMemcpyAsync(&h, t_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  ZK_TRY(wait_stream(st, "matmul"));
  ZK_CHECK(!(h & 8), ZKVC_ETIMEOUT, "matmul: a tensor-core wait timed out");
  return ZKVC_OK;
}

size_t zkvc_msm_workspace_bytes(size_t n, int group) {
  if (n == 0) return 0;
  return group == 2 ? msm_api_ws<Fp2>(n) : msm_api_ws<Fp>(n);
}

int zkvc_msm_g1(const uint8_t* d_points, const uint8_t* d_scalars, size_t n, void* d_ws, size_t ws_bytes,
                uint8_t out[64], void* stream) {
  clear_error();
  return msm_api<Fp>(d_points, d_scalars, n, d_ws, ws_bytes, out, (cudaStream_t)stream);
}

int zkvc_msm_g2(const uint8_t* d_points, const uint8_t* d_scalars, size_t n, void* d_ws, size_t ws_bytes,
                uint8_t out[128], void* stream) {
  clear_error();
  return msm_api<Fp2>(d_points, d_scalars, n, d_ws, ws_bytes, out, (cudaStream_t)stream);
}

int zkvc_imad_rate(int form, uint32_t iters, double* imad_per_s, double* ms, int* sms, void* stream) {
  clear_error();
  ZK_CHECK(form >= 0 && form <= 10, ZKVC_EINVAL, "imad_rate: form %d", form);
  ZK_CHECK(iters >= 1 && iters <= (1u << 24), ZKVC_EINVAL, "imad_rate: %u iterations outside [1, 2^24]", iters);
  static thread_local uint32_t* t_sink = nullptr;
  static thread_local int t_dev = -1;
  int dev = 0;
  ZK_CUDA(cudaGetDevice(&dev));
  if (!t_sink || t_dev != dev) {
    ZK_CUDA(cudaMalloc(&t_sink, 2 * sizeof(uint32_t)));
    t_dev = dev;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int per_sm = 0;
  auto kern = form == 0 ? k_imad_rate<0> : form == 1 ? k_imad_rate<1> : form == 2 ? k_imad_rate<2>
              : form == 3 ? k_imad_rate<3> : form == 4 ? k_imad_rate<4> : form == 5 ? k_mont_rate<5>
              : form == 6 ? k_mont_rate<6> : form == 7 ? k_mont_rate<7> : form == 8 ? k_mont_rate<8>
              : form == 9 ? k_mont_rate<9> : k_mont_rate<10>;
  ZK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0));
  const int nsm = device_sm_count();
  const bool latency = form >= 9;  // one warp, one dependent chain per thread
  const unsigned blocks = latency ? 1u : (unsigned)(nsm * (per_sm > 0 ? per_sm : 1));
  const unsigned threads = latency ? 32u : 256u;
  cudaEvent_t e0, e1;
  ZK_CUDA(cudaEventCreate(&e0));
  ZK_CUDA(cudaEventCreate(&e1));
  ZK_CUDA(cudaMemsetAsync(t_sink, 0, 2 * sizeof(uint32_t), st));
  kern<<<blocks, threads, 0, st>>>(iters / 8 + 1, 7u, t_sink); ZK_COUNT_LAUNCH();  // warm
  ZK_CUDA(cudaEventRecord(e0, st));
  kern<<<blocks, threads, 0, st>>>(iters, 7u, t_sink); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaEventRecord(e1, st));
  ZK_CUDA(cudaGetLastError());
  ZK_TRY(wait_stream(st, "imad_rate"));
  float t = 0;
  ZK_CUDA(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  uint32_t bad = 0;
  ZK_CUDA(cudaMemcpy(&bad, t_sink + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  ZK_CHECK(bad == 0, ZKVC_ECUDA, "imad_rate: form %d products differ from the reference product in %u threads",
           form, bad);
  const double per_iter = latency ? 264.0 : form >= 5 ? 2.0 * 264.0 : 16.0;
  const double ops = double(blocks) * double(threads) * double(iters) * per_iter;
  if (ms) *ms = t;
  if (imad_per_s) *imad_per_s = t > 0 ? ops / (t * 1e-3) : 0.0;
  if (sms) *sms = nsm;
  return ZKVC_OK;
}

}  // extern "C"
