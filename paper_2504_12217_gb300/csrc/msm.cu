// Pippenger multi-scalar multiplication (the A, B, L and H queries of the Groth16
// prover, zkVC Sec. II / IV; the MSMs dominate proving time).
//
// Scalars are recoded into signed c-bit digits d in (-2^(c-1), 2^(c-1)], so a digit
// selects bucket |d| and the sign negates the base's y coordinate.  Every nonzero digit
// becomes one term (bucket key, base index | sign).  Terms are counting-sorted by key
// (histogram, scan, atomic scatter), then each bucket's terms are summed by a
// load-balanced segmented reduction: level 0 gives every chunk of T0 consecutive terms
// of a bucket to one thread (mixed XYZZ + affine additions), and binary in-place folds
// then add each bucket's partial sums, so heavily skewed buckets (int8 scalars put ~1300
// terms in each of 128 buckets) cost only log2 of their chunk count in depth.
// A window's result sum_v v B_v is evaluated as sum_b 2^b U_b with U_b the sum of the
// buckets whose index has bit b set: wide trees for the U_b, b doublings per bit in
// parallel, and a short tree over the bits -- log-depth instead of a running sum, since a
// single thread's point addition is long-latency (~14 us) on the GPU.
//
// Fixed-base MSMs (proving-key queries) store the multiples 2^(c w) P of each base, so all
// windows share one bucket set and no doubling chain follows; variable-base MSMs keep
// one bucket set per window and combine windows by Horner's rule.
#include <algorithm>

#include "msm.h"

namespace zkvc {

static constexpr uint32_t KEY_NONE = 0xffffffffu;

// ------------------------------------------------------------------ scan
__global__ void k_scan_blocks(const uint32_t* in, size_t n_in, uint32_t* out, size_t n_out, uint32_t* sums) {
  __shared__ uint32_t wsum[32];
  size_t i = size_t(blockIdx.x) * 1024 + threadIdx.x;
  uint32_t v = (i < n_in) ? in[i] : 0u;
  uint32_t x = v;
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= (uint32_t)d) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = wsum[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= (uint32_t)d) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  uint32_t incl = x + (wid ? wsum[wid - 1] : 0u);
  if (i < n_out) out[i] = incl - v;
  if (sums && threadIdx.x == 1023) sums[blockIdx.x] = incl;
}

__global__ void k_scan_add(uint32_t* out, size_t n_out, const uint32_t* add) {
  size_t i = size_t(blockIdx.x) * 1024 + threadIdx.x;
  if (i < n_out) out[i] += add[blockIdx.x];
}

static int scan_rec(const uint32_t* in, size_t n_in, uint32_t* out, size_t n_out, Arena& a, cudaStream_t st) {
  size_t blocks = (n_out + 1023) / 1024;
  if (blocks <= 1) {
    if (!a.measuring) {
      k_scan_blocks<<<1, 1024, 0, st>>>(in, n_in, out, n_out, nullptr); ZK_COUNT_LAUNCH();
      ZK_CUDA(cudaGetLastError());
    }
    return ZKVC_OK;
  }
  uint32_t* sums = a.take<uint32_t>(blocks);
  uint32_t* sums_x = a.take<uint32_t>(blocks);
  ZK_CHECK(!a.overflow(), ZKVC_EINVAL, "scan: workspace too small");
  if (!a.measuring) {
    k_scan_blocks<<<(unsigned)blocks, 1024, 0, st>>>(in, n_in, out, n_out, sums); ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaGetLastError());
  }
  ZK_TRY(scan_rec(sums, blocks, sums_x, blocks, a, st));
  if (!a.measuring) {
    k_scan_add<<<(unsigned)blocks, 1024, 0, st>>>(out, n_out, sums_x); ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaGetLastError());
  }
  return ZKVC_OK;
}

int scan_u32(const uint32_t* in, uint32_t* out, size_t n, Arena& a, cudaStream_t st) {
  return scan_rec(in, n, out, n + 1, a, st);
}

size_t scan_u32_temp_bytes(size_t n) {
  Arena a;
  a.measuring = true;
  scan_rec(nullptr, n, nullptr, n + 1, a, 0);
  return a.off;
}

// ------------------------------------------------------------------ planning
int msm_plan_finalize(MsmPlan& p) {
  uint32_t key = 0;
  for (auto& o : p.outs) {
    ZK_CHECK(o.c >= 2 && o.c <= 20, ZKVC_EINVAL, "msm: window of %u bits", o.c);
    ZK_CHECK(o.win_keys >= 1, ZKVC_EINVAL, "msm: win_keys = 0");
    o.key_off = key;
    o.nkeys = o.win_keys << (o.c - 1);
    key += o.nkeys;
  }
  p.keys = key;
  uint64_t slot = 0;
  uint32_t pts = 0;
  p.max_nd = 0;
  for (auto& s : p.segs) {
    ZK_CHECK(s.out < p.outs.size(), ZKVC_EINVAL, "msm: segment output %u", s.out);
    const MsmOut& o = p.outs[s.out];
    uint32_t nd;
    switch (s.kind) {
      case SK_ONE: nd = 1; break;
      case SK_I8: nd = (8 + o.c) / o.c; break;            // |v| <= 128 needs c (nd) > 8
      case SK_I32: nd = (32 + o.c - 1) / o.c; break;
      case SK_I16: nd = o.c >= 16 ? 1 : (16 + o.c) / o.c; break;  // |v| <= 2^15 needs c (nd) > 16
      case SK_FR_MONT:
      case SK_FR_CANON: nd = (255 + o.c - 1) / o.c; break;
      default: ZK_CHECK(false, ZKVC_EINVAL, "msm: scalar kind %d", s.kind);
    }
    if (s.kind == SK_I8 && o.c >= 8) nd = 1;
    if (o.win_keys > 1) {
      ZK_CHECK(s.nwin >= 1 && nd <= o.win_keys, ZKVC_EINVAL, "msm: %u digits for %u key windows", nd, o.win_keys);
    } else {
      ZK_CHECK(s.nwin >= nd, ZKVC_EINVAL, "msm: %u digits but %u stored windows", nd, s.nwin);
    }
    ZK_CHECK(s.base_off + uint64_t(s.count) * s.nwin <= 0x80000000ull, ZKVC_EINVAL, "msm: base index overflow");
    s.nd = nd;
    s.slot_off = slot;
    s.point_off = pts;
    slot += uint64_t(s.count) * nd;
    pts += s.count;
    p.max_nd = std::max(p.max_nd, nd);
  }
  ZK_CHECK(slot < 0xffffffffull, ZKVC_EINVAL, "msm: too many digit slots");
  p.chunk = p.tune.chunk ? p.tune.chunk : (slot < (2u << 20) ? 16u : 32u);
  ZK_CHECK(p.chunk >= 1 && p.chunk <= 1024, ZKVC_EINVAL, "msm: chunk of %u terms", p.chunk);
  ZK_CHECK(p.tune.accum_threads >= 32 && p.tune.accum_threads <= 256 && p.tune.accum_threads % 32 == 0,
           ZKVC_EINVAL, "msm: %u accumulation threads", p.tune.accum_threads);
  ZK_CHECK(p.tune.fold_blocks >= 1, ZKVC_EINVAL, "msm: fold grid of 0 blocks");
  p.slots = slot;
  p.points = pts;
  // outputs with their own base arrays: every output must name one, and all must have
  // the same power-of-two key count, so that a key's output is key >> key_shift
  p.key_shift = -1;
  bool any = false, all = true;
  for (const auto& o : p.outs) {
    if (o.bases) any = true; else all = false;
  }
  if (any) {
    ZK_CHECK(all, ZKVC_EINVAL, "msm: some outputs name a base array and some do not");
    const uint32_t nk = p.outs[0].nkeys;
    ZK_CHECK((nk & (nk - 1)) == 0, ZKVC_EINVAL, "msm: %u keys per output is not a power of two", nk);
    for (const auto& o : p.outs) ZK_CHECK(o.nkeys == nk, ZKVC_EINVAL, "msm: unequal key counts across outputs");
    int sh = 0;
    while ((1u << sh) < nk) sh++;
    p.key_shift = sh;
  }
  return ZKVC_OK;
}

// ------------------------------------------------------------------ digits
__device__ __forceinline__ uint32_t bits_at(const uint32_t (&m)[8], uint32_t pos, uint32_t c) {
  uint32_t w = pos >> 5, sh = pos & 31;
  uint64_t x = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    if ((uint32_t)i == w) x |= m[i];
    if ((uint32_t)i == w + 1) x |= (uint64_t)m[i] << 32;
  }
  return (uint32_t)(x >> sh) & ((1u << c) - 1u);
}

__global__ void k_digits(const MsmSeg* __restrict__ segs, int nsegs, const MsmOut* __restrict__ outs,
                         uint32_t total_points, uint32_t* keys, uint32_t* vals) {
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total_points) return;
  int lo = 0, hi = nsegs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (segs[mid].point_off <= t) lo = mid; else hi = mid - 1;
  }
  const MsmSeg sg = segs[lo];
  const uint32_t i = t - sg.point_off;
  const MsmOut o = outs[sg.out];
  uint32_t m[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  bool neg = false;
  if (i != sg.skip) {
    switch (sg.kind) {
      case SK_ONE: m[0] = 1; break;
      case SK_I8: {
        int v = reinterpret_cast<const int8_t*>(sg.scalars)[i];
        neg = v < 0;
        m[0] = (uint32_t)(v < 0 ? -v : v);
        break;
      }
      case SK_I16: {
        int v = reinterpret_cast<const int16_t*>(sg.scalars)[i];
        neg = v < 0;
        m[0] = (uint32_t)(v < 0 ? -v : v);
        break;
      }
      case SK_I32: {
        int32_t v = reinterpret_cast<const int32_t*>(sg.scalars)[i];
        neg = v < 0;
        m[0] = v < 0 ? (uint32_t)(-(int64_t)v) : (uint32_t)v;
        break;
      }
      case SK_FR_MONT: {
        Fr x = f_from_mont(ld_field(reinterpret_cast<const Fr*>(sg.scalars) + i));
#pragma unroll
        for (int l = 0; l < 8; l++) m[l] = x.v[l];
        break;
      }
      default: {
        Fr x = ld_field(reinterpret_cast<const Fr*>(sg.scalars) + i);
#pragma unroll
        for (int l = 0; l < 8; l++) m[l] = x.v[l];
        break;
      }
    }
  }
  const uint32_t c = o.c, half = 1u << (c - 1), NB = half;
  uint32_t carry = 0;
  for (uint32_t w = 0; w < sg.nd; w++) {
    uint32_t raw = bits_at(m, w * c, c) + carry;
    int32_t d;
    if (raw > half) {
      d = (int32_t)raw - (int32_t)(1u << c);
      carry = 1;
    } else {
      d = (int32_t)raw;
      carry = 0;
    }
    uint64_t slot = sg.slot_off + uint64_t(i) * sg.nd + w;
    if (d == 0) {
      keys[slot] = KEY_NONE;
      continue;
    }
    uint32_t mag = (uint32_t)(d < 0 ? -d : d);
    uint32_t sign = ((d < 0) != neg) ? 1u : 0u;
    uint32_t key = o.key_off + (o.win_keys > 1 ? w * NB : 0u) + mag - 1;
    uint64_t base = sg.base_off + uint64_t(i) * sg.nwin + (o.win_keys > 1 ? 0u : w);
    keys[slot] = key;
    vals[slot] = (uint32_t)base | (sign << 31);
  }
}

// Counting sort by key.  A block takes a tile of HB_TILE consecutive slots and counts
// the keys in a window of HB_BINS keys starting at the tile's smallest key in shared
// memory, so a bucket that many terms share (small-scalar runs put thousands of terms in
// each of 128 buckets) costs one global atomic per block instead of one per term; keys
// outside the window fall back to global atomics.  The scatter repeats the count,
// reserves each bin's range with one global atomic, and places the tile's terms with
// shared-memory atomics.  (Positions inside a bucket are in no fixed order; bucket sums
// do not depend on it.)
constexpr int HB_THREADS = 256, HB_PER = 8, HB_TILE = HB_THREADS * HB_PER, HB_BINS = 2048;

__device__ __forceinline__ uint32_t tile_min_key(const uint32_t (&k)[HB_PER], uint32_t* kmin_s) {
  uint32_t m = KEY_NONE;
#pragma unroll
  for (int j = 0; j < HB_PER; j++) m = min(m, k[j]);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, d));
  if ((threadIdx.x & 31) == 0) atomicMin(kmin_s, m);
  __syncthreads();
  return *kmin_s;
}

__global__ void __launch_bounds__(HB_THREADS) k_hist(const uint32_t* __restrict__ keys, uint64_t n, uint32_t* counts) {
  __shared__ uint32_t hist[HB_BINS];
  __shared__ uint32_t kmin_s;
  const uint64_t base = uint64_t(blockIdx.x) * HB_TILE;
  uint32_t k[HB_PER];
#pragma unroll
  for (int j = 0; j < HB_PER; j++) {
    uint64_t i = base + uint64_t(j) * HB_THREADS + threadIdx.x;
    k[j] = i < n ? keys[i] : KEY_NONE;
  }
  for (int b = threadIdx.x; b < HB_BINS; b += HB_THREADS) hist[b] = 0;
  if (threadIdx.x == 0) kmin_s = KEY_NONE;
  __syncthreads();
  const uint32_t k0 = tile_min_key(k, &kmin_s);
  if (k0 == KEY_NONE) return;  // uniform: the whole tile is empty
#pragma unroll
  for (int j = 0; j < HB_PER; j++) {
    if (k[j] == KEY_NONE) continue;
    uint32_t d = k[j] - k0;
    if (d < (uint32_t)HB_BINS)
      atomicAdd(&hist[d], 1u);
    else
      atomicAdd(counts + k[j], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < HB_BINS; b += HB_THREADS) {
    uint32_t c = hist[b];
    if (c) atomicAdd(counts + k0 + b, c);
  }
}

__global__ void __launch_bounds__(HB_THREADS) k_scatter(const uint32_t* __restrict__ keys,
                                                        const uint32_t* __restrict__ vals, uint64_t n,
                                                        uint32_t* cursor, uint32_t* sorted) {
  __shared__ uint32_t hist[HB_BINS];
  __shared__ uint32_t start[HB_BINS];
  __shared__ uint32_t kmin_s;
  const uint64_t base = uint64_t(blockIdx.x) * HB_TILE;
  uint32_t k[HB_PER];
#pragma unroll
  for (int j = 0; j < HB_PER; j++) {
    uint64_t i = base + uint64_t(j) * HB_THREADS + threadIdx.x;
    k[j] = i < n ? keys[i] : KEY_NONE;
  }
  for (int b = threadIdx.x; b < HB_BINS; b += HB_THREADS) hist[b] = 0;
  if (threadIdx.x == 0) kmin_s = KEY_NONE;
  __syncthreads();
  const uint32_t k0 = tile_min_key(k, &kmin_s);
  if (k0 == KEY_NONE) return;
#pragma unroll
  for (int j = 0; j < HB_PER; j++) {
    if (k[j] == KEY_NONE) continue;
    uint32_t d = k[j] - k0;
    if (d < (uint32_t)HB_BINS) atomicAdd(&hist[d], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < HB_BINS; b += HB_THREADS) {
    uint32_t c = hist[b];
    if (c) start[b] = atomicAdd(cursor + k0 + b, c);
    hist[b] = 0;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < HB_PER; j++) {
    if (k[j] == KEY_NONE) continue;
    uint64_t i = base + uint64_t(j) * HB_THREADS + threadIdx.x;
    uint32_t d = k[j] - k0;
    uint32_t pos = d < (uint32_t)HB_BINS ? start[d] + atomicAdd(&hist[d], 1u) : atomicAdd(cursor + k[j], 1u);
    sorted[pos] = vals[i];
  }
}

__global__ void k_chunks(const uint32_t* counts, uint32_t K, uint32_t T0, uint32_t* nch) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < K) nch[k] = (counts[k] + T0 - 1) / T0;
}

// largest k in [0, K) with off[k] <= q
__device__ __forceinline__ uint32_t find_key(const uint32_t* off, uint32_t K, uint32_t q) {
  uint32_t lo = 0, hi = K - 1;
  while (lo < hi) {
    uint32_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= q) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------ bucket sums
__global__ void k_chunk_keys(const uint32_t* __restrict__ choff, uint32_t K, uint32_t* chunk_key, uint32_t* max_chunks) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  uint32_t a = choff[k], b = choff[k + 1];
  for (uint32_t q = a; q < b; q++) chunk_key[q] = k;
  if (b > a + 1) atomicMax(max_chunks, b - a);
}

// level 0: chunk q sums up to T0 consecutive terms of its bucket (mixed additions)
template <class F>
__global__ void __launch_bounds__(256) k_accum0(const uint32_t* __restrict__ sorted, const uint32_t* __restrict__ offs,
                                                const uint32_t* __restrict__ choff, const uint32_t* __restrict__ chunk_key,
                                                uint32_t K, uint32_t T0, const Affine<F>* __restrict__ bases,
                                                const Affine<F>* const* __restrict__ obases, int key_shift,
                                                XYZZ<F>* part) {
  uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= choff[K]) return;
  uint32_t k = chunk_key[q];
  uint32_t j = q - choff[k];
  uint32_t start = offs[k] + j * T0;
  uint32_t end = min(start + T0, offs[k + 1]);
  if (key_shift >= 0) bases = obases[k >> key_shift];
  XYZZ<F> acc = XYZZ<F>::inf();
  for (uint32_t p = start; p < end; p++) {
    uint32_t v = sorted[p];
    Affine<F> P = ld_field(bases + (v & 0x7fffffffu));
    if (v >> 31) P.y = f_neg(P.y);
    acc = p_add_affine(acc, P);
  }
  st_field(part + q, acc);
}

// binary fold of the partial sums of each bucket, in place: at level l the partial at
// local index i (a multiple of 2^(l+1)) absorbs the one at i + 2^l.  Levels at or above
// log2 of the largest chunk count exit at once (the count is only known on the device).
// (A block-per-heavy-bucket variant measured slower on GB300: barrier stalls while one
// warp finishes each block's tree.)
template <class F>
__global__ void __launch_bounds__(256) k_fold(XYZZ<F>* part, const uint32_t* __restrict__ choff,
                                              const uint32_t* __restrict__ chunk_key, uint32_t K,
                                              const uint32_t* __restrict__ max_chunks, uint32_t l) {
  const uint32_t step = 1u << l;
  if (step >= *max_chunks) return;
  const uint32_t total = choff[K];
  // grid-stride over the chunk slots (the grid is small, so levels above the largest
  // chunk count cost little more than the launch)
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    uint32_t k = chunk_key[q];
    uint32_t base = choff[k], i = q - base, np = choff[k + 1] - base;
    if ((i & (2 * step - 1)) != 0 || i + step >= np) continue;
    st_field(part + q, p_add(ld_field(part + q), ld_field(part + q + step)));
  }
}

template <class F>
__device__ __forceinline__ XYZZ<F> bucket_at(const XYZZ<F>* fin, const uint32_t* counts, const uint32_t* choff,
                                             uint32_t key) {
  if (counts[key] == 0) return XYZZ<F>::inf();
  return ld_field(fin + choff[key]);
}

// Window result sum_{v=1}^{NB} v B_v = sum_b 2^b U_b with U_b = sum_{v : bit b of v} B_v.
// One BitSeg per (output, window, bit): the U_b sum starts as pairs of buckets and is
// finished by strided tree levels; then 2^b U_b (b doublings, all bits in parallel) and a
// tree over the bits of each (output, window).
struct BitSeg {
  uint32_t key0;  // key of bucket v = 1 of this (output, window)
  uint32_t b, c;  // bit, window bits
  uint32_t uoff;  // first pair in the U buffer
  uint32_t dslot; // slot of 2^b U_b in the D buffer
};

__device__ __forceinline__ uint32_t nth_with_bit(uint32_t b, uint32_t c, uint32_t idx) {
  if (b == c - 1) return 1u << (c - 1);
  return ((idx >> b) << (b + 1)) | (1u << b) | (idx & ((1u << b) - 1u));
}

template <class F>
__global__ void __launch_bounds__(256) k_bits_first(const XYZZ<F>* __restrict__ fin, const uint32_t* __restrict__ counts,
                                                    const uint32_t* __restrict__ choff, const BitSeg* __restrict__ segs,
                                                    uint32_t nseg, uint32_t total, XYZZ<F>* U) {
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  uint32_t lo = 0, hi = nseg - 1;
  while (lo < hi) {
    uint32_t mid = (lo + hi + 1) >> 1;
    if (segs[mid].uoff <= t) lo = mid; else hi = mid - 1;
  }
  const BitSeg s = segs[lo];
  const uint32_t j = t - s.uoff;
  const uint32_t cnt = (s.b == s.c - 1) ? 1u : (1u << (s.c - 2));
  XYZZ<F> acc = bucket_at(fin, counts, choff, s.key0 + nth_with_bit(s.b, s.c, 2 * j) - 1);
  if (2 * j + 1 < cnt) acc = p_add(acc, bucket_at(fin, counts, choff, s.key0 + nth_with_bit(s.b, s.c, 2 * j + 1) - 1));
  st_field(U + t, acc);
}

template <class F>
__global__ void __launch_bounds__(64) k_bits_scale(const XYZZ<F>* __restrict__ U, const BitSeg* __restrict__ segs,
                                                   uint32_t nseg, XYZZ<F>* D) {
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nseg) return;
  BitSeg s = segs[t];
  XYZZ<F> x = ld_field(U + s.uoff);
  for (uint32_t i = 0; i < s.b; i++) x = p_dbl(x);
  st_field(D + s.dslot, x);
}

// In-place tree over segments: at level l, element i*2^(l+1) absorbs element
// i*2^(l+1) + 2^l of the same segment.  Threads map only to pairs that exist at this
// level (cum[s] counts the pairs of the segments before s), so no lane is idle.
struct TreeSeg {
  uint32_t off;  // first element
  uint32_t len;  // elements
};

template <class F>
__global__ void __launch_bounds__(256) k_tree_level(XYZZ<F>* x, const TreeSeg* __restrict__ segs,
                                                    const uint32_t* __restrict__ cum, uint32_t nseg, uint32_t total,
                                                    uint32_t l) {
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  uint32_t lo = 0, hi = nseg - 1;
  while (lo < hi) {
    uint32_t mid = (lo + hi + 1) >> 1;
    if (cum[mid] <= t) lo = mid; else hi = mid - 1;
  }
  TreeSeg s = segs[lo];
  uint32_t i = t - cum[lo];
  uint64_t a = s.off + (uint64_t(i) << (l + 1)), b = a + (1ull << l);
  st_field(x + a, p_add(ld_field(x + a), ld_field(x + b)));
}

// host-side per-level pair counts of a tree over segments
struct TreePlan {
  std::vector<TreeSeg> segs;
  std::vector<uint32_t> cum;     // levels x nseg
  std::vector<uint32_t> totals;  // per level
  uint32_t levels = 0;
  void finish() {
    uint32_t maxlen = 1;
    for (auto& s : segs) maxlen = std::max(maxlen, s.len);
    levels = 0;
    while ((1u << levels) < maxlen) levels++;
    cum.assign(size_t(levels) * segs.size(), 0);
    totals.assign(levels, 0);
    for (uint32_t l = 0; l < levels; l++) {
      uint32_t acc = 0, step = 1u << l;
      for (size_t s = 0; s < segs.size(); s++) {
        cum[size_t(l) * segs.size() + s] = acc;
        uint32_t len = segs[s].len;
        acc += len > step ? (len - step + 2 * step - 1) / (2 * step) : 0;
      }
      totals[l] = acc;
    }
  }
};

// results[o] = sum_w 2^(c w) W[o][w] by Horner's rule (windows of variable-base outputs).
struct OutItem {
  uint32_t first;     // index of window 0's result in D
  uint32_t stride;    // distance between windows' results
  uint32_t nwin;
  uint32_t c;
};

template <class F>
__global__ void k_combine_windows(const XYZZ<F>* D, const OutItem* outs, uint32_t nouts, XYZZ<F>* results) {
  uint32_t o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nouts) return;
  OutItem it = outs[o];
  XYZZ<F> acc = ld_field(D + it.first + (it.nwin - 1) * it.stride);
  for (int w = (int)it.nwin - 2; w >= 0; w--) {
    for (uint32_t i = 0; i < it.c; i++) acc = p_dbl(acc);
    acc = p_add(acc, ld_field(D + it.first + uint32_t(w) * it.stride));
  }
  st_field(results + o, acc);
}

// ------------------------------------------------------------------ driver
struct Layout {
  uint32_t *keys, *vals, *sorted, *counts, *offs, *cursor, *nch, *choff, *chunk_key, *max_chunks;
  void *part, *U, *D;
  MsmSeg* segs;
  MsmOut* outs;
  const void** obases;
  BitSeg* bsegs;
  TreeSeg *useg, *dseg;
  uint32_t *ucum, *dcum;
  OutItem* oitems;
  uint32_t qmax, nbits, utotal, dtotal;
};

struct HostTables {
  std::vector<BitSeg> bsegs;
  TreePlan ut, dt;
  std::vector<OutItem> oitems;
  std::vector<const void*> obases;
};

struct MsmExecState {
  Layout L;
  HostTables h;
  Arena after_layout;  // the arena once the tables are carved: scans take from a copy
  bool uploaded = false;
};

MsmExec::~MsmExec() { delete st; }

static void tables(const MsmPlan& p, HostTables& h, Layout& L) {
  h.bsegs.clear();
  h.ut = TreePlan();
  h.dt = TreePlan();
  h.oitems.clear();
  h.obases.clear();
  uint32_t uoff = 0, dslot = 0;
  for (const auto& o : p.outs) {
    const uint32_t nb = 1u << (o.c - 1);
    h.oitems.push_back({dslot, o.c, o.win_keys, o.c});
    h.obases.push_back(o.bases);
    for (uint32_t w = 0; w < o.win_keys; w++) {
      h.dt.segs.push_back({dslot, o.c});
      for (uint32_t b = 0; b < o.c; b++) {
        uint32_t cnt = (b == o.c - 1) ? 1u : (1u << (o.c - 2));
        uint32_t pairs = (cnt + 1) / 2;
        h.bsegs.push_back({o.key_off + w * nb, b, o.c, uoff, dslot + b});
        h.ut.segs.push_back({uoff, pairs});
        uoff += pairs;
      }
      dslot += o.c;
    }
  }
  h.ut.finish();
  h.dt.finish();
  L.nbits = (uint32_t)h.bsegs.size();
  L.utotal = uoff;
  L.dtotal = dslot;
}

template <class F>
static void layout(const MsmPlan& p, Arena& a, Layout& L, HostTables& h) {
  const size_t S = p.slots, K = p.keys;
  const uint32_t T0 = p.chunk ? p.chunk : 32;
  L.keys = a.take<uint32_t>(S);
  L.vals = a.take<uint32_t>(S);
  L.sorted = a.take<uint32_t>(S);
  L.counts = a.take<uint32_t>(K);
  L.offs = a.take<uint32_t>(K + 1);
  L.cursor = a.take<uint32_t>(K);
  L.nch = a.take<uint32_t>(K);
  L.choff = a.take<uint32_t>(K + 1);
  L.qmax = (uint32_t)(S / T0 + K + 1);
  L.chunk_key = a.take<uint32_t>(L.qmax);
  L.max_chunks = a.take<uint32_t>(1);
  L.part = a.take<XYZZ<F>>(L.qmax);
  tables(p, h, L);
  L.U = a.take<XYZZ<F>>(L.utotal);
  L.D = a.take<XYZZ<F>>(L.dtotal);
  L.segs = a.take<MsmSeg>(p.segs.size());
  L.outs = a.take<MsmOut>(p.outs.size());
  L.obases = a.take<const void*>(p.outs.size());
  L.bsegs = a.take<BitSeg>(h.bsegs.size());
  L.useg = a.take<TreeSeg>(h.ut.segs.size());
  L.ucum = a.take<uint32_t>(std::max<size_t>(1, h.ut.cum.size()));
  L.dseg = a.take<TreeSeg>(h.dt.segs.size());
  L.dcum = a.take<uint32_t>(std::max<size_t>(1, h.dt.cum.size()));
  L.oitems = a.take<OutItem>(h.oitems.size());
}

template <class F>
size_t msm_workspace_bytes(const MsmPlan& p) {
  Arena a;
  a.measuring = true;
  Layout L;
  HostTables h;
  layout<F>(p, a, L, h);
  a.off += scan_u32_temp_bytes(p.keys) + scan_u32_temp_bytes(p.keys) + 256;
  return a.off;
}

template <class F>
static int run_tree(XYZZ<F>* x, const TreePlan& t, const TreeSeg* dsegs, const uint32_t* dcum, cudaStream_t st) {
  const uint32_t nseg = (uint32_t)t.segs.size();
  for (uint32_t l = 0; l < t.levels; l++) {
    uint32_t total = t.totals[l];
    if (total == 0) continue;
    k_tree_level<F><<<(total + 255) / 256, 256, 0, st>>>(x, dsegs, dcum + size_t(l) * nseg, nseg, total, l); ZK_COUNT_LAUNCH();
  }
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

template <class F>
int msm_prepare(const MsmPlan& p, void* ws, size_t ws_bytes, MsmExec* ex) {
  ZK_CHECK(p.keys > 0 && !p.outs.empty(), ZKVC_EINVAL, "msm: empty plan");
  ZK_CHECK(ex, ZKVC_EINVAL, "msm: null exec");
  delete ex->st;
  ex->st = new MsmExecState();
  ex->plan = p;
  Arena a;
  a.base = reinterpret_cast<uint8_t*>(ws);
  a.cap = ws_bytes;
  layout<F>(ex->plan, a, ex->st->L, ex->st->h);
  ZK_CHECK(!a.overflow(), ZKVC_EINVAL, "msm: workspace of %zu bytes is too small", ws_bytes);
  ex->st->after_layout = a;
  return ZKVC_OK;
}

int msm_upload(MsmExec* ex, cudaStream_t st) {
  ZK_CHECK(ex && ex->st, ZKVC_EINVAL, "msm: exec not prepared");
  const MsmPlan& p = ex->plan;
  Layout& L = ex->st->L;
  HostTables& h = ex->st->h;
  ZK_CUDA(cudaMemcpyAsync(L.segs, p.segs.data(), p.segs.size() * sizeof(MsmSeg), cudaMemcpyHostToDevice, st));
  ZK_CUDA(cudaMemcpyAsync(L.outs, p.outs.data(), p.outs.size() * sizeof(MsmOut), cudaMemcpyHostToDevice, st));
  ZK_CUDA(cudaMemcpyAsync(L.obases, h.obases.data(), h.obases.size() * sizeof(void*), cudaMemcpyHostToDevice, st));
  ZK_CUDA(cudaMemcpyAsync(L.bsegs, h.bsegs.data(), h.bsegs.size() * sizeof(BitSeg), cudaMemcpyHostToDevice, st));
  ZK_CUDA(cudaMemcpyAsync(L.useg, h.ut.segs.data(), h.ut.segs.size() * sizeof(TreeSeg), cudaMemcpyHostToDevice, st));
  if (!h.ut.cum.empty())
    ZK_CUDA(cudaMemcpyAsync(L.ucum, h.ut.cum.data(), h.ut.cum.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
  ZK_CUDA(cudaMemcpyAsync(L.dseg, h.dt.segs.data(), h.dt.segs.size() * sizeof(TreeSeg), cudaMemcpyHostToDevice, st));
  if (!h.dt.cum.empty())
    ZK_CUDA(cudaMemcpyAsync(L.dcum, h.dt.cum.data(), h.dt.cum.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
  ZK_CUDA(cudaMemcpyAsync(L.oitems, h.oitems.data(), h.oitems.size() * sizeof(OutItem), cudaMemcpyHostToDevice, st));
  ex->st->uploaded = true;
  return ZKVC_OK;
}

template <class F>
int msm_launch(const MsmExec* ex, const Affine<F>* bases, XYZZ<F>* results, cudaStream_t st, int accum_stage) {
  ZK_CHECK(ex && ex->st && ex->st->uploaded, ZKVC_EINVAL, "msm: exec not uploaded");
  const MsmPlan& p = ex->plan;
  const Layout& L = ex->st->L;
  const HostTables& h = ex->st->h;
  Arena a = ex->st->after_layout;
  const uint32_t K = p.keys;
  const uint64_t S = p.slots;
  const uint32_t T0 = p.chunk;
  ZK_CHECK(T0 >= 1, ZKVC_EINVAL, "msm: plan not finalized");
  ZK_CHECK(p.key_shift >= 0 || bases, ZKVC_EINVAL, "msm: no base array");

  // digits -> terms
  if (p.points > 0) {
    k_digits<<<(p.points + 255) / 256, 256, 0, st>>>(L.segs, (int)p.segs.size(), L.outs, p.points, L.keys, L.vals); ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaGetLastError());
  }
  // counting sort by bucket key
  ZK_CUDA(cudaMemsetAsync(L.counts, 0, size_t(K) * sizeof(uint32_t), st));
  ZK_CUDA(cudaMemsetAsync(L.max_chunks, 0, sizeof(uint32_t), st));
  unsigned sb = (unsigned)((S + HB_TILE - 1) / HB_TILE);
  if (S > 0) {
    k_hist<<<sb, HB_THREADS, 0, st>>>(L.keys, S, L.counts); ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaGetLastError());
  }
  ZK_TRY(scan_u32(L.counts, L.offs, K, a, st));
  ZK_CUDA(cudaMemcpyAsync(L.cursor, L.offs, size_t(K) * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
  if (S > 0) {
    k_scatter<<<sb, HB_THREADS, 0, st>>>(L.keys, L.vals, S, L.cursor, L.sorted); ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaGetLastError());
  }
  // chunks of T0 terms per bucket
  k_chunks<<<(K + 255) / 256, 256, 0, st>>>(L.counts, K, T0, L.nch); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  ZK_TRY(scan_u32(L.nch, L.choff, K, a, st));
  ZK_CHECK(!a.overflow(), ZKVC_EINVAL, "msm: workspace too small for scans");
  k_chunk_keys<<<(K + 255) / 256, 256, 0, st>>>(L.choff, K, L.chunk_key, L.max_chunks); ZK_COUNT_LAUNCH();
  XYZZ<F>* part = reinterpret_cast<XYZZ<F>*>(L.part);
  const uint32_t at = p.tune.accum_threads;
  unsigned qb = (L.qmax + at - 1) / at;
  if (accum_stage >= 0) prof_mark(accum_stage, true, st);
  k_accum0<F><<<qb, at, 0, st>>>(L.sorted, L.offs, L.choff, L.chunk_key, K, T0, bases,
                                 reinterpret_cast<const Affine<F>* const*>(L.obases), p.key_shift, part); ZK_COUNT_LAUNCH();
  if (accum_stage >= 0) {
    prof_mark(accum_stage, false, st);
    if (uint32_t* hu = prof_units(accum_stage)) ZK_CUDA(cudaMemcpyAsync(hu, L.offs + K, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  }
  ZK_CUDA(cudaGetLastError());
  // fold each bucket's partials into its first slot (enough levels for the largest
  // possible chunk count; levels beyond the actual largest exit at once)
  uint32_t levels = 0;
  while ((uint64_t(1) << levels) < (S + T0 - 1) / T0 + 1) levels++;
  for (uint32_t l = 0; l < levels; l++) {
    unsigned fb = (L.qmax + 255) / 256;
    if (fb > p.tune.fold_blocks) fb = p.tune.fold_blocks;
    k_fold<F><<<fb, 256, 0, st>>>(part, L.choff, L.chunk_key, K, L.max_chunks, l); ZK_COUNT_LAUNCH();
  }
  ZK_CUDA(cudaGetLastError());
  // sum_v v B_v per (output, window) by bit decomposition
  XYZZ<F>* U = reinterpret_cast<XYZZ<F>*>(L.U);
  XYZZ<F>* D = reinterpret_cast<XYZZ<F>*>(L.D);
  k_bits_first<F><<<(L.utotal + 255) / 256, 256, 0, st>>>(part, L.counts, L.choff, L.bsegs, L.nbits, L.utotal, U); ZK_COUNT_LAUNCH();
  ZK_TRY(run_tree<F>(U, h.ut, L.useg, L.ucum, st));
  k_bits_scale<F><<<(L.nbits + 63) / 64, 64, 0, st>>>(U, L.bsegs, L.nbits, D); ZK_COUNT_LAUNCH();
  ZK_TRY(run_tree<F>(D, h.dt, L.dseg, L.dcum, st));
  k_combine_windows<F><<<((uint32_t)p.outs.size() + 63) / 64, 64, 0, st>>>(D, L.oitems, (uint32_t)p.outs.size(), results); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

const uint32_t* msm_term_count(const MsmExec* ex) {
  if (!ex || !ex->st) return nullptr;
  return ex->st->L.offs + ex->plan.keys;
}

template <class F>
int msm_run(const MsmPlan& p, const Affine<F>* bases, void* ws, size_t ws_bytes, XYZZ<F>* results, cudaStream_t st,
            int accum_stage) {
  MsmExec ex;
  ZK_TRY(msm_prepare<F>(p, ws, ws_bytes, &ex));
  ZK_TRY(msm_upload(&ex, st));
  return msm_launch<F>(&ex, bases, results, st, accum_stage);
}

template size_t msm_workspace_bytes<Fp>(const MsmPlan&);
template size_t msm_workspace_bytes<Fp2>(const MsmPlan&);
template int msm_run<Fp>(const MsmPlan&, const Affine<Fp>*, void*, size_t, XYZZ<Fp>*, cudaStream_t, int);
template int msm_run<Fp2>(const MsmPlan&, const Affine<Fp2>*, void*, size_t, XYZZ<Fp2>*, cudaStream_t, int);
template int msm_prepare<Fp>(const MsmPlan&, void*, size_t, MsmExec*);
template int msm_prepare<Fp2>(const MsmPlan&, void*, size_t, MsmExec*);
template int msm_launch<Fp>(const MsmExec*, const Affine<Fp>*, XYZZ<Fp>*, cudaStream_t, int);
template int msm_launch<Fp2>(const MsmExec*, const Affine<Fp2>*, XYZZ<Fp2>*, cudaStream_t, int);

}  // namespace zkvc
