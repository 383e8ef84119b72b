// Pippenger multi-scalar multiplication (the A, B, L and H queries of the Groth16
// prover, zkVC Sec. II / IV; the MSMs dominate proving time).
//
// Scalars are recoded into signed c-bit digits d in (-2^(c-1), 2^(c-1)], so a digit
// selects bucket |d| and the sign negates the base's y coordinate.  Every nonzero digit
// becomes one term (bucket key, base index | sign).  Terms are counting-sorted by key
// (histogram, scan, atomic scatter), then the sorted terms are summed by a balanced
// segmented reduction: every chunk of T0 consecutive sorted terms goes to one thread
// (mixed XYZZ + affine additions), which stores a partial sum each time a bucket ends
// inside its chunk, so every thread does the same number of additions whatever the
// bucket sizes; the partial sums of a bucket are then added along a binary tree in one
// launch -- of two sibling subtrees, the thread that finishes second (an atomic counter
// per tree node tells it) adds both and climbs on, the first one exits.  Heavily skewed buckets (int8 scalars put ~1300 terms in each of 128
// buckets) so cost only log2 of their chunk count in depth, with no extra launches.
// A window's result sum_v v B_v is evaluated as sum_b 2^b U_b with U_b the sum of the
// buckets whose index has bit b set: one block per slice of a bit's buckets reduces it
// in shared memory, one block per bit adds the slices and doubles b times, one block per
// window adds the bits -- log-depth instead of a running sum, since a point addition is
// long-latency on the GPU (about 10 us for one thread).  Where few sums remain, the
// additions and doublings run on quads of lanes (coop.cuh).
//
// Fixed-base MSMs (proving-key queries) store the multiples 2^(c w) P of each base, so all
// windows share one bucket set and no doubling chain follows; variable-base MSMs keep
// one bucket set per window and combine windows by Horner's rule.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "coop.cuh"
#include "msm.h"
#include "sliced.cuh"

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

// Exclusive scan of n_in values into n_out outputs by one block of 1024 threads, in
// tiles of 4096 consecutive entries (each thread four of them, loaded and stored as one
// 16-byte vector where the tile is whole, so every warp access is coalesced), with a
// block-wide scan per tile and the running total carried between tiles; also writes the
// first n_copy outputs to copy (if non-null).  in, out and copy are 16-byte aligned (the
// MSM workspace's).  For outputs up to SCAN1_MAX: one launch instead of three.
constexpr size_t SCAN1_MAX = 1024 * 64;
__global__ void __launch_bounds__(1024) k_scan_single(const uint32_t* __restrict__ in, size_t n_in, uint32_t* out,
                                                      size_t n_out, uint32_t* copy, size_t n_copy) {
  __shared__ uint32_t wsum[32];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t carry = 0;
  for (size_t t0 = 0; t0 < n_out; t0 += 4096) {
    const size_t i0 = t0 + size_t(threadIdx.x) * 4;
    uint32_t v[4];
    if (i0 + 4 <= n_in) {
      const uint4 q = *reinterpret_cast<const uint4*>(in + i0);
      v[0] = q.x;
      v[1] = q.y;
      v[2] = q.z;
      v[3] = q.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; j++) v[j] = i0 + j < n_in ? in[i0 + j] : 0u;
    }
    const uint32_t tot = v[0] + v[1] + v[2] + v[3];
    uint32_t x = tot;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= (uint32_t)d) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      uint32_t w = wsum[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
        if (lane >= (uint32_t)d) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    uint32_t e[4];
    e[0] = carry + x - tot + (wid ? wsum[wid - 1] : 0u);
    e[1] = e[0] + v[0];
    e[2] = e[1] + v[1];
    e[3] = e[2] + v[2];
    if (i0 + 4 <= n_out) {
      *reinterpret_cast<uint4*>(out + i0) = make_uint4(e[0], e[1], e[2], e[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; j++)
        if (i0 + j < n_out) out[i0 + j] = e[j];
    }
    if (copy) {
      if (i0 + 4 <= n_copy) {
        *reinterpret_cast<uint4*>(copy + i0) = make_uint4(e[0], e[1], e[2], e[3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; j++)
          if (i0 + j < n_copy) copy[i0 + j] = e[j];
      }
    }
    carry += wsum[31];
    __syncthreads();  // every thread has read wsum before the next tile writes it
  }
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

int scan_u32(const uint32_t* in, uint32_t* out, size_t n, Arena& a, cudaStream_t st, uint32_t* copy) {
  const bool aligned16 = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out) |
                           reinterpret_cast<uintptr_t>(copy)) & 15u) == 0;  // k_scan_single's vector accesses
  if (n + 1 <= SCAN1_MAX && (aligned16 || a.measuring)) {
    if (!a.measuring) {
      k_scan_single<<<1, 1024, 0, st>>>(in, n, out, n + 1, copy, copy ? n : 0); ZK_COUNT_LAUNCH();
      ZK_CUDA(cudaGetLastError());
    }
    return ZKVC_OK;
  }
  ZK_TRY(scan_rec(in, n, out, n + 1, a, st));
  if (copy && !a.measuring) ZK_CUDA(cudaMemcpyAsync(copy, out, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
  return ZKVC_OK;
}

size_t scan_u32_temp_bytes(size_t n) {
  Arena a;
  a.measuring = true;
  scan_rec(nullptr, n, nullptr, n + 1, a, 0);
  return a.off;
}

// ------------------------------------------------------------------ planning
// Threads of the G1 accumulation kernel resident on the whole GPU at `at` threads per
// block (one per chunk), from the occupancy of its register use; cached per block size.
static uint64_t accum_resident_threads(uint32_t at);

int msm_plan_finalize(MsmPlan& p) {
  uint32_t key = 0;
  for (auto& o : p.outs) {
    ZK_CHECK(o.c >= 2 && o.c <= 20, ZKVC_EINVAL, "msm: window of %u bits", o.c);
    ZK_CHECK(o.win_keys >= 1, ZKVC_EINVAL, "msm: win_keys = 0");
    // k_bits_chain stages an output's window sums in its shared array (64 points in G2)
    ZK_CHECK(o.win_keys <= 64, ZKVC_EINVAL, "msm: %u windows in one output (at most 64)", o.win_keys);
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
      case SK_SIGNED127: nd = (128 + o.c - 1) / o.c; break;  // nd c >= 128: the top window takes the last carry
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
  // term indices, bucket offsets and chunk bounds are 32-bit: 2^31 slots leave every sum
  // of an index and a chunk length below 2^32
  ZK_CHECK(slot <= (1ull << 31), ZKVC_EINVAL, "msm: %llu digit slots (at most 2^31)", (unsigned long long)slot);
  // default chunk: about two chunks per bucket, but at least ~40 k chunks so that the
  // accumulation fills the GPU, and 16 at the least; and at least the chunk that puts
  // every term into one wave of resident accumulation threads (the chunks are balanced,
  // so a second, partial wave would only add a tail)
  if (p.tune.chunk) {
    p.chunk = p.tune.chunk;
  } else {
    const uint64_t per_bucket = slot / (2ull * std::max<uint32_t>(key, 1u));
    const uint64_t fill = slot / 40960ull;
    // (7/8 of the resident threads: the prover's other streams hold some SM slots)
    const uint64_t resident = accum_resident_threads(p.tune.accum_threads) * 7 / 8;
    const uint64_t one_wave = resident ? (slot + resident - 1) / resident : 0;
    p.chunk = (uint32_t)std::min<uint64_t>(
        std::max<uint64_t>(std::max<uint64_t>(16, std::min(per_bucket, fill)), one_wave), 1024);
  }
  ZK_CHECK(p.chunk >= 1 && p.chunk <= 1024, ZKVC_EINVAL, "msm: chunk of %u terms", p.chunk);
  ZK_CHECK(p.tune.accum_threads >= 32 && p.tune.accum_threads <= 256 && p.tune.accum_threads % 32 == 0,
           ZKVC_EINVAL, "msm: %u accumulation threads", p.tune.accum_threads);
  ZK_CHECK(p.tune.lanes == 0 || p.tune.lanes == 1 || p.tune.lanes == 4, ZKVC_EINVAL, "msm: %u lanes per chunk",
           p.tune.lanes);
  p.slots = slot;
  p.points = pts;
  // lanes per chunk: quads where the run has too few chunks to fill the GPU (their point
  // operations have a third of a thread's latency), one thread where it is throughput-bound
  p.lanes = p.tune.lanes ? p.tune.lanes : (slot / p.chunk < 40960 ? 4u : 1u);
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

// counts (non-null): also counts each key (global atomics), for runs whose terms spread
// over many buckets, where k_hist's shared-memory window would not help anyway.
__global__ void k_digits(const MsmSeg* __restrict__ segs, int nsegs, const MsmOut* __restrict__ outs,
                         uint32_t total_points, uint32_t* keys, uint32_t* vals, uint32_t* counts) {
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
      case SK_SIGNED127: {
        const uint4 v = reinterpret_cast<const uint4*>(sg.scalars)[i];
        m[0] = v.x;
        m[1] = v.y;
        m[2] = v.z;
        m[3] = v.w & 0x7fffffffu;
        neg = (v.w >> 31) != 0;
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
    if (counts) atomicAdd(counts + key, 1u);
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

// Partial-sum slots of the balanced accumulation.  Chunk q covers the sorted terms
// [q T0, (q + 1) T0); bucket k covers [offs[k], offs[k+1]).  A (chunk, bucket) pair that
// overlaps stores its partial sum at slot q + k: walking the terms in order, each step to
// the next overlapping pair moves to the next chunk, the next non-empty bucket or both, so
// q + k strictly increases and the slots are distinct.  Bucket k (count > 0) owns the
// contiguous slots [choff[k], choff[k] + nch[k]) with choff[k] = offs[k] / T0 + k and nch[k]
// the chunks it overlaps; choff[K] bounds all slots.
//
// A bucket with 2 .. FOLD_SERIAL slots also names itself in flist at its first chunk
// boundary (index offs[k] / T0 + 1, one bucket per boundary at most), so that sparse folds
// can run over the boundaries instead of over every bucket.  Entries no bucket names keep
// stale values, which the fold rejects.
constexpr uint32_t FOLD_SERIAL = 4;
__global__ void k_chunk_layout(const uint32_t* __restrict__ counts, const uint32_t* __restrict__ offs, uint32_t K,
                               uint32_t T0, uint32_t* nch, uint32_t* choff, uint32_t* chunk_key, uint32_t* flist) {
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > K) return;
  if (k == K) {
    choff[K] = (offs[K] + T0 - 1) / T0 + K;
    return;
  }
  const uint32_t lo = offs[k] / T0;
  const uint32_t c = lo + k, np = counts[k] ? (offs[k + 1] - 1) / T0 - lo + 1 : 0u;
  choff[k] = c;
  nch[k] = np;
  for (uint32_t q = c; q < c + np; q++) chunk_key[q] = k;  // the bucket of each of its slots
  if (np >= 2 && np <= FOLD_SERIAL) flist[lo + 1] = k;
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
// fetch-and-add with release (this thread's earlier stores) and acquire (its later
// loads) semantics at GPU scope
__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// point loads that bypass L1: a sibling's partial sum written by another SM
template <class F>
__device__ __forceinline__ XYZZ<F> ld_point_cg(const XYZZ<F>* p) {
  XYZZ<F> r;
  uint32_t* d = reinterpret_cast<uint32_t*>(&r);
  const uint4* s = reinterpret_cast<const uint4*>(p);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(XYZZ<F>) / 16); i++) {
    uint4 q = __ldcg(s + i);
    d[4 * i] = q.x;
    d[4 * i + 1] = q.y;
    d[4 * i + 2] = q.z;
    d[4 * i + 3] = q.w;
  }
  return r;
}

// Lanes per chunk (QL): one thread, or a quad of lanes (coop.cuh) whose point operations
// have a third of a thread's latency for four times the lanes.  G2 chunks always take a
// quad (the G2 runs of a proof are latency-bound); a G1 run takes what its tuning says
// (MsmTune::lanes: quads pay where the run is latency-bound, one thread where it fills
// the GPU).
template <int QL, class F>
__device__ __forceinline__ XYZZ<F> madd_lanes(const XYZZ<F>& p, const Affine<F>& q) {
  if constexpr (QL == 1) return p_add_affine(p, q);
  else return p_add_affine_quad(p, q);
}

#ifndef ZKVC_ACCUM_MINB
#define ZKVC_ACCUM_MINB 1
#endif
template <class F>
struct AccumMinB {
  static constexpr int value = sizeof(F) > 32 ? 1 : ZKVC_ACCUM_MINB;
};

// level 0: chunk q sums the sorted terms [q T0, (q + 1) T0) with mixed additions, storing
// its running sum at slot q + k whenever bucket k ends inside the chunk and at its end
template <class F, int QL>
__global__ void __launch_bounds__(256, AccumMinB<F>::value) k_accum0(const uint32_t* __restrict__ sorted,
                                                                    const uint32_t* __restrict__ offs, uint32_t K,
                                                                    uint32_t T0, const Affine<F>* __restrict__ bases,
                                                                    const Affine<F>* const* __restrict__ obases,
                                                                    int key_shift, XYZZ<F>* part) {
  const uint32_t q = (blockIdx.x * blockDim.x + threadIdx.x) / QL;
  const uint32_t S = offs[K];
  const uint64_t start64 = uint64_t(q) * T0;
  if (start64 >= S) return;  // uniform within a quad
  const uint32_t start = (uint32_t)start64;
  const uint64_t end64 = start64 + T0;
  const uint32_t end = end64 < S ? (uint32_t)end64 : S;
  uint32_t k = find_key(offs, K, start);  // the bucket holding term `start`
  uint32_t next = offs[k + 1];
  if (key_shift >= 0) bases = obases[k >> key_shift];
  const bool lead = QL == 1 || quad_lane() == 0;
  XYZZ<F> acc = XYZZ<F>::inf();
  // one loop of exactly end - start additions for every lane (no divergence between
  // lanes whose buckets end at different terms); a bucket's end stores the partial sum
  // and restarts the sum at infinity (ZZ = 0)
  for (uint32_t p = start; p < end; p++) {
    if (p >= next) {
      if (lead) st_field(part + q + k, acc);
      acc.ZZ = F::zero();
      acc.ZZZ = F::zero();
      do {  // the next non-empty bucket
        k++;
        next = offs[k + 1];
      } while (p >= next);
      if (key_shift >= 0) bases = obases[k >> key_shift];
    }
    uint32_t v = sorted[p];
    Affine<F> P = ld_field(bases + (v & 0x7fffffffu));
    if (v >> 31) P.y = f_neg(P.y);
    acc = madd_lanes<QL>(acc, P);
  }
  if (lead) st_field(part + q + k, acc);
}

// Buckets with at most FOLD_SERIAL partial sums (the common case of a balanced
// accumulation: a bucket split by one or two chunk boundaries) are folded by one thread
// (or quad) per bucket, serially, without counters; the tree (fold_tree_at) takes the
// larger ones.
// Where chunk boundaries are fewer than buckets (large chunks over many small buckets),
// the quads go over the boundaries' fold list instead (flist non-null, nlist entries), so
// that every launched quad has a bucket to fold.
template <class F, int QL>
__device__ __forceinline__ void fold_serial_at(uint32_t i, const uint32_t* __restrict__ choff,
                                               const uint32_t* __restrict__ nch, uint32_t K, XYZZ<F>* part,
                                               const uint32_t* __restrict__ flist, uint32_t nlist,
                                               const uint32_t* __restrict__ offs, uint32_t T0) {
  uint32_t k = i;
  if (flist) {
    if (i == 0 || i >= nlist) return;  // uniform within a quad
    k = flist[i];
    if (k >= K || offs[k] / T0 + 1 != i) return;  // no bucket's first boundary (stale entry)
  } else if (k >= K) {
    return;
  }
  const uint32_t np = nch[k];
  if (np < 2 || np > FOLD_SERIAL) return;
  const uint32_t base = choff[k];
  XYZZ<F> acc = ld_field(part + base);
  for (uint32_t i = 1; i < np; i++) {
    const XYZZ<F> o = ld_field(part + base + i);
    if (QL > 1)
      acc = p_add_quad(acc, o);
    else
      acc = p_add(acc, o);
  }
  if (QL == 1 || quad_lane() == 0) st_field(part + base, acc);
}

static uint64_t accum_resident_threads(uint32_t at) {
  static std::atomic<int> per_sm[9];
  if (at < 32 || at > 256 || at % 32) return 0;
  int nb = per_sm[at / 32].load(std::memory_order_relaxed);
  if (nb <= 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_accum0<Fp, 1>, (int)at, 0) != cudaSuccess || nb <= 0) {
      cudaGetLastError();
      return 0;
    }
    per_sm[at / 32].store(nb, std::memory_order_relaxed);
  }
  return uint64_t(nb) * at * (uint64_t)device_sm_count();
}

// The partial sums of each bucket (its np = nch[k] slots from choff[k]) are added along
// the binary tree over slot positions 0..np-1, in one launch: at span s the subtree at position i (a multiple of s) pairs
// with the one at i ^ s.  Each sibling counts in at the node's counter (index: left
// position + s - 1, distinct over all levels since it ends in exactly log2 s one-bits);
// the first to arrive exits, the second adds both sums and climbs on.  A left subtree
// with no right sibling climbs without waiting.  A subtree's sum sits at its left
// position: a climber stores only sums it has changed (a chunk's own sum is there from
// the accumulation launch).  The bucket total ends in part[choff[k]].  `arrive` holds one
// zeroed counter per chunk.  The counter's fetch-and-add releases the climber's store
// and acquires its sibling's.  QL lanes per chunk as in the accumulation.
template <class F, int QL>
__device__ __forceinline__ void fold_tree_at(uint32_t q, const uint32_t* __restrict__ choff,
                                             const uint32_t* __restrict__ nch, const uint32_t* __restrict__ chunk_key,
                                             uint32_t K, XYZZ<F>* part, uint32_t* arrive) {
  if (q >= choff[K]) return;  // uniform within a quad
  // chunk_key is written only for owned slots: any other value (a previous run's, or
  // never written) fails the range check
  const uint32_t k = chunk_key[q];
  if (k >= K) return;
  const uint32_t base = choff[k], np = nch[k];
  if (q < base || q >= base + np) return;  // a slot no bucket owns
  if (np <= FOLD_SERIAL) return;  // folded serially
  const bool lead = QL == 1 || quad_lane() == 0;
  uint32_t pos = q - base;
  XYZZ<F> acc;
  bool have = false;  // acc holds this subtree's sum (else it is only in part[])
  for (uint32_t span = 1; span < np; span <<= 1) {
    const bool left = (pos & span) == 0;
    const uint32_t sib = pos ^ span;
    if (left && sib >= np) continue;
    uint32_t first = 0;
    if (lead) {
      if (have) st_field(part + base + pos, acc);
      first = atom_add_acq_rel(arrive + base + (left ? pos : sib) + span - 1, 1u) == 0;
    }
    if (QL > 1) {
      first = __shfl_sync(quad_mask(), first, quad_base());
      __syncwarp(quad_mask());  // orders the lead's acquire before the quad's loads
    }
    if (first) return;
    if (!have) acc = ld_point_cg(part + base + pos);
    const XYZZ<F> o = ld_point_cg(part + base + sib);
    if (QL > 1)
      acc = left ? p_add_quad(acc, o) : p_add_quad(o, acc);
    else
      acc = left ? p_add(acc, o) : p_add(o, acc);
    have = true;
    pos = left ? pos : sib;
  }
  if (have && lead) st_field(part + base, acc);
}

// Both folds in one launch (disjoint buckets: at most FOLD_SERIAL partials go serially,
// more along the tree): quad (or thread) i takes serial entry i (bucket i, or boundary i
// of the fold list) and tree slot i.
template <class F, int QL>
__global__ void __launch_bounds__(128) k_fold(const uint32_t* __restrict__ choff, const uint32_t* __restrict__ nch,
                                              const uint32_t* __restrict__ chunk_key, uint32_t K, XYZZ<F>* part,
                                              uint32_t* arrive, const uint32_t* __restrict__ flist, uint32_t nlist,
                                              const uint32_t* __restrict__ offs, uint32_t T0, uint32_t n_serial) {
  const uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) / QL;
  if (i < n_serial) fold_serial_at<F, QL>(i, choff, nch, K, part, flist, nlist, offs, T0);
  fold_tree_at<F, QL>(i, choff, nch, chunk_key, K, part, arrive);
}

template <class F>
__device__ __forceinline__ XYZZ<F> bucket_at(const XYZZ<F>* fin, const uint32_t* counts, const uint32_t* choff,
                                             uint32_t key) {
  if (counts[key] == 0) return XYZZ<F>::inf();
  return ld_field(fin + choff[key]);
}

// Sum of m points get(0..m-1) by a block of BT threads (a multiple of 4), returned to
// every thread; sh holds BT points.  G1 levels with more pairs than quads give a pair to
// a thread, the others a pair (or several in turn) to a quad (coop.cuh); G2 levels always
// use quads.  Every thread of the block must call it.
template <class F, int BT, class Get>
__device__ XYZZ<F> block_sum(Get get, uint32_t m, XYZZ<F>* sh) {
  constexpr bool all_quads = sizeof(F) > 32;
  constexpr uint32_t NQ = BT / 4;
  const uint32_t t = threadIdx.x, qd = t >> 2;
  const bool lead = (t & 3) == 0;
  uint32_t n;
  if (m > 2 * BT) {
    if (all_quads) {
      XYZZ<F> acc = XYZZ<F>::inf();
      for (uint32_t i = qd; i < m; i += NQ) acc = p_add_quad(acc, get(i));
      if (lead) st_field(sh + qd, acc);
      n = NQ;
    } else {
      XYZZ<F> acc = XYZZ<F>::inf();
      for (uint32_t i = t; i < m; i += BT) acc = p_add(acc, get(i));
      st_field(sh + t, acc);
      n = BT;
    }
  } else {
    const uint32_t pairs = (m + 1) / 2;
    if (!all_quads && pairs > NQ) {
      if (t < pairs) {
        XYZZ<F> a = get(2 * t);
        if (2 * t + 1 < m) a = p_add(a, get(2 * t + 1));
        st_field(sh + t, a);
      }
    } else {
      for (uint32_t pr = qd; pr < pairs; pr += NQ) {
        XYZZ<F> a = get(2 * pr);
        if (2 * pr + 1 < m) a = p_add_quad(a, get(2 * pr + 1));
        if (lead) st_field(sh + pr, a);
      }
    }
    n = pairs;
  }
  __syncthreads();
  while (n > 1) {
    const uint32_t h = (n + 1) / 2, pairs = n - h;  // entry i < pairs absorbs entry i + h
    if (!all_quads && pairs > NQ) {
      if (t < pairs) st_field(sh + t, p_add(ld_field(sh + t), ld_field(sh + t + h)));
    } else {
      for (uint32_t pr = qd; pr < pairs; pr += NQ) {
        const XYZZ<F> r = p_add_quad(ld_field(sh + pr), ld_field(sh + pr + h));
        __syncwarp(quad_mask());  // the quad's reads of sh[pr] precede the lead's store
        if (lead) st_field(sh + pr, r);
      }
    }
    __syncthreads();
    n = h;
  }
  return m ? ld_field(sh) : XYZZ<F>::inf();
}

// Window result sum_{v=1}^{NB} v B_v = sum_b 2^b U_b with U_b = sum_{v : bit b of v} B_v.
// One BitSeg per (output, window, bit); its cnt buckets are cut into slices, each summed
// by one block (serial sums per thread first, then the block's tree).
//
// Large windows (c >= SPLIT_MIN_C: the fixed-base outputs over stored multiples and every
// window of a large variable-base MSM) first split every
// bucket index as v = 2^h hi + lo: sum_v v B_v = sum_lo lo C_lo + 2^h sum_hi hi D_hi with
// C_lo = sum_{v : low h bits = lo} B_v and D_hi = sum_{v : v >> h = hi} B_v (each bucket
// added twice, by k_split_gather), and the bit decomposition then runs over the two small
// "pseudo-bucket" sets: lo in [1, 2^h) with bits 0 .. h-1, hi in [1, 2^(c-1-h)] with bits
// 0 .. c-1-h whose terms are doubled b + h times.  For c = 16: 2 x 32 k additions to
// gather and 1.5 k for the bits, instead of 246 k for the bits alone.
constexpr uint32_t SPLIT_MIN_C = 12;
constexpr uint32_t BS_PSEUDO = 0x100;  // BitSeg::mode: key0 indexes the pseudo-bucket array
struct BitSeg {
  uint32_t key0;    // key of bucket v = 1 of this (output, window), or of pseudo-bucket 1
  uint32_t b, c;    // bit, window bits (of the pseudo set for pseudo-buckets)
  uint32_t cnt;     // buckets with bit b
  uint32_t soff;    // first slice in the slice-sum buffer
  uint32_t nsl;     // slices
  uint32_t dslot;   // slot of 2^shift U_b in the D buffer
  uint32_t mode;    // bits 0-7: shift (doublings of U_b); BS_PSEUDO
  uint32_t win;     // the window's TreeSeg
};

// One split window: the pseudo-buckets C_1 .. C_(2^h - 1) then D_1 .. D_(2^(c-1-h)) at
// P[pbase ...], one k_split_gather block each, blocks blk0 ...
struct SplitWin {
  uint32_t key0;  // key of bucket v = 1
  uint32_t c, h;
  uint32_t pbase;
  uint32_t blk0;
  uint32_t pad[3];
};

__device__ __forceinline__ uint32_t nth_with_bit(uint32_t b, uint32_t c, uint32_t idx) {
  if (b == c - 1) return 1u << (c - 1);
  return ((idx >> b) << (b + 1)) | (1u << b) | (idx & ((1u << b) - 1u));
}

// 128 (G1) or 64 (G2) threads: several blocks fit an SM beside the register-heavy point
// formulas, so SMs stay busy while a block's tree narrows
template <class F>
struct SliceBT {
  static constexpr int value = sizeof(F) > 32 ? 64 : 128;
};
// one wave of slice blocks: three resident per SM
static uint32_t slice_wave() { return 3u * (uint32_t)device_sm_count(); }

// block per pseudo-bucket of a split window: C_lo (members v = 2^h hi + lo, hi <
// 2^(c-1-h)) or D_hi (members v = 2^h hi + lo, lo < 2^h, v <= 2^(c-1))
template <class F>
__global__ void __launch_bounds__(SliceBT<F>::value) k_split_gather(const XYZZ<F>* __restrict__ fin,
                                                                     const uint32_t* __restrict__ counts,
                                                                     const uint32_t* __restrict__ choff,
                                                                     const SplitWin* __restrict__ wins, uint32_t nwin,
                                                                     XYZZ<F>* P) {
  constexpr int BT = SliceBT<F>::value;
  __shared__ XYZZ<F> sh[BT];
  uint32_t lo = 0, hi = nwin - 1;
  while (lo < hi) {
    uint32_t mid = (lo + hi + 1) >> 1;
    if (wins[mid].blk0 <= blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const SplitWin g = wins[lo];
  const uint32_t cls = blockIdx.x - g.blk0, nlo = (1u << g.h) - 1u, nb = 1u << (g.c - 1);
  uint32_t m, step, first;
  if (cls < nlo) {  // C_(cls + 1)
    first = cls + 1;
    step = 1u << g.h;
    m = 1u << (g.c - 1 - g.h);
  } else {          // D_(cls - nlo + 1)
    first = (cls - nlo + 1) << g.h;
    step = 1;
    m = min(1u << g.h, nb - first + 1);
  }
  auto get = [&](uint32_t i) { return bucket_at(fin, counts, choff, g.key0 + first + i * step - 1); };
  const XYZZ<F> r = block_sum<F, BT>(get, m, sh);
  if (threadIdx.x == 0) st_field(P + g.pbase + cls, r);
}

// block per (output, window): the window's c terms 2^b U_b, summed into the first slot
struct TreeSeg {
  uint32_t off;  // first element
  uint32_t len;  // elements
  uint32_t out;  // its output
};

// results[o] = sum_w 2^(c w) W[o][w] by Horner's rule for variable-base outputs (a chain
// of c (nwin - 1) doublings), the window's sum itself for the rest.
struct OutItem {
  uint32_t first;     // index of window 0's result in D
  uint32_t stride;    // distance between windows' results
  uint32_t nwin;
  uint32_t c;
};

// The bucket sums after the folds, in one launch whose levels hand over through counters
// instead of launch boundaries:
//   slice  block per slice of one bit's buckets: the slice's sum (serial per thread, then
//          the block's tree) into S;
//   bit    the last slice block of a bit to finish sums the bit's slices (U_b) and doubles
//          it b times (2^b U_b; G1 on one warp in limb-sliced arithmetic, G2 on a quad);
//   window the last bit of a window sums the window's c terms 2^b U_b;
//   output the last window of an output applies Horner's rule over the output's windows
//          (variable base; G1 on a sliced warp, G2 on a quad) or copies its one window.
// Each hand-over: the finishing block's stores, a fence by every storing thread, a
// barrier, then a fetch-and-add on the level's counter (zeroed before the launch) by one
// thread; the block that brings the count to the total goes on, after a fence, reading
// the others' results around L1.  No block waits.
template <class F>
__global__ void __launch_bounds__(SliceBT<F>::value) k_bits_chain(
    const XYZZ<F>* __restrict__ fin, const uint32_t* __restrict__ counts, const uint32_t* __restrict__ choff,
    const BitSeg* __restrict__ segs, uint32_t nseg, uint32_t slice, const XYZZ<F>* __restrict__ P, XYZZ<F>* S,
    XYZZ<F>* D, const TreeSeg* __restrict__ dsegs, const OutItem* __restrict__ oitems, XYZZ<F>* results,
    uint32_t* cnt_bit, uint32_t* cnt_win, uint32_t* cnt_out) {
  constexpr int BT = SliceBT<F>::value;
  __shared__ XYZZ<F> sh[BT];
  __shared__ XYZZ<F> xs;
  __shared__ uint32_t last;
  const uint32_t sl = blockIdx.x;
  uint32_t lo = 0, hi = nseg - 1;
  while (lo < hi) {
    uint32_t mid = (lo + hi + 1) >> 1;
    if (segs[mid].soff <= sl) lo = mid; else hi = mid - 1;
  }
  const BitSeg g = segs[lo];
  // slice
  {
    const uint32_t first = (sl - g.soff) * slice;
    const uint32_t m = min(slice, g.cnt - first);
    const bool pseudo = (g.mode & BS_PSEUDO) != 0;
    auto get = [&](uint32_t i) {
      const uint32_t v = nth_with_bit(g.b, g.c, first + i);
      return pseudo ? ld_field(P + g.key0 + v - 1) : bucket_at(fin, counts, choff, g.key0 + v - 1);
    };
    const XYZZ<F> r = block_sum<F, BT>(get, m, sh);
    if (threadIdx.x == 0) {
      st_field(S + sl, r);
      __threadfence();
      last = atomicAdd(cnt_bit + lo, 1u) == g.nsl - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
  }
  // bit
  {
    auto get = [&](uint32_t i) { return ld_point_cg(S + g.soff + i); };
    XYZZ<F> x = block_sum<F, BT>(get, g.nsl, sh);
    const uint32_t shift = g.mode & 0xffu;
    if constexpr (sizeof(F) == sizeof(Fp)) {
      if (threadIdx.x == 0) st_field(&xs, x);
      __syncthreads();
      if (threadIdx.x < 32) {
        SlG1 y = sl_ld(&xs);
        for (uint32_t i = 0; i < shift; i++) y = sl_pdbl(y);
        sl_st(D + g.dslot, y);  // eight lanes store a word of each coordinate
      }
    } else {
      if (threadIdx.x < 4) {
        for (uint32_t i = 0; i < shift; i++) x = p_dbl_quad(x);
        if (threadIdx.x == 0) st_field(D + g.dslot, x);
      }
    }
    __threadfence();  // by every storing lane, before the barrier and the count below
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      last = atomicAdd(cnt_win + g.win, 1u) == dsegs[g.win].len - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
  }
  // window
  const TreeSeg w = dsegs[g.win];
  {
    auto get = [&](uint32_t i) { return ld_point_cg(D + w.off + i); };
    const XYZZ<F> r = block_sum<F, BT>(get, w.len, sh);
    if (threadIdx.x == 0) {
      st_field(D + w.off, r);
      __threadfence();
      last = atomicAdd(cnt_out + w.out, 1u) == oitems[w.out].nwin - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
  }
  // output (at most 64 windows, which the shared array holds: checked by the planner)
  const OutItem it = oitems[w.out];
  for (uint32_t i = threadIdx.x; i < it.nwin; i += BT) st_field(sh + i, ld_point_cg(D + it.first + i * it.stride));
  __syncthreads();
  if constexpr (sizeof(F) == sizeof(Fp)) {
    if (threadIdx.x >= 32) return;
    SlG1 acc = sl_ld(sh + it.nwin - 1);
    for (int v = (int)it.nwin - 2; v >= 0; v--) {
      for (uint32_t i = 0; i < it.c; i++) acc = sl_pdbl(acc);
      acc = sl_padd(acc, sl_ld(sh + v));
    }
    sl_st(results + w.out, acc);
  } else {
    if (threadIdx.x >= 4) return;
    XYZZ<F> acc = ld_field(sh + it.nwin - 1);
    for (int v = (int)it.nwin - 2; v >= 0; v--) {
      for (uint32_t i = 0; i < it.c; i++) acc = p_dbl_quad(acc);
      acc = p_add_quad(acc, ld_field(sh + v));
    }
    if (threadIdx.x == 0) st_field(results + w.out, acc);
  }
}

// ------------------------------------------------------------------ driver
struct Layout {
  uint32_t *keys, *vals, *sorted, *counts, *offs, *cursor, *nch, *choff, *chunk_key, *arrive, *flist;
  void *part, *S, *D;
  MsmSeg* segs;
  MsmOut* outs;
  const void** obases;
  BitSeg* bsegs;
  TreeSeg* dseg;
  OutItem* oitems;
  SplitWin* swins;
  void* P;         // pseudo-buckets of the split windows
  uint32_t* cnt;   // k_bits_chain's counters: per bit, per window, per output
  uint32_t qmax, nbits, nslices, dtotal, slice, nswin, ngather, npseudo;
};

struct HostTables {
  std::vector<BitSeg> bsegs;
  std::vector<TreeSeg> dsegs;
  std::vector<OutItem> oitems;
  std::vector<const void*> obases;
  std::vector<SplitWin> swins;
};

struct MsmExecState {
  Layout L;
  HostTables h;
  Arena after_layout;  // the arena once the tables are carved: scans take from a copy
  bool uploaded = false;
};

MsmExec::~MsmExec() { delete st; }

// Slices of bt * r buckets, r >= 2 chosen so that the slice kernel fills about one wave
// of `wave` blocks (a lone wave's blocks each run their tree once; more buckets per
// slice are serial sums, which the SMs run at full rate).
static bool split_window(const MsmOut& o) { return o.c >= SPLIT_MIN_C; }

// additions of the bit decomposition of one window of c bits (plain or split)
static uint64_t bit_work(const MsmOut& o) {
  if (!split_window(o)) return (o.c - 1) * (1ull << (o.c - 2)) + 1;
  const uint32_t h = o.c / 2, ch = o.c - h;
  return uint64_t(h) * (1ull << (h - 1)) + (ch - 1) * (1ull << (ch - 2)) + 1;
}

static void tables(const MsmPlan& p, uint32_t bt, uint32_t wave, HostTables& h, Layout& L) {
  uint64_t total = 0;
  for (const auto& o : p.outs) total += uint64_t(o.win_keys) * bit_work(o);
  uint64_t r = (total + uint64_t(bt) * wave - 1) / (uint64_t(bt) * wave);
  r = std::min<uint64_t>(std::max<uint64_t>(r, 2), 64);
  const uint32_t slice = (uint32_t)(bt * r);
  L.slice = slice;
  h.bsegs.clear();
  h.dsegs.clear();
  h.oitems.clear();
  h.obases.clear();
  h.swins.clear();
  uint32_t soff = 0, dslot = 0, pbase = 0, blk = 0;
  auto add_bits = [&](uint32_t key0, uint32_t c, uint32_t b_from, uint32_t b_to, uint32_t shift0, uint32_t slot0,
                      uint32_t mode) {
    for (uint32_t b = b_from; b < b_to; b++) {
      const uint32_t cnt = (b == c - 1) ? 1u : (1u << (c - 2));
      const uint32_t nsl = (cnt + slice - 1) / slice;
      h.bsegs.push_back(
          {key0, b, c, cnt, soff, nsl, slot0 + b - b_from, mode | (shift0 + b), (uint32_t)h.dsegs.size() - 1});
      soff += nsl;
    }
  };
  for (const auto& o : p.outs) {
    const uint32_t nb = 1u << (o.c - 1);
    h.oitems.push_back({dslot, o.c, o.win_keys, o.c});
    h.obases.push_back(o.bases);
    for (uint32_t w = 0; w < o.win_keys; w++) {
      h.dsegs.push_back({dslot, o.c, (uint32_t)h.oitems.size() - 1});
      const uint32_t key0 = o.key_off + w * nb;
      if (split_window(o)) {
        // lo in [1, 2^h): bits 0 .. h-1 of a (h+1)-bit set; hi in [1, 2^(c-1-h)]: bits
        // 0 .. c-h-1 of a (c-h)-bit set, doubled h more times; c slots in all
        const uint32_t hh = o.c / 2, nlo = (1u << hh) - 1u, nhi = 1u << (o.c - 1 - hh);
        h.swins.push_back({key0, o.c, hh, pbase, blk, {0, 0, 0}});
        add_bits(pbase, hh + 1, 0, hh, 0, dslot, BS_PSEUDO);
        add_bits(pbase + nlo, o.c - hh, 0, o.c - hh, hh, dslot + hh, BS_PSEUDO);
        pbase += nlo + nhi;
        blk += nlo + nhi;
      } else {
        add_bits(key0, o.c, 0, o.c, 0, dslot, 0);
      }
      dslot += o.c;
    }
  }
  L.nbits = (uint32_t)h.bsegs.size();
  L.nslices = soff;
  L.dtotal = dslot;
  L.nswin = (uint32_t)h.swins.size();
  L.ngather = blk;
  L.npseudo = pbase;
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
  L.arrive = a.take<uint32_t>(L.qmax);
  L.flist = a.take<uint32_t>(L.qmax);
  L.part = a.take<XYZZ<F>>(L.qmax);
  tables(p, SliceBT<F>::value, slice_wave(), h, L);
  L.S = a.take<XYZZ<F>>(L.nslices);
  L.D = a.take<XYZZ<F>>(L.dtotal);
  L.segs = a.take<MsmSeg>(p.segs.size());
  L.outs = a.take<MsmOut>(p.outs.size());
  L.obases = a.take<const void*>(p.outs.size());
  L.bsegs = a.take<BitSeg>(h.bsegs.size());
  L.dseg = a.take<TreeSeg>(h.dsegs.size());
  L.oitems = a.take<OutItem>(h.oitems.size());
  L.swins = a.take<SplitWin>(h.swins.size());
  L.P = a.take<XYZZ<F>>(L.npseudo);
  L.cnt = a.take<uint32_t>(h.bsegs.size() + h.dsegs.size() + h.oitems.size());
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

// Pinned host memory that this thread's uploads take their table images from while a
// launch sequence that includes the uploads is being captured (the copy nodes then read
// it on every replay, so it must outlive the graph and keep its contents).
static thread_local uint8_t* t_stage = nullptr;
static thread_local size_t t_stage_cap = 0, t_stage_off = 0;

void msm_table_stage(uint8_t* host, size_t cap) {
  t_stage = host;
  t_stage_cap = host ? cap : 0;
  t_stage_off = 0;
}

// The tables are carved one after another (segs, outs, obases, bsegs, dseg, oitems, swins), so
// one image of their span, with each table at its device offset, goes up in one copy.
int msm_upload(MsmExec* ex, cudaStream_t st) {
  ZK_CHECK(ex && ex->st, ZKVC_EINVAL, "msm: exec not prepared");
  const MsmPlan& p = ex->plan;
  Layout& L = ex->st->L;
  HostTables& h = ex->st->h;
  uint8_t* const dev0 = reinterpret_cast<uint8_t*>(L.segs);
  uint8_t* const dev1 = h.swins.empty() ? reinterpret_cast<uint8_t*>(L.oitems) + h.oitems.size() * sizeof(OutItem)
                                        : reinterpret_cast<uint8_t*>(L.swins) + h.swins.size() * sizeof(SplitWin);
  ZK_CHECK(dev0 && dev1 > dev0, ZKVC_EINVAL, "msm: tables not carved");
  const size_t span = size_t(dev1 - dev0);
  std::vector<uint8_t> tmp;
  uint8_t* img = nullptr;
  if (t_stage) {
    ZK_CHECK(t_stage_off + span <= t_stage_cap, ZKVC_ENOMEM, "msm: %zu bytes of table staging are not enough",
             t_stage_cap);
    img = t_stage + t_stage_off;
    t_stage_off += (span + 255) & ~size_t(255);
  } else {
    tmp.resize(span);
    img = tmp.data();
  }
  auto put = [&](const void* dev, const void* src, size_t bytes) -> bool {
    const uint8_t* d = reinterpret_cast<const uint8_t*>(dev);
    if (bytes == 0) return true;
    if (d < dev0 || d + bytes > dev1) return false;
    std::memcpy(img + (d - dev0), src, bytes);
    return true;
  };
  const bool ok = put(L.segs, p.segs.data(), p.segs.size() * sizeof(MsmSeg)) &&
                  put(L.outs, p.outs.data(), p.outs.size() * sizeof(MsmOut)) &&
                  put(L.obases, h.obases.data(), h.obases.size() * sizeof(void*)) &&
                  put(L.bsegs, h.bsegs.data(), h.bsegs.size() * sizeof(BitSeg)) &&
                  put(L.dseg, h.dsegs.data(), h.dsegs.size() * sizeof(TreeSeg)) &&
                  put(L.oitems, h.oitems.data(), h.oitems.size() * sizeof(OutItem)) &&
                  put(L.swins, h.swins.data(), h.swins.size() * sizeof(SplitWin));
  ZK_CHECK(ok, ZKVC_EINVAL, "msm: tables outside their span");
  ZK_CUDA(cudaMemcpyAsync(dev0, img, span, cudaMemcpyHostToDevice, st));
  ex->st->uploaded = true;
  return ZKVC_OK;
}

template <class F>
int msm_launch(const MsmExec* ex, const Affine<F>* bases, XYZZ<F>* results, cudaStream_t st, int accum_stage,
               cudaEvent_t after_accum) {
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

  // digits -> terms, and the bucket counts of the counting sort: counted by the digits
  // kernel itself where every output has at least 2^11 buckets per window (random digits
  // then rarely repeat a key within a tile), else by k_hist
  bool spread = true;
  for (const auto& o : p.outs) spread = spread && o.c >= 12;
  ZK_CUDA(cudaMemsetAsync(L.counts, 0, size_t(K) * sizeof(uint32_t), st));
  if (p.points > 0) {
    k_digits<<<(p.points + 255) / 256, 256, 0, st>>>(L.segs, (int)p.segs.size(), L.outs, p.points, L.keys, L.vals,
                                                     spread ? L.counts : nullptr);
    ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaGetLastError());
  }
  unsigned sb = (unsigned)((S + HB_TILE - 1) / HB_TILE);
  if (S > 0 && !spread) {
    k_hist<<<sb, HB_THREADS, 0, st>>>(L.keys, S, L.counts); ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaGetLastError());
  }
  ZK_TRY(scan_u32(L.counts, L.offs, K, a, st, L.cursor));
  if (S > 0) {
    k_scatter<<<sb, HB_THREADS, 0, st>>>(L.keys, L.vals, S, L.cursor, L.sorted); ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaGetLastError());
  }
  // chunks of T0 sorted terms and the buckets' partial-sum slots
  k_chunk_layout<<<(K + 1 + 255) / 256, 256, 0, st>>>(L.counts, L.offs, K, T0, L.nch, L.choff, L.chunk_key,
                                                       L.flist);
  ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  ZK_CHECK(!a.overflow(), ZKVC_EINVAL, "msm: workspace too small for scans");
  ZK_CUDA(cudaMemsetAsync(L.arrive, 0, size_t(L.qmax) * sizeof(uint32_t), st));
  XYZZ<F>* part = reinterpret_cast<XYZZ<F>*>(L.part);
  const uint32_t at = p.tune.accum_threads;
  const int lanes = p.lanes == 4 ? 4 : 1;
  // the folds run on quads whatever the accumulation uses: after a balanced accumulation
  // they only see a few partial sums per bucket (or few, large buckets), so they are
  // latency-bound, and a quad's addition has a third of a lone thread's latency
  const int flanes = 4;
  unsigned qb = (unsigned)((uint64_t(L.qmax) * lanes + at - 1) / at);
  unsigned fb = (unsigned)((uint64_t(L.qmax) * flanes + 127) / 128);
  if (accum_stage >= 0) prof_mark(accum_stage, true, st);
  const auto* ob = reinterpret_cast<const Affine<F>* const*>(L.obases);
  if (lanes == 4)
    k_accum0<F, 4><<<qb, at, 0, st>>>(L.sorted, L.offs, K, T0, bases, ob, p.key_shift, part);
  else
    k_accum0<F, 1><<<qb, at, 0, st>>>(L.sorted, L.offs, K, T0, bases, ob, p.key_shift, part);
  ZK_COUNT_LAUNCH();
  if (accum_stage >= 0) {
    prof_mark(accum_stage, false, st);
    if (uint32_t* hu = prof_units(accum_stage)) ZK_CUDA(cudaMemcpyAsync(hu, L.offs + K, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  }
  ZK_CUDA(cudaGetLastError());
  if (after_accum) ZK_CUDA(cudaEventRecord(after_accum, st));
  // chunk boundaries 1 .. chunks - 1 index the fold list (chunks <= slots / T0 + 1)
  const uint64_t nlist = p.slots / T0 + 2;
  const bool by_boundary = nlist < K;
  const uint32_t* fl = by_boundary ? L.flist : nullptr;
  const uint64_t n_serial = by_boundary ? nlist : uint64_t(K);
  const unsigned sfb = (unsigned)((n_serial * flanes + 127) / 128);
  const unsigned fab = std::max(sfb, fb);
  if (flanes == 4)
    k_fold<F, 4><<<fab, 128, 0, st>>>(L.choff, L.nch, L.chunk_key, K, part, L.arrive, fl, (uint32_t)nlist, L.offs, T0,
                                      (uint32_t)n_serial);
  else
    k_fold<F, 1><<<fab, 128, 0, st>>>(L.choff, L.nch, L.chunk_key, K, part, L.arrive, fl, (uint32_t)nlist, L.offs, T0,
                                      (uint32_t)n_serial);
  ZK_COUNT_LAUNCH();
  // sum_v v B_v per (output, window) by bit decomposition
  XYZZ<F>* Sl = reinterpret_cast<XYZZ<F>*>(L.S);
  XYZZ<F>* D = reinterpret_cast<XYZZ<F>*>(L.D);
  XYZZ<F>* Pb = reinterpret_cast<XYZZ<F>*>(L.P);
  if (L.ngather) {
    k_split_gather<F><<<L.ngather, SliceBT<F>::value, 0, st>>>(part, L.counts, L.choff, L.swins, L.nswin, Pb);
    ZK_COUNT_LAUNCH();
  }
  const size_t nbits = h.bsegs.size(), nwins = h.dsegs.size(), nouts = h.oitems.size();
  ZK_CUDA(cudaMemsetAsync(L.cnt, 0, (nbits + nwins + nouts) * sizeof(uint32_t), st));
  k_bits_chain<F><<<L.nslices, SliceBT<F>::value, 0, st>>>(part, L.counts, L.choff, L.bsegs, L.nbits, L.slice, Pb, Sl, D,
                                                            L.dseg, L.oitems, results, L.cnt, L.cnt + nbits,
                                                            L.cnt + nbits + nwins);
  ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

const uint32_t* msm_term_count(const MsmExec* ex) {
  if (!ex || !ex->st) return nullptr;
  return ex->st->L.offs + ex->plan.keys;
}

template <class F>
int msm_run(const MsmPlan& p, const Affine<F>* bases, void* ws, size_t ws_bytes, XYZZ<F>* results, cudaStream_t st,
            int accum_stage, cudaEvent_t after_accum) {
  MsmExec ex;
  ZK_TRY(msm_prepare<F>(p, ws, ws_bytes, &ex));
  ZK_TRY(msm_upload(&ex, st));
  return msm_launch<F>(&ex, bases, results, st, accum_stage, after_accum);
}

template size_t msm_workspace_bytes<Fp>(const MsmPlan&);
template size_t msm_workspace_bytes<Fp2>(const MsmPlan&);
template int msm_run<Fp>(const MsmPlan&, const Affine<Fp>*, void*, size_t, XYZZ<Fp>*, cudaStream_t, int, cudaEvent_t);
template int msm_run<Fp2>(const MsmPlan&, const Affine<Fp2>*, void*, size_t, XYZZ<Fp2>*, cudaStream_t, int, cudaEvent_t);
template int msm_prepare<Fp>(const MsmPlan&, void*, size_t, MsmExec*);
template int msm_prepare<Fp2>(const MsmPlan&, void*, size_t, MsmExec*);
template int msm_launch<Fp>(const MsmExec*, const Affine<Fp>*, XYZZ<Fp>*, cudaStream_t, int, cudaEvent_t);
template int msm_launch<Fp2>(const MsmExec*, const Affine<Fp2>*, XYZZ<Fp2>*, cudaStream_t, int, cudaEvent_t);

}  // namespace zkvc
