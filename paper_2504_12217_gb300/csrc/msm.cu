// Pippenger multi-scalar multiplication (the A, B, L and H queries of the Groth16
// prover, zkVC Sec. II / IV; the MSMs dominate proving time).
//
// Scalars are recoded into signed c-bit digits d in (-2^(c-1), 2^(c-1)], so a digit
// selects bucket |d| and the sign negates the base's y coordinate.  Every nonzero digit
// becomes one term (bucket key, base index | sign).  Terms are counting-sorted by key
// (histogram, scan, atomic scatter), then each bucket's terms are summed by a
// load-balanced segmented reduction: level 0 gives every chunk of T0 consecutive terms
// of a bucket to one thread (mixed XYZZ + affine additions), and later levels fold T
// partial sums at a time until one remains per bucket, so heavily skewed buckets (int8
// scalars put ~1300 points in each of 128 buckets) cost no more depth than uniform ones.
// A window's result is sum_v v B_v: threads take runs of `sz` buckets (running sums plus
// a short multiplication by the run's offset) and a strided in-place tree adds the runs.
//
// Fixed-base MSMs (proving-key queries) store the multiples 2^(c w) P of each base, so all
// windows share one bucket set and no doubling chain follows; variable-base MSMs keep
// one bucket set per window and combine windows by Horner's rule.
#include <algorithm>

#include "msm.h"

namespace zkvc {

static constexpr uint32_t KEY_NONE = 0xffffffffu;
static constexpr uint32_t T0 = 16;  // terms per level-0 chunk
static constexpr uint32_t TL = 8;   // partial sums folded per later level

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
      k_scan_blocks<<<1, 1024, 0, st>>>(in, n_in, out, n_out, nullptr);
      ZK_CUDA(cudaGetLastError());
    }
    return ZKVC_OK;
  }
  uint32_t* sums = a.take<uint32_t>(blocks);
  uint32_t* sums_x = a.take<uint32_t>(blocks);
  ZK_CHECK(!a.overflow(), ZKVC_EINVAL, "scan: workspace too small");
  if (!a.measuring) {
    k_scan_blocks<<<(unsigned)blocks, 1024, 0, st>>>(in, n_in, out, n_out, sums);
    ZK_CUDA(cudaGetLastError());
  }
  ZK_TRY(scan_rec(sums, blocks, sums_x, blocks, a, st));
  if (!a.measuring) {
    k_scan_add<<<(unsigned)blocks, 1024, 0, st>>>(out, n_out, sums_x);
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
  p.slots = slot;
  p.points = pts;
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

__global__ void k_hist(const uint32_t* keys, uint64_t n, uint32_t* counts) {
  uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t k = keys[i];
  if (k != KEY_NONE) atomicAdd(counts + k, 1u);
}

__global__ void k_scatter(const uint32_t* keys, const uint32_t* vals, uint64_t n, uint32_t* cursor, uint32_t* sorted) {
  uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t k = keys[i];
  if (k == KEY_NONE) return;
  uint32_t pos = atomicAdd(cursor + k, 1u);
  sorted[pos] = vals[i];
}

__global__ void k_chunks(const uint32_t* counts, uint32_t K, uint32_t* nch) {
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
template <class F>
__global__ void __launch_bounds__(256) k_accum0(const uint32_t* __restrict__ sorted, const uint32_t* __restrict__ offs,
                                                const uint32_t* __restrict__ choff, uint32_t K,
                                                const Affine<F>* __restrict__ bases, XYZZ<F>* part) {
  uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= choff[K]) return;
  uint32_t k = find_key(choff, K, q);
  uint32_t j = q - choff[k];
  uint32_t start = offs[k] + j * T0;
  uint32_t end = min(start + T0, offs[k + 1]);
  XYZZ<F> acc = XYZZ<F>::inf();
  for (uint32_t p = start; p < end; p++) {
    uint32_t v = sorted[p];
    Affine<F> P = ld_field(bases + (v & 0x7fffffffu));
    if (v >> 31) P.y = f_neg(P.y);
    acc = p_add_affine(acc, P);
  }
  st_field(part + q, acc);
}

template <class F>
__global__ void __launch_bounds__(256) k_accum_level(const XYZZ<F>* __restrict__ in, XYZZ<F>* out,
                                                     const uint32_t* __restrict__ counts,
                                                     const uint32_t* __restrict__ choff, uint32_t K, uint32_t D) {
  uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= choff[K]) return;
  uint32_t k = find_key(choff, K, q);
  uint32_t j = q - choff[k];
  uint32_t pc = (uint32_t)((uint64_t(counts[k]) + D - 1) / D);  // inputs at this level
  uint32_t np = (pc + TL - 1) / TL;
  if (j >= np) return;
  uint32_t b = choff[k];
  uint32_t s = j * TL, e = min(s + TL, pc);
  XYZZ<F> acc = ld_field(in + b + s);
  for (uint32_t i = s + 1; i < e; i++) acc = p_add(acc, ld_field(in + b + i));
  st_field(out + b + j, acc);
}

template <class F>
__device__ __forceinline__ XYZZ<F> bucket_at(const XYZZ<F>* fin, const uint32_t* counts, const uint32_t* choff,
                                             uint32_t key) {
  if (counts[key] == 0) return XYZZ<F>::inf();
  return ld_field(fin + choff[key]);
}

template <class F>
__device__ __forceinline__ XYZZ<F> p_mul_small(const XYZZ<F>& p, uint32_t k) {
  XYZZ<F> r = XYZZ<F>::inf();
  if (k == 0) return r;
  int top = 31 - __clz(k);
  r = p;
  for (int b = top - 1; b >= 0; b--) {
    r = p_dbl(r);
    if ((k >> b) & 1u) r = p_add(r, p);
  }
  return r;
}

struct GroupItem {  // one run of buckets: output o, window w, buckets [v0, v0 + sz)
  uint32_t key0;    // key of bucket v0
  uint32_t v0;
  uint32_t sz;
};

// R = sum_{v in run} (v - v0 + 1) B_v + (v0 - 1) sum_{v in run} B_v = sum_{v in run} v B_v
template <class F>
__global__ void __launch_bounds__(256) k_bucket_runs(const XYZZ<F>* __restrict__ fin, const uint32_t* __restrict__ counts,
                                                     const uint32_t* __restrict__ choff, const GroupItem* __restrict__ items,
                                                     uint32_t nitems, XYZZ<F>* grp) {
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nitems) return;
  GroupItem it = items[t];
  XYZZ<F> acc = XYZZ<F>::inf(), sum = XYZZ<F>::inf();
  for (int v = (int)it.sz - 1; v >= 0; v--) {
    acc = p_add(acc, bucket_at(fin, counts, choff, it.key0 + (uint32_t)v));
    sum = p_add(sum, acc);
  }
  if (it.v0 > 1) sum = p_add(sum, p_mul_small(acc, it.v0 - 1));
  st_field(grp + t, sum);
}

// In-place strided tree over segments: at level l, element i*2^(l+1) absorbs
// element i*2^(l+1) + 2^l of the same segment.
struct TreeSeg {
  uint32_t off;  // first element
  uint32_t len;  // elements
  uint32_t cum;  // cumulative len/2 rounded up, for the thread mapping
};

template <class F>
__global__ void __launch_bounds__(256) k_tree_level(XYZZ<F>* x, const TreeSeg* segs, uint32_t nseg, uint32_t total,
                                                    uint32_t l) {
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  uint32_t lo = 0, hi = nseg - 1;
  while (lo < hi) {
    uint32_t mid = (lo + hi + 1) >> 1;
    if (segs[mid].cum <= t) lo = mid; else hi = mid - 1;
  }
  TreeSeg s = segs[lo];
  uint32_t i = t - s.cum;
  uint64_t a = uint64_t(i) << (l + 1), b = a + (1ull << l);
  if (b >= s.len) return;
  XYZZ<F> u = ld_field(x + s.off + a), v = ld_field(x + s.off + b);
  st_field(x + s.off + a, p_add(u, v));
}

// results[o] = sum_w 2^(c w) W[o][w] by Horner's rule (windows of variable-base outputs).
struct OutItem {
  uint32_t first;     // index of window 0's tree result in grp
  uint32_t stride;    // distance between windows' tree results
  uint32_t nwin;
  uint32_t c;
};

template <class F>
__global__ void k_combine_windows(const XYZZ<F>* grp, const OutItem* outs, uint32_t nouts, XYZZ<F>* results) {
  uint32_t o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nouts) return;
  OutItem it = outs[o];
  XYZZ<F> acc = ld_field(grp + it.first + (it.nwin - 1) * it.stride);
  for (int w = (int)it.nwin - 2; w >= 0; w--) {
    for (uint32_t i = 0; i < it.c; i++) acc = p_dbl(acc);
    acc = p_add(acc, ld_field(grp + it.first + uint32_t(w) * it.stride));
  }
  st_field(results + o, acc);
}

// ------------------------------------------------------------------ driver
static uint32_t run_size(uint32_t nb) { return nb < 8 ? nb : 8; }

struct Layout {
  uint32_t *keys, *vals, *sorted, *counts, *offs, *cursor, *nch, *choff;
  void *partA, *partB, *grp;
  MsmSeg* segs;
  MsmOut* outs;
  GroupItem* items;
  TreeSeg* tsegs;
  OutItem* oitems;
  uint32_t qmax, nitems, ntseg, ttotal, maxlen;
};

template <class F>
static int layout(const MsmPlan& p, Arena& a, Layout& L, std::vector<GroupItem>* items,
                  std::vector<TreeSeg>* tsegs, std::vector<OutItem>* oitems) {
  const size_t S = p.slots, K = p.keys;
  L.keys = a.take<uint32_t>(S);
  L.vals = a.take<uint32_t>(S);
  L.sorted = a.take<uint32_t>(S);
  L.counts = a.take<uint32_t>(K);
  L.offs = a.take<uint32_t>(K + 1);
  L.cursor = a.take<uint32_t>(K);
  L.nch = a.take<uint32_t>(K);
  L.choff = a.take<uint32_t>(K + 1);
  L.qmax = (uint32_t)(S / T0 + K + 1);
  L.partA = a.take<XYZZ<F>>(L.qmax);
  L.partB = a.take<XYZZ<F>>(L.qmax);
  // bucket runs: one item per run of sz buckets of every (output, window)
  items->clear();
  tsegs->clear();
  oitems->clear();
  uint32_t cum = 0;
  L.maxlen = 1;
  for (const auto& o : p.outs) {
    uint32_t nb = 1u << (o.c - 1);
    uint32_t sz = run_size(nb);
    uint32_t runs = nb / sz;
    OutItem oi{(uint32_t)items->size(), runs, o.win_keys, o.c};
    for (uint32_t w = 0; w < o.win_keys; w++) {
      TreeSeg ts{(uint32_t)items->size(), runs, cum};
      cum += (runs + 1) / 2;
      tsegs->push_back(ts);
      L.maxlen = std::max(L.maxlen, runs);
      for (uint32_t r = 0; r < runs; r++) items->push_back({o.key_off + w * nb + r * sz, r * sz + 1, sz});
    }
    oitems->push_back(oi);
  }
  L.nitems = (uint32_t)items->size();
  L.ntseg = (uint32_t)tsegs->size();
  L.ttotal = cum;
  L.grp = a.take<XYZZ<F>>(L.nitems);
  L.segs = a.take<MsmSeg>(p.segs.size());
  L.outs = a.take<MsmOut>(p.outs.size());
  L.items = a.take<GroupItem>(L.nitems);
  L.tsegs = a.take<TreeSeg>(L.ntseg);
  L.oitems = a.take<OutItem>(p.outs.size());
  return ZKVC_OK;
}

template <class F>
size_t msm_workspace_bytes(const MsmPlan& p) {
  Arena a;
  a.measuring = true;
  Layout L;
  std::vector<GroupItem> items;
  std::vector<TreeSeg> tsegs;
  std::vector<OutItem> oitems;
  layout<F>(p, a, L, &items, &tsegs, &oitems);
  a.off += scan_u32_temp_bytes(p.keys) + scan_u32_temp_bytes(p.keys) + 256;
  return a.off;
}

template <class F>
int msm_run(const MsmPlan& p, const Affine<F>* bases, void* ws, size_t ws_bytes, XYZZ<F>* results, cudaStream_t st) {
  ZK_CHECK(p.keys > 0 && !p.outs.empty(), ZKVC_EINVAL, "msm: empty plan");
  Arena a;
  a.base = reinterpret_cast<uint8_t*>(ws);
  a.cap = ws_bytes;
  Layout L;
  std::vector<GroupItem> items;
  std::vector<TreeSeg> tsegs;
  std::vector<OutItem> oitems;
  layout<F>(p, a, L, &items, &tsegs, &oitems);
  ZK_CHECK(!a.overflow(), ZKVC_EINVAL, "msm: workspace of %zu bytes is too small", ws_bytes);
  const uint32_t K = p.keys;
  const uint64_t S = p.slots;

  ZK_CUDA(cudaMemcpyAsync(L.segs, p.segs.data(), p.segs.size() * sizeof(MsmSeg), cudaMemcpyHostToDevice, st));
  ZK_CUDA(cudaMemcpyAsync(L.outs, p.outs.data(), p.outs.size() * sizeof(MsmOut), cudaMemcpyHostToDevice, st));
  ZK_CUDA(cudaMemcpyAsync(L.items, items.data(), items.size() * sizeof(GroupItem), cudaMemcpyHostToDevice, st));
  ZK_CUDA(cudaMemcpyAsync(L.tsegs, tsegs.data(), tsegs.size() * sizeof(TreeSeg), cudaMemcpyHostToDevice, st));
  ZK_CUDA(cudaMemcpyAsync(L.oitems, oitems.data(), oitems.size() * sizeof(OutItem), cudaMemcpyHostToDevice, st));

  // digits -> terms
  if (p.points > 0) {
    k_digits<<<(p.points + 255) / 256, 256, 0, st>>>(L.segs, (int)p.segs.size(), L.outs, p.points, L.keys, L.vals);
    ZK_CUDA(cudaGetLastError());
  }
  // counting sort by bucket key
  ZK_CUDA(cudaMemsetAsync(L.counts, 0, size_t(K) * sizeof(uint32_t), st));
  unsigned sb = (unsigned)((S + 255) / 256);
  if (S > 0) {
    k_hist<<<sb, 256, 0, st>>>(L.keys, S, L.counts);
    ZK_CUDA(cudaGetLastError());
  }
  ZK_TRY(scan_u32(L.counts, L.offs, K, a, st));
  ZK_CUDA(cudaMemcpyAsync(L.cursor, L.offs, size_t(K) * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
  if (S > 0) {
    k_scatter<<<sb, 256, 0, st>>>(L.keys, L.vals, S, L.cursor, L.sorted);
    ZK_CUDA(cudaGetLastError());
  }
  // chunks of T0 terms per bucket
  k_chunks<<<(K + 255) / 256, 256, 0, st>>>(L.counts, K, L.nch);
  ZK_CUDA(cudaGetLastError());
  ZK_TRY(scan_u32(L.nch, L.choff, K, a, st));
  ZK_CHECK(!a.overflow(), ZKVC_EINVAL, "msm: workspace too small for scans");
  XYZZ<F>* pa = reinterpret_cast<XYZZ<F>*>(L.partA);
  XYZZ<F>* pb = reinterpret_cast<XYZZ<F>*>(L.partB);
  unsigned qb = (L.qmax + 255) / 256;
  k_accum0<F><<<qb, 256, 0, st>>>(L.sorted, L.offs, L.choff, K, bases, pa);
  ZK_CUDA(cudaGetLastError());
  uint64_t D = T0;
  while (D < S) {
    k_accum_level<F><<<qb, 256, 0, st>>>(pa, pb, L.counts, L.choff, K, (uint32_t)D);
    ZK_CUDA(cudaGetLastError());
    std::swap(pa, pb);
    D *= TL;
  }
  // sum_v v B_v per (output, window)
  XYZZ<F>* grp = reinterpret_cast<XYZZ<F>*>(L.grp);
  k_bucket_runs<F><<<(L.nitems + 255) / 256, 256, 0, st>>>(pa, L.counts, L.choff, L.items, L.nitems, grp);
  ZK_CUDA(cudaGetLastError());
  for (uint32_t l = 0; (1u << l) < L.maxlen; l++) {
    k_tree_level<F><<<(L.ttotal + 255) / 256, 256, 0, st>>>(grp, L.tsegs, L.ntseg, L.ttotal, l);
    ZK_CUDA(cudaGetLastError());
  }
  k_combine_windows<F><<<((uint32_t)p.outs.size() + 63) / 64, 64, 0, st>>>(grp, L.oitems, (uint32_t)p.outs.size(), results);
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

template size_t msm_workspace_bytes<Fp>(const MsmPlan&);
template size_t msm_workspace_bytes<Fp2>(const MsmPlan&);
template int msm_run<Fp>(const MsmPlan&, const Affine<Fp>*, void*, size_t, XYZZ<Fp>*, cudaStream_t);
template int msm_run<Fp2>(const MsmPlan&, const Affine<Fp2>*, void*, size_t, XYZZ<Fp2>*, cudaStream_t);

}  // namespace zkvc
