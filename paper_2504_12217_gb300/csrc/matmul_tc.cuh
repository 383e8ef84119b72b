// The witness matmul Y = X W (int8 x int8 -> int32, exact) on the 5th-generation tensor
// cores (tcgen05).  The matrix product is the computation zkVC proves (Sec. II, the
// matmul relation; Sec. III-A builds the CRPC constraints on it); here it is the first
// step of the witness.
//
// Exactness: int8 values are exact in bf16 (8 significant bits), a product has
// |x w| <= 2^14, and the tensor core accumulates in fp32 (24 significant bits).  The K
// dimension is taken in passes of at most KPASS = 256 products, so every partial sum is
// an integer of magnitude <= 256 * 2^14 = 2^22 and exact in fp32; after each pass the
// accumulator is read back from tensor memory and added to int32 registers.
//
// Tile: one CTA of 128 threads computes the transpose tile Y^T[j0..j0+128) x [i0..i0+64)
// as D = A B^T with A = W^T (M = 128 rows j) and B = X (N = 64 rows i) over a range of K,
// both staged as bf16 in shared memory in the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, K-adjacent core matrices 128 bytes apart (leading byte
// offset), 8-row groups 1024 bytes apart (stride byte offset), for K tiles of 64.  Two
// stages: while the MMAs of one K tile run, the threads fill the other.  One thread
// issues four 128 x 64 x 16 MMAs per K tile and commits them to the stage's mbarrier; the
// accumulator (64 fp32 columns) sits in tensor memory, lane t = row j0 + t, so the
// epilogue stores are coalesced along j.  Loads are 4 bytes of W (4 columns j) and 16
// bytes of X per thread where the rows are aligned, else single bytes; the int8 -> bf16
// conversion runs through registers, so no TMA alignment rule applies to X or W.  When
// the output grid is small, K is split over CTAs that add their exact int32 partial sums
// into a zeroed Y with atomics.
//
// Every wait (the mbarriers of the MMAs) has a time limit (first_wait_ns, normally
// MATMUL_WAIT_NS; 0 makes the first wait give up at once, to exercise this path); on
// expiry the kernel sets bit MATMUL_TIMEOUT_FLAG in *flags, waits once more for its MMAs
// with the full MATMUL_WAIT_NS limit, frees its tensor memory and leaves its part of Y
// unwritten.
#pragma once
#include <cstdint>

namespace zkvc {

constexpr int MM_M = 128, MM_N = 64, MM_BK = 64, MM_KPASS = 256, MM_THREADS = 128;
constexpr int MATMUL_TIMEOUT_FLAG = 8;
constexpr uint64_t MATMUL_WAIT_NS = 200ull * 1000 * 1000;  // 200 ms

// Dynamic shared memory of a matmul CTA (48 KB of tiles: at most 4 CTAs per SM, so at
// most 4 x 64 of the 512 tensor-memory columns are held at once).
struct MatmulSmem {
  uint8_t a[2][MM_M * MM_BK * 2];  // W^T tiles, bf16
  uint8_t b[2][MM_N * MM_BK * 2];  // X tiles, bf16
  uint64_t bar[2];
  uint32_t taddr;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// canonical K-major, no swizzle: LBO 128 bytes, SBO 1024 bytes, version 1 (bits 46-47)
__device__ __forceinline__ uint64_t mm_desc(uint32_t saddr) {
  return uint64_t((saddr >> 4) & 0x3FFF) | (uint64_t(128 >> 4) << 16) | (uint64_t(1024 >> 4) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: D f32 (bits 4-5 = 1), A and B bf16 (bits 7-9, 10-12
// = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t MM_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(MM_N >> 3) << 17) |
                              (uint32_t(MM_M >> 4) << 24);

// byte offset of element (row r, k) of a K-major canonical tile with MM_BK columns
__device__ __forceinline__ uint32_t mm_off(uint32_t r, uint32_t k) {
  return (((r >> 3) * (MM_BK / 8) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1);
}

__device__ __forceinline__ uint32_t bf16x2(int lo, int hi) {
  // int8 values are exact in bf16: the top 16 bits of the fp32 value
  return (__float_as_uint((float)lo) >> 16) | (__float_as_uint((float)hi) & 0xFFFF0000u);
}

// false on timeout
__device__ __forceinline__ bool mm_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = global_ns();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ uint32_t bf16_pair_of_bytes(uint32_t w, int q) {
  // bytes q and q + 1 of w, as int8, to two bf16
  return bf16x2((int)(int8_t)(w >> (8 * q)), (int)(int8_t)(w >> (8 * q + 8)));
}

// Stage a K tile (64 columns from k0, zero beyond kend) of W^T and X into one buffer.
__device__ __forceinline__ void mm_fill(const int8_t* __restrict__ X, const int8_t* __restrict__ W, int a, int n,
                                        int b, int j0, int i0, int k0, int kend, bool vec_w, bool vec_x,
                                        uint8_t* sa, uint8_t* sb) {
  const int t = threadIdx.x;
  {
    // A = W^T: thread t takes columns j .. j+3 (j = j0 + 4 (t & 31)) of K rows 16 (t >> 5) .. +15
    const int j = j0 + 4 * (t & 31), kq = 16 * (t >> 5);
    uint32_t w[16];
#pragma unroll
    for (int r = 0; r < 16; r++) {
      const int k = k0 + kq + r;
      uint32_t v = 0;
      if (k < kend) {
        const int8_t* row = W + size_t(k) * b;
        if (vec_w && j < b) {
          v = *reinterpret_cast<const uint32_t*>(row + j);
        } else {
#pragma unroll
          for (int q = 0; q < 4; q++)
            if (j + q < b) v |= uint32_t(uint8_t(row[j + q])) << (8 * q);
        }
      }
      w[r] = v;
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
#pragma unroll
      for (int h = 0; h < 2; h++) {
        uint32_t e[4];
#pragma unroll
        for (int p = 0; p < 4; p++) {
          const uint32_t lo = w[8 * h + 2 * p] >> (8 * q), hi = w[8 * h + 2 * p + 1] >> (8 * q);
          e[p] = bf16x2((int)(int8_t)lo, (int)(int8_t)hi);
        }
        *reinterpret_cast<uint4*>(sa + mm_off(4 * (t & 31) + q, kq + 8 * h)) = make_uint4(e[0], e[1], e[2], e[3]);
      }
    }
  }
  {
    // B = X: thread t takes row i0 + (t >> 1), K columns 32 (t & 1) .. +31
    const int r = t >> 1, i = i0 + r, kh = 32 * (t & 1);
#pragma unroll
    for (int c = 0; c < 2; c++) {
      const int kb = k0 + kh + 16 * c;
      uint32_t v[4] = {0, 0, 0, 0};
      if (i < a && kb < kend) {
        const int8_t* row = X + size_t(i) * n;
        if (vec_x && kb + 15 < kend) {
          const uint4 q = *reinterpret_cast<const uint4*>(row + kb);
          v[0] = q.x;
          v[1] = q.y;
          v[2] = q.z;
          v[3] = q.w;
        } else {
#pragma unroll
          for (int q = 0; q < 16; q++)
            if (kb + q < kend) v[q >> 2] |= uint32_t(uint8_t(row[kb + q])) << (8 * (q & 3));
        }
      }
#pragma unroll
      for (int hh = 0; hh < 2; hh++) {
        const uint32_t w0 = v[2 * hh], w1 = v[2 * hh + 1];
        *reinterpret_cast<uint4*>(sb + mm_off(r, kh + 16 * c + 8 * hh)) =
            make_uint4(bf16_pair_of_bytes(w0, 0), bf16_pair_of_bytes(w0, 2), bf16_pair_of_bytes(w1, 0),
                       bf16_pair_of_bytes(w1, 2));
      }
    }
  }
}

// Y[i0 .. i0+64) x [j0 .. j0+128) of Y = X W over K in [kb, ke); every thread of the CTA
// calls it.  accumulate_y: add into Y with atomics (K split over CTAs; Y zeroed before).
__device__ __forceinline__ void matmul_tc_tile(const int8_t* __restrict__ X, const int8_t* __restrict__ W,
                                               int32_t* __restrict__ Y, int a, int n, int b, int j0, int i0,
                                               int kb, int ke, bool accumulate_y, MatmulSmem& sm, int* flags,
                                               uint64_t first_wait_ns = MATMUL_WAIT_NS) {
  const int t = threadIdx.x, warp = t >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.taddr)),
                 "r"(MM_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = sm.taddr;
  const uint64_t limit = MATMUL_WAIT_NS;
  const bool vec_w = (b % 4 == 0) && (reinterpret_cast<uintptr_t>(W) % 4 == 0);
  const bool vec_x = (n % 16 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0);
  int acc[MM_N];
#pragma unroll
  for (int c = 0; c < MM_N; c++) acc[c] = 0;
  // every commit to a stage's barrier is waited exactly once, in order: its parity is the
  // count of earlier waits on that barrier
  uint32_t waits[2] = {0, 0};
  bool pending[2] = {false, false};
  bool ok = true;
  auto wait_stage = [&](int s) {
    if (!pending[s] || !ok) return;  // (after a timeout the cleanup below waits for it)
    ok = __syncthreads_and(first_wait_ns != 0 && mm_wait(smem_u32(&sm.bar[s]), waits[s] & 1, first_wait_ns)) != 0;
    if (!ok) return;
    waits[s]++;
    pending[s] = false;
  };
  int it = 0;
  for (int kp = kb; kp < ke && ok; kp += MM_KPASS) {
    const int kend = min(ke, kp + MM_KPASS);
    for (int k0 = kp; k0 < kend && ok; k0 += MM_BK, it++) {
      const int s = it & 1;
      wait_stage(s);  // the MMAs of the tile before last have read this stage
      if (!ok) break;
      mm_fill(X, W, a, n, b, j0, i0, k0, kend, vec_w, vec_x, sm.a[s], sm.b[s]);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (t == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a_base = smem_u32(sm.a[s]), b_base = smem_u32(sm.b[s]);
#pragma unroll
        for (int q = 0; q < MM_BK / 16; q++) {
          const uint64_t ad = mm_desc(a_base + q * 256), bd = mm_desc(b_base + q * 256);
          const uint32_t accumulate = (k0 > kp || q > 0) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
              "l"(ad), "l"(bd), "r"(MM_IDESC), "r"(accumulate));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&sm.bar[s]))
                     : "memory");
      }
      pending[s] = true;
    }
    // pass done: all its MMAs have finished, D holds exact fp32 integers
    wait_stage(it & 1);
    wait_stage((it + 1) & 1);
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
    for (int c0 = 0; c0 < MM_N; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr + (uint32_t(warp * 32) << 16) + uint32_t(c0)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int q = 0; q < 16; q++) acc[c0 + q] += __float2int_rn(__uint_as_float(r[q]));
    }
    // every thread has read D before the next pass overwrites it
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  const int j = j0 + t;
  if (!ok) {
    if (t == 0) atomicOr(flags, MATMUL_TIMEOUT_FLAG);
    for (int s = 0; s < 2; s++)  // commits still outstanding, if any
      if (pending[s]) mm_wait(smem_u32(&sm.bar[s]), waits[s] & 1, limit);
  } else if (j < b) {
#pragma unroll
    for (int c = 0; c < MM_N; c++) {
      const int i = i0 + c;
      if (i < a) {
        if (accumulate_y)
          atomicAdd(Y + size_t(i) * b + j, acc[c]);
        else
          Y[size_t(i) * b + j] = acc[c];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(MM_N));
}

}  // namespace zkvc
