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
// as D = A B^T with A = W^T (M = 128 rows j, K = n) and B = X (N = 64 rows i, K = n), both
// staged as bf16 in shared memory in the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, K-adjacent core matrices 128 bytes apart (leading byte
// offset), 8-row groups 1024 bytes apart (stride byte offset), for K tiles of 64.  One
// thread issues four 128 x 64 x 16 MMAs per K tile and commits them to an mbarrier; the
// accumulator (64 fp32 columns) sits in tensor memory, lane t = row j0 + t, so the
// epilogue stores are coalesced along j.  The int8 -> bf16 conversion runs through
// registers, so no TMA alignment rule applies to X or W.
//
// Every wait (the mbarrier of the MMAs) has a time limit; on expiry the kernel sets bit
// MATMUL_TIMEOUT_FLAG in *flags, waits once more (again bounded) for its MMAs, frees its
// tensor memory and leaves Y unwritten.
#pragma once
#include <cstdint>

namespace zkvc {

constexpr int MM_M = 128, MM_N = 64, MM_BK = 64, MM_KPASS = 256, MM_THREADS = 128;
constexpr int MATMUL_TIMEOUT_FLAG = 8;

struct __align__(1024) MatmulSmem {
  uint8_t a[MM_M * MM_BK * 2];  // W^T tile, bf16
  uint8_t b[MM_N * MM_BK * 2];  // X tile, bf16
  uint64_t bar;
  uint32_t taddr;
  uint8_t pad[8192 - 16];       // caps residency at 7 CTAs per SM (7 x 64 <= 512 TMEM columns)
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

// Y[i0 .. i0+64) x [j0 .. j0+128) of Y = X W; every thread of the CTA calls it.
__device__ __forceinline__ void matmul_tc_tile(const int8_t* __restrict__ X, const int8_t* __restrict__ W,
                                               int32_t* __restrict__ Y, int a, int n, int b, int j0, int i0,
                                               MatmulSmem& sm, int* flags) {
  const int t = threadIdx.x, warp = t >> 5;
  const uint32_t bar = smem_u32(&sm.bar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.taddr)),
                 "r"(MM_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = sm.taddr;
  const uint32_t a_base = smem_u32(sm.a), b_base = smem_u32(sm.b);
  const uint64_t limit = 200ull * 1000 * 1000;  // 200 ms
  int acc[MM_N];
#pragma unroll
  for (int c = 0; c < MM_N; c++) acc[c] = 0;
  uint32_t phase = 0;
  bool ok = true;
  const int j = j0 + t;
  for (int kp = 0; kp < n && ok; kp += MM_KPASS) {
    const int kend = min(n, kp + MM_KPASS);
    for (int k0 = kp; k0 < kend && ok; k0 += MM_BK) {
      // A: thread t owns row j = j0 + t; 8 rows of 8 K values -> one 16-byte core row each
#pragma unroll 2
      for (int kk = 0; kk < MM_BK; kk += 8) {
        int v[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const int k = k0 + kk + q;
          v[q] = (j < b && k < kend) ? (int)W[size_t(k) * b + j] : 0;
        }
        *reinterpret_cast<uint4*>(sm.a + mm_off(t, kk)) =
            make_uint4(bf16x2(v[0], v[1]), bf16x2(v[2], v[3]), bf16x2(v[4], v[5]), bf16x2(v[6], v[7]));
      }
      // B: 64 rows x 64 K; thread t fills row t >> 1, K half (t & 1)
      {
        const int r = t >> 1, i = i0 + r, kh = (t & 1) * 32;
#pragma unroll
        for (int kk = 0; kk < 32; kk += 8) {
          int v[8];
#pragma unroll
          for (int q = 0; q < 8; q++) {
            const int k = k0 + kh + kk + q;
            v[q] = (i < a && k < kend) ? (int)X[size_t(i) * n + k] : 0;
          }
          *reinterpret_cast<uint4*>(sm.b + mm_off(r, kh + kk)) =
              make_uint4(bf16x2(v[0], v[1]), bf16x2(v[2], v[3]), bf16x2(v[4], v[5]), bf16x2(v[6], v[7]));
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (t == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
        for (int s = 0; s < MM_BK / 16; s++) {
          const uint64_t ad = mm_desc(a_base + s * 256), bd = mm_desc(b_base + s * 256);
          const uint32_t accumulate = (k0 > kp || s > 0) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
              "l"(ad), "l"(bd), "r"(MM_IDESC), "r"(accumulate));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                     : "memory");
      }
      // the MMAs have read the tiles (and updated D) before the next fill; the verdict is
      // made uniform so that every thread takes the same path
      ok = __syncthreads_and(mm_wait(bar, phase, limit)) != 0;
      phase ^= 1;
    }
    if (!ok) break;
    // pass done: D holds exact fp32 integers; add them to the int32 sums
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
  if (!ok) {
    if (t == 0) atomicOr(flags, MATMUL_TIMEOUT_FLAG);
    mm_wait(bar, phase ^ 1, limit);  // the last commit, if it is still outstanding
  } else if (j < b) {
#pragma unroll
    for (int c = 0; c < MM_N; c++) {
      const int i = i0 + c;
      if (i < a) Y[size_t(i) * b + j] = acc[c];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(MM_N));
}

}  // namespace zkvc
