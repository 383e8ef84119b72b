// NTT over Fr: domain tables and pass launchers (internal).
#pragma once
#include "field.cuh"
#include "internal.h"

namespace zkvc {

// Tables of one evaluation domain H = <omega_N>, N = 2^logN, all in Montgomery form and
// resident on the device that built them.  The coset shift is g = 5.
struct NttDomain {
  uint32_t logN = 0;
  size_t N = 0;
  Fr* tw_fwd = nullptr;   // omega^e,  e < N/2
  Fr* tw_inv = nullptr;   // omega^-e, e < N/2
  Fr* g_lo = nullptr;     // g^l,           l < 1024
  Fr* gi_lo = nullptr;    // g^-l
  Fr* g_hi = nullptr;     // g^(1024 h),    h < max(1, N/1024)
  Fr* g_hi_n = nullptr;   // N^-1 g^(1024 h)
  Fr* gi_hi_n = nullptr;  // N^-1 g^-(1024 h)
  Fr* consts = nullptr;   // [0] N^-1, [1] 1/(g^N - 1), [2] omega, [3] omega^-1, [4] g, [5] g^-1
};

enum ScaleMode : int {
  SC_NONE = 0,  // x
  SC_G = 1,     // x g^i
  SC_NG = 2,    // x N^-1 g^i
  SC_NGI = 3,   // x N^-1 g^-i
  SC_N = 4,     // x N^-1
};

// Sets the pass kernels' shared-memory limit (64 KB blocks); call once before capturing
// NTT launches in a graph (the first NTT call does it otherwise).
int ntt_init();

// Cached per (device, logN); built on first use (allocates; do not call under capture).
int ntt_domain(uint32_t logN, const NttDomain** out);

// Decimation-in-frequency: natural-order input, bit-reversed output, in place.
//   load_scale  multiplies input i (natural index) before the first stage;
//   store_scale multiplies output position p by the factor of natural index bitrev(p).
//   to_mont     converts canonical input to Montgomery form on load.
// batch arrays of N elements each, batch_stride elements apart.  elog = log2 of the
// elements a block stages in shared memory (8 .. 11; passes take min(elog, 10) stages).
int ntt_dif(Fr* data, int batch, size_t batch_stride, const NttDomain* d, bool inverse, int load_scale,
            int store_scale, bool to_mont, cudaStream_t st, int elog = 10);

// Decimation-in-time: bit-reversed input, natural-order output, in place.
int ntt_dit(Fr* data, int batch, size_t batch_stride, const NttDomain* d, bool inverse, cudaStream_t st,
            int elog = 10);

// In-place bit-reversal permutation with an optional scale by natural index and an
// optional conversion out of Montgomery form.
int ntt_bitrev(Fr* data, const NttDomain* d, int scale, bool from_mont, cudaStream_t st);

// The prover's quotient chain for m instances of one domain: ev holds the arrays A_0 ..
// A_(m-1), B_0 .., C_0 .., H_0 .. (N_stride elements apart) with A, B, C the evaluations
// on H (natural order); on return H_i holds the coefficients of h_i = (A_i B_i - C_i) / t
// (bit-reversed order), computed as INTT, coset NTT, pointwise quotient, coset INTT with
// the turns between transforms fused into single passes.  A, B, C are overwritten.
int ntt_quotient_chain(Fr* ev, int m, size_t N_stride, const NttDomain* d, cudaStream_t st, int elog = 10);

// h_ev[i] = (A[i] B[i] - C[i]) / (g^N - 1): the quotient on the coset gH, for i < count
// (count = 0: N; several instances of one domain lie back to back).
int ntt_quotient(const Fr* A, const Fr* B, const Fr* C, Fr* H, const NttDomain* d, cudaStream_t st,
                 size_t count = 0);

}  // namespace zkvc
