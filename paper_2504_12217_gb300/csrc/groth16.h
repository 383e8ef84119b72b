// Proving / verifying key layout of the CRPC + PSQ Groth16 prover (internal).
#pragma once
#include <vector>

#include "curve.cuh"
#include "internal.h"
#include "ntt.h"

// Window widths of the fixed-base MSMs.  The large G1 runs (prefix sums, the H query, the
// s w_v terms over the public inputs) use signed 16-bit digits over bases stored with
// their 16 multiples 2^(16 w) P; the small-scalar and n-point runs use 8-bit digits (int8
// in one digit, int32 in four, full scalars over 32 stored multiples 2^(8 w) P), as does G2.
//
// CRPC structure of the W side (Sec. III-A): the QAP polynomials of W_kj are multiples of
// row k's Lagrange basis, B_(W_kj) = z^j L_k and L_(W_kj) = alpha z^j L_k / delta, so
//   sum_(k,j) w_kj [B_(W_kj)] = sum_k b_k [L_k(tau)],   b_k = sum_j z^j w_kj,
// and likewise for L; the X part of the A query is z^(ib) L_k plus the input row.  The
// prover therefore needs only the n per-row points [L_k(tau)]1,2 and [alpha L_k / delta]1
// (the j = 0 entries of the standard queries) with the full-scalar CRPC values a_k, b_k,
// instead of n b int8 terms per query; the proof is the same group element.  The standard
// queries are kept with one window each for export.
#define ZKVC_C1 16u
#define ZKVC_W1 16u
#define ZKVC_C2 8u
#define ZKVC_W2_FULL 32u

namespace zkvc {

// Regions of the G1 base array, in order.  An entry stores nwin consecutive bases
// 2^(c w) P (w < nwin) so that every window of one MSM shares one bucket set.
enum G1Region : int {
  R1_A = 0,    // A-query, variables v = 0 .. l (export)          l + 1   x1
  R1_ALPHA,    // [alpha]1                                       1       x16
  R1_BETA,     // [beta]1                                        1       x16
  R1_DELTA,    // [delta]1                                       1       x16
  R1_B,        // B-query in G1, W variables (export)            n b     x1
  R1_LW,       // L-query, W variables (export)                  n b     x1
  R1_LS,       // L-query, S variables (prefix sums)             n - 1   x16
  R1_H,        // H-query, bit-reversed positions                N       x16
  R1_AY8,      // A-query, Y variables, 2^(8 w) multiples         a b     x4   (c = 8)
  R1_DELTA8,   // [delta]1, 2^(8 w) multiples                    1       x32  (c = 8)
  R1_AIN,      // input rows [L_(n+v)]1, v = 0 .. l              l + 1   x16
  R1_LK,       // [L_k]1, k < n, 2^(8 w) multiples               n       x32  (c = 8)
  R1_ALK,      // [alpha L_k / delta]1, 2^(8 w) multiples        n       x32  (c = 8)
  R1_COUNT
};

enum G2Region : int {
  R2_B = 0,    // B-query in G2 (export)                         n b     x1
  R2_BETA,     // [beta]2                                        1
  R2_DELTA,    // [delta]2                                       1       x32  (c = 8)
  R2_GAMMA,    // [gamma]2 (verifying key only)                  1
  R2_LK,       // [L_k]2, k < n, 2^(8 w) multiples               n       x32  (c = 8)
  R2_COUNT
};

struct Region {
  uint64_t off;    // first base
  uint32_t count;  // entries
  uint32_t nwin;   // windows per entry
  uint32_t c;      // window bits
  int32_t kind;    // G1Region / G2Region / IC
};

struct Shape {
  int a = 0, n = 0, b = 0;
  uint32_t l = 0;       // public inputs a n + a b
  uint32_t n_vars = 0;  // 1 + l + n b + n - 1
  uint32_t rows = 0;    // n + l + 1
  uint32_t logN = 0;
  size_t N = 0;
};

int make_shape(int a, int n, int b, Shape* s);

struct Layout {
  Region g1[R1_COUNT];
  Region g2[R2_COUNT];
  uint64_t n_g1 = 0, n_g2 = 0;
};

Layout make_layout(const Shape& s);

}  // namespace zkvc

namespace zkvc {
struct GenericKey;
struct ProveGraph;
void prove_graph_free(ProveGraph* g);
}

struct zkvc_pk {
  zkvc::Shape shape;
  zkvc::Layout lay;
  int device = 0;
  zkvc::G1A* g1 = nullptr;   // device, Montgomery affine
  zkvc::G2A* g2 = nullptr;
  zkvc::Fr* zA = nullptr;    // z^(i b), i < a
  zkvc::Fr* zB = nullptr;    // z^j, j < b
  const zkvc::NttDomain* dom = nullptr;
  zkvc::GenericKey* gen = nullptr;  // set for keys of zkvc_setup_circuit (generic R1CS layout)
  // launch shape of the one-proof prover, chosen by zkvc_pk_autotune: terms per level-0
  // chunk of the MSM runs (small, rest, h, g2; 0 = the default rule), log2 of the NTT
  // elements per block (0 = 10), when the side MSM starts (the rest MSM in fold mode, the
  // small-digit MSM in chain mode: 0 at once, 1 after the NTTs, 2 after the H
  // accumulation), zkvc_prove's mode (ZKVC_PROVE_FOLD or _CHAIN), when the G2 MSM starts
  // (0 at once, 1 after the NTTs), quad-lane chunks in the H and small-digit runs (0, 1)
  uint32_t prove_tune[ZKVC_PK_TUNING_LEN] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  // captured one-proof graph of zkvc_prove (prove.cu), created on first use
  mutable zkvc::ProveGraph* graph = nullptr;
};

struct zkvc_vk {
  zkvc::Shape shape;
  int circuit = 0;    // ZKVC_CIRCUIT_*
  int public_io = 0;  // ZKVC_PUBLIC_*: X and Y public, or no public inputs
  // canonical affine encodings (host)
  std::vector<uint8_t> alpha1, beta2, gamma2, delta2;  // 64 / 128 / 128 / 128 bytes
  std::vector<uint8_t> ic;                             // (l + 1) x 64 bytes
};
