// Generic sparse-R1CS Groth16 (zkVC Sec. II Gen / Prove) for the circuit variants of the
// paper's ablation (Sec. V, Table II) and the private-input mode:
//
//   ZKVC_CIRCUIT_CRPC_PSQ  CRPC rows (Sec. III-A) with the PSQ chain (Sec. III-B)
//   ZKVC_CIRCUIT_CRPC      CRPC rows with product variables and one summing row
//   ZKVC_CIRCUIT_PSQ       per output y_ij a prefix-sum chain over its n products
//   ZKVC_CIRCUIT_VANILLA   one row per product x_ik w_kj = p_ijk, one summing row per y_ij
//   ZKVC_CIRCUIT_SOFTMAX   CRPC + PSQ, then the Sec. III-C SoftMax gadgets on each row of Y
//                          (max verification, exponential by clipping and squaring)
//   ZKVC_CIRCUIT_GELU      CRPC + PSQ, then the Sec. III-C GELU polynomial on every entry
//
// with X and Y public (ZKVC_PUBLIC_XY) or private (ZKVC_PUBLIC_NONE).  The rows are built on
// the host in the same order and with the same variable numbering as the specialised
// CRPC + PSQ prover (one | X | Y | W | auxiliary; input-consistency rows last), stored on
// the device by rows (the prover's domain evaluations) and by columns (setup's per-variable
// sums).  Coefficients are indices into a small table: 1, -1, the CRPC powers z^e and,
// for the gadget circuits, signed powers of two and three gadget constants.
//
// Setup evaluates L_k(tau) for every row, sums A_v(tau), B_v(tau), C_v(tau) per variable
// over its column, and turns the query scalars into fixed-base points with the windows the
// prover's MSMs read.  Prove computes the witness (Y, then the circuit's auxiliary
// variables on the device), the domain evaluations by a sparse matrix-vector product over
// Fr (a thread per row, a block per long row), the quotient through the same NTT chain as
// the specialised prover, and the chain-mode MSMs (A, the private part of C and B1 in one
// run; H; B in G2; then s A and r B1 by variable-base multiplication).
#include <algorithm>
#include <cstring>
#include <vector>

#include "circuit.h"
#include "glv.h"
#include "msm.h"
#include "setup_common.h"
#include "witness.cuh"

namespace zkvc {

// kernels of the specialised prover reused here (defined in prove.cu)
__global__ void k_crpc_ab(const int8_t* X, const int8_t* W, const Fr* zA, const Fr* zB, int a, int n, int b, Fr* ak,
                          Fr* bk);
__global__ void k_crpc_y(const int32_t* Y, const Fr* zA, const Fr* zB, int b, Fr* part);
__global__ void k_psq(const Fr* ak, const Fr* bk, const Fr* ypart, int a, int n, Fr* S, Fr* Aev, Fr* Bev, Fr* Cev,
                      int* flags);
__global__ void k_randomness(Fr* rs, int* flags);
__global__ void k_check_h(const Fr* H, size_t N, int* flags);
__global__ void k_chains(const GlvScalar* gs, const G1J* small, G1J* chain, G1J* cpart, uint8_t* proof);

static constexpr uint32_t COEF_ONE = 0, COEF_NEG = 1, COEF_Z0 = 2;
static constexpr uint32_t LONG_ROW = 64;
static constexpr uint32_t C1 = 16, C2 = 8;

// Sec. III-C gadgets on Y as fixed point with GF fractional bits: d = x_max - y in GD
// bits, u = |T| - d + 2^32 in GU bits (top bit: d <= |T|), base beta = c (2^GF - d / 2^GM),
// GM squarings.  Per entry: GD + GU bits, beta, GM powers.
static constexpr uint32_t GF = ZKVC_GADGET_FRAC_BITS, GM = ZKVC_GADGET_EXP_SQUARINGS;
static constexpr uint64_t GT = 1ull << (GF + GM);
static constexpr uint32_t GD = 32, GU = 33;
static constexpr uint32_t G_PER_ENTRY = GD + GU + 1 + GM;
static constexpr uint32_t G_ROWS_PER_ENTRY = GD + 1 + GU + 1 + 1 + GM;

static bool is_gadget(int circuit) { return circuit == ZKVC_CIRCUIT_SOFTMAX || circuit == ZKVC_CIRCUIT_GELU; }
static bool uses_crpc(int circuit) {
  return circuit == ZKVC_CIRCUIT_CRPC_PSQ || circuit == ZKVC_CIRCUIT_CRPC || is_gadget(circuit);
}
__host__ __device__ static inline uint64_t softmax_row_aux(uint64_t b) { return 1 + (b > 2 ? b - 2 : 0) + b * G_PER_ENTRY; }

// Coefficient table: 1, -1, z^0 .. z^(nz-1); for the gadget circuits then 2^0 .. 2^GU-1
// (pow2), -2^0 .. -2^(GD-GM-1) (npow2) and -(|T| + 2^32), -2^(GF+1), -2^(2GF+2) (consts).
struct CoefLayout {
  uint32_t nz = 0, pow2 = 0, npow2 = 0, consts = 0, total = 0;
};

static CoefLayout coef_layout(const GShape& s) {
  CoefLayout L;
  L.nz = uses_crpc(s.circuit) ? (uint32_t)(uint64_t(s.a) * s.b) : 0u;
  L.total = COEF_Z0 + L.nz;
  if (is_gadget(s.circuit)) {
    L.pow2 = L.total;
    L.npow2 = L.pow2 + GU;
    L.consts = L.npow2 + (GD - GM);
    L.total = L.consts + 3;
  }
  return L;
}

GenericKey::~GenericKey() {
  for (auto& c : csr) {
    cudaFree(c.rowptr);
    cudaFree(c.col);
    cudaFree(c.coef);
  }
  cudaFree(coef_tab);
  cudaFree(long_rows);
}

static uint32_t windows_for(int kind, uint32_t c) {
  switch (kind) {
    case SK_ONE: return 1;
    case SK_I8: return c >= 8 ? 1 : (8 + c) / c;
    case SK_I16: return c >= 16 ? 1 : (16 + c) / c;
    case SK_I32: return (32 + c - 1) / c;
    default: return (255 + c - 1) / c;
  }
}

int make_gshape(int a, int n, int b, int circuit, int pub, GShape* s) {
  ZK_CHECK(a >= 1 && n >= 1 && b >= 1, ZKVC_EINVAL, "shape (%d, %d, %d): every dimension must be >= 1", a, n, b);
  ZK_CHECK(circuit >= ZKVC_CIRCUIT_CRPC_PSQ && circuit <= ZKVC_CIRCUIT_GELU, ZKVC_EINVAL, "circuit %d", circuit);
  ZK_CHECK(pub == ZKVC_PUBLIC_XY || pub == ZKVC_PUBLIC_NONE, ZKVC_EINVAL, "public-input mode %d", pub);
  const uint64_t A = a, Nn = n, B = b;
  GShape g;
  g.a = a;
  g.n = n;
  g.b = b;
  g.circuit = circuit;
  g.pub = pub;
  g.n_io = A * Nn + A * B;
  g.l = pub == ZKVC_PUBLIC_XY ? g.n_io : 0;
  int aux_kind = SK_FR_MONT;
  switch (circuit) {
    case ZKVC_CIRCUIT_CRPC_PSQ: g.n_aux = Nn - 1; g.n_crows = Nn; break;
    case ZKVC_CIRCUIT_CRPC: g.n_aux = Nn; g.n_crows = Nn + 1; break;
    case ZKVC_CIRCUIT_PSQ: g.n_aux = A * B * (Nn - 1); g.n_crows = A * B * Nn; aux_kind = SK_I32; break;
    case ZKVC_CIRCUIT_SOFTMAX:
      g.n_aux = Nn - 1 + A * softmax_row_aux(B);
      g.n_crows = Nn + A * (B * G_ROWS_PER_ENTRY + (B > 1 ? B - 1 : 1));
      break;
    case ZKVC_CIRCUIT_GELU: g.n_aux = Nn - 1 + A * B; g.n_crows = Nn + A * B; break;
    default: g.n_aux = A * B * Nn; g.n_crows = A * B * Nn + A * B; aux_kind = SK_I16; break;
  }
  g.n_vars = 1 + g.n_io + Nn * B + g.n_aux;
  g.n_rows = g.n_crows + g.l + 1;
  ZK_CHECK(g.n_rows <= (1ull << 26) && g.n_vars < (1ull << 30), ZKVC_EINVAL,
           "circuit %d of shape (%d, %d, %d) has %llu rows / %llu variables: too large", circuit, a, n, b,
           (unsigned long long)g.n_rows, (unsigned long long)g.n_vars);
  g.logN = ceil_log2(g.n_rows);
  if (g.logN < 1) g.logN = 1;
  g.N = size_t(1) << g.logN;
  const uint64_t cnt[G_COUNT] = {1, A * Nn, A * B, Nn * B, g.n_aux};
  const int kinds[G_COUNT] = {SK_ONE, SK_I8, SK_I32, SK_I8, aux_kind};
  uint64_t f = 0;
  for (int i = 0; i < G_COUNT; i++) {
    g.first[i] = f;
    g.count[i] = cnt[i];
    g.kind[i] = kinds[i];
    f += cnt[i];
  }
  *s = g;
  return ZKVC_OK;
}

// ------------------------------------------------------------------ host rows
struct HostMat {
  std::vector<uint64_t> rowptr;
  std::vector<uint32_t> col, coef;
};

struct HostR1cs {
  HostMat m[3];
  void row() {
    for (auto& x : m) x.rowptr.push_back(x.col.size());
  }
  void add(int mi, uint64_t var, uint32_t c) {
    m[mi].col.push_back((uint32_t)var);
    m[mi].coef.push_back(c);
  }
  void finish() {
    for (auto& x : m) x.rowptr.push_back(x.col.size());
  }
};

// Rows of the Sec. III-C gadgets over Y; the gadget's auxiliary block starts at aux0.
// SoftMax, per row i of Y (block: x_max, P_1 .. P_(b-2), then per entry the GD bits of d,
// the GU bits of u, beta, the GM powers): per entry the bit rows b * b = b and the
// recomposition of d = x_max - y, the same for u = |T| - d + 2^32, beta = c (2^GF - q)
// with c the top bit of u and q the bits of d from GM up, e_t = e_(t-1)^2; then the chain
// (x_max - y_0)(x_max - y_1) = P_1, P_(j-1) (x_max - y_j) = P_j, closing at 0.  GELU: per
// entry y * y = G - 2^(GF+1) y - 2^(2GF+2).
template <class YV>
static void gadget_rows(const GShape& s, YV Yv, uint64_t aux0, HostR1cs& R) {
  const uint64_t a = s.a, b = s.b;
  const CoefLayout L = coef_layout(s);
  if (s.circuit == ZKVC_CIRCUIT_GELU) {
    for (uint64_t i = 0; i < a; i++)
      for (uint64_t j = 0; j < b; j++) {
        const uint64_t y = Yv(i, j);
        R.row();
        R.add(0, y, COEF_ONE);
        R.add(1, y, COEF_ONE);
        R.add(2, aux0 + i * b + j, COEF_ONE);
        R.add(2, y, L.consts + 1);
        R.add(2, 0, L.consts + 2);
      }
    return;
  }
  const uint64_t per_row = softmax_row_aux(b), nprod = b > 2 ? b - 2 : 0;
  for (uint64_t i = 0; i < a; i++) {
    const uint64_t mx = aux0 + i * per_row, p1 = mx + 1, ent0 = mx + 1 + nprod;
    for (uint64_t j = 0; j < b; j++) {
      const uint64_t y = Yv(i, j), e0 = ent0 + j * G_PER_ENTRY;
      for (uint32_t k = 0; k < GD; k++) {
        R.row();
        R.add(0, e0 + k, COEF_ONE);
        R.add(1, e0 + k, COEF_ONE);
        R.add(2, e0 + k, COEF_ONE);
      }
      R.row();  // sum 2^k d_k - x_max + y = 0
      for (uint32_t k = 0; k < GD; k++) R.add(0, e0 + k, L.pow2 + k);
      R.add(0, mx, COEF_NEG);
      R.add(0, y, COEF_ONE);
      R.add(1, 0, COEF_ONE);
      const uint64_t u0 = e0 + GD;
      for (uint32_t k = 0; k < GU; k++) {
        R.row();
        R.add(0, u0 + k, COEF_ONE);
        R.add(1, u0 + k, COEF_ONE);
        R.add(2, u0 + k, COEF_ONE);
      }
      R.row();  // sum 2^k u_k - (|T| + 2^32) + x_max - y = 0
      for (uint32_t k = 0; k < GU; k++) R.add(0, u0 + k, L.pow2 + k);
      R.add(0, 0, L.consts);
      R.add(0, mx, COEF_ONE);
      R.add(0, y, COEF_NEG);
      R.add(1, 0, COEF_ONE);
      const uint64_t beta = u0 + GU;
      R.row();  // c * (2^GF - q) = beta
      R.add(0, u0 + GU - 1, COEF_ONE);
      R.add(1, 0, L.pow2 + GF);
      for (uint32_t k = GM; k < GD; k++) R.add(1, e0 + k, L.npow2 + (k - GM));
      R.add(2, beta, COEF_ONE);
      uint64_t prev = beta;
      for (uint32_t t = 0; t < GM; t++) {  // e_t = e_(t-1)^2
        R.row();
        R.add(0, prev, COEF_ONE);
        R.add(1, prev, COEF_ONE);
        R.add(2, beta + 1 + t, COEF_ONE);
        prev = beta + 1 + t;
      }
    }
    if (b == 1) {  // (x_max - y_0) * 1 = 0
      R.row();
      R.add(0, mx, COEF_ONE);
      R.add(0, Yv(i, 0), COEF_NEG);
      R.add(1, 0, COEF_ONE);
    } else {
      for (uint64_t j = 1; j < b; j++) {
        R.row();
        if (j == 1) {
          R.add(0, mx, COEF_ONE);
          R.add(0, Yv(i, 0), COEF_NEG);
        } else {
          R.add(0, p1 + (j - 2), COEF_ONE);
        }
        R.add(1, mx, COEF_ONE);
        R.add(1, Yv(i, j), COEF_NEG);
        if (j + 1 < b) R.add(2, p1 + (j - 1), COEF_ONE);
      }
    }
  }
}

// The rows of the circuit, in the order of the oracle's definition.
static void build_rows(const GShape& s, HostR1cs& R) {
  const uint64_t a = s.a, n = s.n, b = s.b, an = a * n;
  auto X = [&](uint64_t i, uint64_t k) { return 1 + i * n + k; };
  auto Yv = [&](uint64_t i, uint64_t j) { return 1 + an + i * b + j; };
  auto Wv = [&](uint64_t k, uint64_t j) { return 1 + s.n_io + k * b + j; };
  auto AUX = [&](uint64_t t) { return 1 + s.n_io + n * b + t; };
  for (auto& x : R.m) x.rowptr.reserve(s.n_rows + 1);
  if (uses_crpc(s.circuit)) {
    for (uint64_t k = 0; k < n; k++) {
      R.row();
      for (uint64_t i = 0; i < a; i++) R.add(0, X(i, k), COEF_Z0 + (uint32_t)(i * b));
      for (uint64_t j = 0; j < b; j++) R.add(1, Wv(k, j), COEF_Z0 + (uint32_t)j);
      if (s.circuit == ZKVC_CIRCUIT_CRPC) {
        R.add(2, AUX(k), COEF_ONE);
      } else if (k + 1 < n) {
        R.add(2, AUX(k), COEF_ONE);
        if (k >= 1) R.add(2, AUX(k - 1), COEF_NEG);
      } else {
        for (uint64_t i = 0; i < a; i++)
          for (uint64_t j = 0; j < b; j++) R.add(2, Yv(i, j), COEF_Z0 + (uint32_t)(i * b + j));
        if (n >= 2) R.add(2, AUX(n - 2), COEF_NEG);
      }
    }
    if (s.circuit == ZKVC_CIRCUIT_CRPC) {  // (p_0 + ... + p_(n-1)) * 1 = Y(z)
      R.row();
      for (uint64_t k = 0; k < n; k++) R.add(0, AUX(k), COEF_ONE);
      R.add(1, 0, COEF_ONE);
      for (uint64_t i = 0; i < a; i++)
        for (uint64_t j = 0; j < b; j++) R.add(2, Yv(i, j), COEF_Z0 + (uint32_t)(i * b + j));
    }
    if (is_gadget(s.circuit)) gadget_rows(s, Yv, AUX(n - 1), R);
  } else {
    const bool van = s.circuit == ZKVC_CIRCUIT_VANILLA;
    for (uint64_t i = 0; i < a; i++)
      for (uint64_t j = 0; j < b; j++)
        for (uint64_t k = 0; k < n; k++) {
          R.row();
          R.add(0, X(i, k), COEF_ONE);
          R.add(1, Wv(k, j), COEF_ONE);
          if (van) {
            R.add(2, AUX((i * b + j) * n + k), COEF_ONE);
          } else {
            if (k + 1 < n)
              R.add(2, AUX((i * b + j) * (n - 1) + k), COEF_ONE);
            else
              R.add(2, Yv(i, j), COEF_ONE);
            if (k >= 1) R.add(2, AUX((i * b + j) * (n - 1) + k - 1), COEF_NEG);
          }
        }
    if (van)
      for (uint64_t i = 0; i < a; i++)
        for (uint64_t j = 0; j < b; j++) {  // (p_ij0 + ... + p_ij(n-1)) * 1 = y_ij
          R.row();
          for (uint64_t k = 0; k < n; k++) R.add(0, AUX((i * b + j) * n + k), COEF_ONE);
          R.add(1, 0, COEF_ONE);
          R.add(2, Yv(i, j), COEF_ONE);
        }
  }
  for (uint64_t v = 0; v <= s.l; v++) {  // input-consistency rows
    R.row();
    R.add(0, v, COEF_ONE);
  }
  R.finish();
}

// by-column copy of one matrix: colptr over variables, (row, coef) entries
struct HostCsc {
  std::vector<uint64_t> colptr;
  std::vector<uint32_t> row, coef;
};

static void to_csc(const HostMat& m, uint64_t n_vars, HostCsc& c) {
  c.colptr.assign(n_vars + 1, 0);
  for (uint32_t v : m.col) c.colptr[v + 1]++;
  for (uint64_t v = 0; v < n_vars; v++) c.colptr[v + 1] += c.colptr[v];
  c.row.resize(m.col.size());
  c.coef.resize(m.col.size());
  std::vector<uint64_t> cur(c.colptr.begin(), c.colptr.end() - 1);
  const uint64_t rows = m.rowptr.size() - 1;
  for (uint64_t r = 0; r < rows; r++)
    for (uint64_t e = m.rowptr[r]; e < m.rowptr[r + 1]; e++) {
      uint64_t at = cur[m.col[e]]++;
      c.row[at] = (uint32_t)r;
      c.coef[at] = m.coef[e];
    }
}

template <class T>
static int upload(const std::vector<T>& h, T** d, cudaStream_t st) {
  size_t bytes = std::max<size_t>(1, h.size()) * sizeof(T);
  if (cudaMalloc(d, bytes) != cudaSuccess) {
    cudaGetLastError();
    *d = nullptr;
    set_error("setup: cannot allocate %zu bytes for the constraint matrices", bytes);
    return ZKVC_ENOMEM;
  }
  if (!h.empty()) ZK_CUDA(cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return ZKVC_OK;
}

// ------------------------------------------------------------------ setup kernels
// 2^k in Montgomery form (k < 64)
__device__ Fr fr_pow2(uint32_t k) {
  Fr x = Fr::zero();
  x.v[k >> 5] = 1u << (k & 31);
  return f_to_mont(x);
}

__global__ void k_gen_coef_tab(const SetupConsts* sc, Fr* tab, CoefLayout L) {
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L.total) return;
  Fr v;
  if (t == COEF_ONE)
    v = Fr::one();
  else if (t == COEF_NEG)
    v = f_neg(Fr::one());
  else if (t < COEF_Z0 + L.nz)
    v = pow_u32(sc->z, t - COEF_Z0);
  else if (t < L.npow2)
    v = fr_pow2(t - L.pow2);
  else if (t < L.consts)
    v = f_neg(fr_pow2(t - L.npow2));
  else if (t == L.consts)
    v = f_neg(f_add(fr_pow2(GF + GM), fr_pow2(GD)));
  else if (t == L.consts + 1)
    v = f_neg(fr_pow2(GF + 1));
  else
    v = f_neg(fr_pow2(2 * GF + 2));
  st_field(tab + t, v);
}

// out[v] = sum over the column of v of coef * L_row
__global__ void k_gen_colsums(const uint64_t* __restrict__ colptr, const uint32_t* __restrict__ row,
                              const uint32_t* __restrict__ coef, const Fr* __restrict__ tab, const Fr* __restrict__ L,
                              uint64_t n_vars, Fr* out) {
  uint64_t v = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= n_vars) return;
  Fr acc = Fr::zero();
  for (uint64_t e = colptr[v]; e < colptr[v + 1]; e++) {
    uint32_t c = coef[e];
    Fr Lr = ld_field(L + row[e]);
    if (c == COEF_ONE)
      acc = f_add(acc, Lr);
    else if (c == COEF_NEG)
      acc = f_sub(acc, Lr);
    else
      acc = f_add(acc, f_mul(ld_field(tab + c), Lr));
  }
  st_field(out + v, acc);
}

enum : int { J_A = 0, J_B, J_L, J_IC, J_H, J_ALPHA, J_BETA, J_DELTA, J_GAMMA };

struct Job {
  int type;
  uint32_t nwin, c;
  uint64_t first_var;  // first variable (A, B, L, IC)
  uint64_t count;
  uint64_t off;        // first output scalar
  uint64_t entry0;     // cumulative entries before this job
};

static constexpr int MAX_JOBS = 24;
struct JobTab {
  Job j[MAX_JOBS];
  int n;
  uint64_t total;
};

__global__ void k_gen_scalars(JobTab tab, const SetupConsts* __restrict__ scp, const Fr* __restrict__ At,
                              const Fr* __restrict__ Bt, const Fr* __restrict__ Ct, uint32_t logN, Fr* out) {
  uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= tab.total) return;
  int ji = 0;
  while (ji + 1 < tab.n && tab.j[ji + 1].entry0 <= t) ji++;
  const Job jb = tab.j[ji];
  const uint64_t e = t - jb.entry0;
  const uint64_t v = jb.first_var + e;
  const SetupConsts& sc = *scp;
  Fr s = Fr::zero();
  switch (jb.type) {
    case J_A: s = ld_field(At + v); break;
    case J_B: s = ld_field(Bt + v); break;
    case J_L:
    case J_IC: {
      Fr q = f_add(f_add(f_mul(sc.beta, ld_field(At + v)), f_mul(sc.alpha, ld_field(Bt + v))), ld_field(Ct + v));
      s = f_mul(q, jb.type == J_L ? sc.dinv : sc.ginv);
      break;
    }
    case J_H: {
      uint32_t j = bitrev_n((uint32_t)e, logN);
      if (j + 1 < (1u << logN)) s = f_mul(pow_u32(sc.tau, j), f_mul(sc.tN1, sc.dinv));
      break;
    }
    case J_ALPHA: s = sc.alpha; break;
    case J_BETA: s = sc.beta; break;
    case J_DELTA: s = sc.delta; break;
    default: s = sc.gamma; break;
  }
  Fr step = f_from_int<FrCfg>((int32_t)(1u << jb.c));
  uint64_t base = jb.off + e * jb.nwin;
  for (uint32_t w = 0; w < jb.nwin; w++) {
    st_field(out + base + w, s);
    s = f_mul(s, step);
  }
}

static void add_job(JobTab& t, int type, const GRegion& r, uint64_t first_var) {
  if (r.count == 0) return;
  Job j{};
  j.type = type;
  j.nwin = r.nwin;
  j.c = r.c;
  j.first_var = first_var;
  j.count = r.count;
  j.off = r.off;
  j.entry0 = t.total;
  t.j[t.n++] = j;
  t.total += r.count;
}

static GRegion take(uint64_t& off, uint64_t count, uint32_t nwin, uint32_t c) {
  GRegion r;
  r.off = off;
  r.count = count;
  r.nwin = nwin;
  r.c = c;
  off += count * nwin;
  return r;
}

int setup_generic(int a, int n, int b, int circuit, int pub, const uint8_t* toxic, cudaStream_t st, zkvc_pk** pk_out,
                  zkvc_vk** vk_out) {
  GShape sh;
  ZK_TRY(make_gshape(a, n, b, circuit, pub, &sh));
  const NttDomain* dom = nullptr;
  ZK_TRY(ntt_domain(sh.logN, &dom));
  ZK_TRY(ntt_init());
  G1A* T1 = nullptr;
  G2A* T2 = nullptr;
  ZK_TRY(fb_tables(&T1, &T2, st));

  DevTemps tmp;
  Fr* d_toxic = nullptr;
  SetupConsts* d_sc = nullptr;
  ZK_TRY(tmp.alloc(&d_toxic, 6));
  ZK_TRY(tmp.alloc(&d_sc, 1));
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

  // rows on the host; by-row copy kept in the key, by-column copy for the sums below
  HostR1cs R;
  build_rows(sh, R);
  ZK_CHECK(R.m[0].rowptr.size() == sh.n_rows + 1, ZKVC_EINVAL, "setup: row count mismatch");
  bool support[3][G_COUNT] = {};
  HostCsc csc[3];
  for (int mi = 0; mi < 3; mi++) {
    to_csc(R.m[mi], sh.n_vars, csc[mi]);
    for (int g = 0; g < G_COUNT; g++)
      support[mi][g] = csc[mi].colptr[sh.first[g] + sh.count[g]] > csc[mi].colptr[sh.first[g]];
  }
  std::vector<uint32_t> long_rows;
  for (uint64_t r = 0; r < sh.n_rows; r++) {
    bool lg = false;
    for (int mi = 0; mi < 3; mi++) lg |= R.m[mi].rowptr[r + 1] - R.m[mi].rowptr[r] > LONG_ROW;
    if (lg) long_rows.push_back((uint32_t)r);
  }

  zkvc_pk* pk = new zkvc_pk();
  GenericKey* G = new GenericKey();
  pk->gen = G;
  G->sh = sh;
  pk->dom = dom;
  pk->shape.a = a;
  pk->shape.n = n;
  pk->shape.b = b;
  pk->shape.l = (uint32_t)sh.l;
  pk->shape.n_vars = (uint32_t)sh.n_vars;
  pk->shape.rows = (uint32_t)sh.n_rows;
  pk->shape.logN = sh.logN;
  pk->shape.N = sh.N;
  ZK_CUDA(cudaGetDevice(&pk->device));
  auto fail = [&](int rc) {
    cudaFree(pk->g1);
    cudaFree(pk->g2);
    cudaFree(pk->zA);
    cudaFree(pk->zB);
    delete pk->gen;
    delete pk;
    return rc;
  };
  // layout: G1 at c = 16, G2 at c = 8
  uint64_t o1 = 0, o2 = 0;
  for (int g = 0; g < G_COUNT; g++) {
    const uint64_t cnt = sh.count[g];
    const int kd = sh.kind[g];
    if (support[0][g] && cnt) G->g1q[GQ_A][g] = take(o1, cnt, windows_for(kd, C1), C1);
    if (support[1][g] && cnt) G->g1q[GQ_B1][g] = take(o1, cnt, windows_for(kd, C1), C1);
    if (sh.first[g] > sh.l && cnt) G->g1q[GQ_L][g] = take(o1, cnt, windows_for(kd, C1), C1);
    if (support[1][g] && cnt) G->B2[g] = take(o2, cnt, windows_for(kd, C2), C2);
  }
  G->H = take(o1, sh.N, windows_for(SK_FR_MONT, C1), C1);
  G->ALPHA = take(o1, 1, 1, C1);
  G->BETA = take(o1, 1, 1, C1);
  G->DELTA = take(o1, 1, windows_for(SK_FR_MONT, C1), C1);
  G->BETA2 = take(o2, 1, 1, C2);
  G->DELTA2 = take(o2, 1, windows_for(SK_FR_MONT, C2), C2);
  G->GAMMA2 = take(o2, 1, 1, C2);
  G->n_g1 = o1;
  G->n_g2 = o2;
  if (o1 >= (1ull << 31) || o2 >= (1ull << 31)) {
    set_error("setup: %llu G1 bases exceed the MSM's 31-bit base index", (unsigned long long)o1);
    return fail(ZKVC_EINVAL);
  }
  pk->lay.n_g1 = o1;
  pk->lay.n_g2 = o2;
  int rc = ZKVC_OK;
  do {
    if (cudaMalloc(&pk->g1, o1 * sizeof(G1A)) != cudaSuccess || cudaMalloc(&pk->g2, o2 * sizeof(G2A)) != cudaSuccess ||
        cudaMalloc(&pk->zA, sh.a * sizeof(Fr)) != cudaSuccess || cudaMalloc(&pk->zB, sh.b * sizeof(Fr)) != cudaSuccess) {
      cudaGetLastError();
      set_error("setup: proving key allocation failed (%llu G1 + %llu G2 bases)", (unsigned long long)o1,
                (unsigned long long)o2);
      rc = ZKVC_ENOMEM;
      break;
    }
    for (int mi = 0; mi < 3 && rc == ZKVC_OK; mi++) {
      Csr& c = G->csr[mi];
      c.nnz = R.m[mi].col.size();
      if ((rc = upload(R.m[mi].rowptr, &c.rowptr, st)) != ZKVC_OK) break;
      if ((rc = upload(R.m[mi].col, &c.col, st)) != ZKVC_OK) break;
      rc = upload(R.m[mi].coef, &c.coef, st);
    }
    if (rc != ZKVC_OK) break;
    G->n_long = (uint32_t)long_rows.size();
    if ((rc = upload(long_rows, &G->long_rows, st)) != ZKVC_OK) break;
    // coefficient table and the CRPC powers used by the witness kernels
    const bool crpc = uses_crpc(circuit);
    const CoefLayout CL = coef_layout(sh);
    G->n_coef = CL.total;
    if (cudaMalloc(&G->coef_tab, G->n_coef * sizeof(Fr)) != cudaSuccess) {
      cudaGetLastError();
      set_error("setup: coefficient table allocation failed");
      rc = ZKVC_ENOMEM;
      break;
    }
    k_gen_coef_tab<<<(G->n_coef + 255) / 256, 256, 0, st>>>(d_sc, G->coef_tab, CL); ZK_COUNT_LAUNCH();
    // zA[i] = z^(ib), zB[j] = z^j are entries of the table
    for (int i = 0; i < a && crpc; i++)
      ZK_CUDA(cudaMemcpyAsync(pk->zA + i, G->coef_tab + COEF_Z0 + size_t(i) * b, sizeof(Fr), cudaMemcpyDeviceToDevice, st));
    if (crpc)
      ZK_CUDA(cudaMemcpyAsync(pk->zB, G->coef_tab + COEF_Z0, size_t(b) * sizeof(Fr), cudaMemcpyDeviceToDevice, st));
    // Lagrange values and per-variable sums
    Fr* d_L = nullptr;
    Fr* At = nullptr;
    if ((rc = tmp.alloc(&d_L, sh.n_rows)) != ZKVC_OK) break;
    if ((rc = tmp.alloc(&At, 3 * sh.n_vars)) != ZKVC_OK) break;
    Fr* Bt = At + sh.n_vars;
    Fr* Ct = Bt + sh.n_vars;
    size_t lag_threads = (sh.n_rows + LAG_CHUNK - 1) / LAG_CHUNK;
    k_lagrange<<<(unsigned)((lag_threads + 127) / 128), 128, 0, st>>>(d_sc, dom->tw_fwd, sh.N, (uint32_t)sh.n_rows, d_L); ZK_COUNT_LAUNCH();
    for (int mi = 0; mi < 3 && rc == ZKVC_OK; mi++) {
      uint64_t* cp = nullptr;
      uint32_t *rw = nullptr, *cf = nullptr;
      if ((rc = tmp.alloc(&cp, csc[mi].colptr.size())) != ZKVC_OK) break;
      if ((rc = tmp.alloc(&rw, std::max<size_t>(1, csc[mi].row.size()))) != ZKVC_OK) break;
      if ((rc = tmp.alloc(&cf, std::max<size_t>(1, csc[mi].coef.size()))) != ZKVC_OK) break;
      ZK_CUDA(cudaMemcpyAsync(cp, csc[mi].colptr.data(), csc[mi].colptr.size() * 8, cudaMemcpyHostToDevice, st));
      if (!csc[mi].row.empty()) {
        ZK_CUDA(cudaMemcpyAsync(rw, csc[mi].row.data(), csc[mi].row.size() * 4, cudaMemcpyHostToDevice, st));
        ZK_CUDA(cudaMemcpyAsync(cf, csc[mi].coef.data(), csc[mi].coef.size() * 4, cudaMemcpyHostToDevice, st));
      }
      k_gen_colsums<<<(unsigned)((sh.n_vars + 255) / 256), 256, 0, st>>>(cp, rw, cf, G->coef_tab, d_L, sh.n_vars,
                                                                         At + mi * sh.n_vars); ZK_COUNT_LAUNCH();
    }
    if (rc != ZKVC_OK) break;
    ZK_CUDA(cudaGetLastError());
    // G1 query scalars and bases
    const size_t chunk = size_t(1) << 20;
    Fr* scal = nullptr;
    XYZZ<Fp2>* xtmp = nullptr;
    if ((rc = tmp.alloc(&scal, std::max<uint64_t>(o1, sh.l + 1))) != ZKVC_OK) break;
    if ((rc = tmp.alloc(&xtmp, chunk)) != ZKVC_OK) break;
    JobTab t1{};
    for (int g = 0; g < G_COUNT; g++) {
      add_job(t1, J_A, G->g1q[GQ_A][g], sh.first[g]);
      add_job(t1, J_B, G->g1q[GQ_B1][g], sh.first[g]);
      add_job(t1, J_L, G->g1q[GQ_L][g], sh.first[g]);
    }
    add_job(t1, J_H, G->H, 0);
    add_job(t1, J_ALPHA, G->ALPHA, 0);
    add_job(t1, J_BETA, G->BETA, 0);
    add_job(t1, J_DELTA, G->DELTA, 0);
    k_gen_scalars<<<(unsigned)((t1.total + 255) / 256), 256, 0, st>>>(t1, d_sc, At, Bt, Ct, sh.logN, scal); ZK_COUNT_LAUNCH();
    if ((rc = points_from_scalars<Fp>(scal, o1, T1, pk->g1, reinterpret_cast<XYZZ<Fp>*>(xtmp), 2 * chunk, st)) != ZKVC_OK)
      break;
    // G2
    JobTab t2{};
    for (int g = 0; g < G_COUNT; g++) add_job(t2, J_B, G->B2[g], sh.first[g]);
    add_job(t2, J_BETA, G->BETA2, 0);
    add_job(t2, J_DELTA, G->DELTA2, 0);
    add_job(t2, J_GAMMA, G->GAMMA2, 0);
    k_gen_scalars<<<(unsigned)((t2.total + 255) / 256), 256, 0, st>>>(t2, d_sc, At, Bt, Ct, sh.logN, scal); ZK_COUNT_LAUNCH();
    if ((rc = points_from_scalars<Fp2>(scal, o2, T2, pk->g2, xtmp, chunk, st)) != ZKVC_OK) break;
    // verifying key: IC_v for v = 0 .. l
    JobTab t3{};
    GRegion ric;
    ric.off = 0;
    ric.count = sh.l + 1;
    ric.nwin = 1;
    ric.c = C1;
    add_job(t3, J_IC, ric, 0);
    G1A* ic = nullptr;
    if ((rc = tmp.alloc(&ic, sh.l + 1)) != ZKVC_OK) break;
    k_gen_scalars<<<(unsigned)((t3.total + 255) / 256), 256, 0, st>>>(t3, d_sc, At, Bt, Ct, sh.logN, scal); ZK_COUNT_LAUNCH();
    if ((rc = points_from_scalars<Fp>(scal, sh.l + 1, T1, ic, reinterpret_cast<XYZZ<Fp>*>(xtmp), 2 * chunk, st)) != ZKVC_OK)
      break;
    if (cudaGetLastError() != cudaSuccess) {
      rc = ZKVC_ECUDA;
      break;
    }
    zkvc_vk* vk = new zkvc_vk();
    Shape vs;
    vs.a = a;
    vs.n = n;
    vs.b = b;
    vs.l = (uint32_t)sh.l;
    vk->shape = vs;
    vk->circuit = circuit;
    vk->public_io = pub;
    vk->alpha1.resize(64);
    vk->beta2.resize(128);
    vk->gamma2.resize(128);
    vk->delta2.resize(128);
    vk->ic.resize(size_t(sh.l + 1) * 64);
    std::vector<uint64_t> idx(sh.l + 1);
    for (size_t i = 0; i <= sh.l; i++) idx[i] = i;
    if ((rc = export_points<Fp>(ic, idx, vk->ic.data(), st)) != ZKVC_OK ||
        (rc = export_points<Fp>(pk->g1, {G->ALPHA.off}, vk->alpha1.data(), st)) != ZKVC_OK ||
        (rc = export_points<Fp2>(pk->g2, {G->BETA2.off}, vk->beta2.data(), st)) != ZKVC_OK ||
        (rc = export_points<Fp2>(pk->g2, {G->GAMMA2.off}, vk->gamma2.data(), st)) != ZKVC_OK ||
        (rc = export_points<Fp2>(pk->g2, {G->DELTA2.off}, vk->delta2.data(), st)) != ZKVC_OK) {
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

// ------------------------------------------------------------------ witness kernels
// crpc: p_k = a_k b_k
__global__ void k_gen_crpc_products(const Fr* __restrict__ ak, const Fr* __restrict__ bk, int n, Fr* P) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) st_field(P + k, f_mul(ld_field(ak + k), ld_field(bk + k)));
}

// psq: S_ijk = sum_(k' <= k) x_ik' w_k'j for k < n - 1 (thread per output y_ij)
__global__ void k_gen_psq_chains(const int8_t* __restrict__ X, const int8_t* __restrict__ W, int a, int n, int b,
                                 int32_t* S) {
  uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= uint64_t(a) * b) return;
  const uint64_t i = t / b, j = t % b;
  int32_t acc = 0;
  for (int k = 0; k + 1 < n; k++) {
    acc += int32_t(X[i * n + k]) * int32_t(W[uint64_t(k) * b + j]);
    S[t * (n - 1) + k] = acc;
  }
}

// vanilla: p_ijk = x_ik w_kj (|p| <= 2^14)
__global__ void k_gen_products(const int8_t* __restrict__ X, const int8_t* __restrict__ W, int a, int n, int b,
                               int16_t* P) {
  uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t total = uint64_t(a) * b * n;
  if (t >= total) return;
  const uint64_t k = t % n, ij = t / n, j = ij % b, i = ij / b;
  P[t] = (int16_t)(int32_t(X[i * n + k]) * int32_t(W[k * b + j]));
}

// canonical v < 2^32 or |v| < 2^63 as Fr in Montgomery form
__device__ __forceinline__ Fr fr_from_u32(uint32_t v) {
  Fr x = Fr::zero();
  x.v[0] = v;
  return f_to_mont(x);
}

__device__ __forceinline__ Fr fr_from_i64(int64_t v) {
  const uint64_t mag = v < 0 ? uint64_t(0) - uint64_t(v) : uint64_t(v);
  Fr x = Fr::zero();
  x.v[0] = (uint32_t)mag;
  x.v[1] = (uint32_t)(mag >> 32);
  x = f_to_mont(x);
  return v < 0 ? f_neg(x) : x;
}

// GELU gadget (Sec. III-C): G = y^2 + 2^(GF+1) y + 2^(2GF+2) for every entry of Y
// (= (y + 2^GF)^2 + 3 2^(2GF) < 2^63 for |y| < 2^31)
__global__ void k_gen_gelu(const int32_t* __restrict__ Y, uint64_t count, Fr* __restrict__ g) {
  uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t y = Y[t];
  st_field(g + t, fr_from_i64(y * y + y * (int64_t(1) << (GF + 1)) + (int64_t(1) << (2 * GF + 2))));
}

// SoftMax gadget (Sec. III-C) for row blockIdx.x of Y (b entries), a block of 256 threads:
// x_max by a block reduction; per entry the bits of d = x_max - y and of
// u = |T| - d + 2^32, beta = [d <= |T|] (2^GF - d / 2^GM) and its GM squarings; then the
// prefix products P_j = (x_max - y_0) .. (x_max - y_j), j = 1 .. b-2, by chunks: each
// thread multiplies its chunk, a log-step scan over the 256 chunk products in shared
// memory gives each chunk its prefix, and a second pass writes the products.
constexpr int SM_THREADS = 256;
__global__ void __launch_bounds__(SM_THREADS) k_gen_softmax(const int32_t* __restrict__ Y, uint32_t b,
                                                            Fr* __restrict__ g) {
  __shared__ int32_t wmax[SM_THREADS / 32];
  __shared__ Fr scan[SM_THREADS];
  const uint32_t tid = threadIdx.x;
  const int32_t* y = Y + uint64_t(blockIdx.x) * b;
  Fr* out = g + uint64_t(blockIdx.x) * softmax_row_aux(b);
  int32_t m = INT32_MIN;
  for (uint32_t j = tid; j < b; j += SM_THREADS) m = max(m, y[j]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) wmax[tid >> 5] = m;
  __syncthreads();
  m = wmax[0];
  for (int w = 1; w < SM_THREADS / 32; w++) m = max(m, wmax[w]);
  if (tid == 0) st_field(out, f_from_int<FrCfg>(m));
  const uint32_t nprod = b > 2 ? b - 2 : 0;
  Fr* ent = out + 1 + nprod;
  const Fr one = Fr::one(), zero = Fr::zero();
  for (uint32_t j = tid; j < b; j += SM_THREADS) {
    const uint32_t d = (uint32_t)(int64_t(m) - int64_t(y[j]));
    const uint64_t u = GT - uint64_t(d) + (1ull << GD);
    Fr* e = ent + uint64_t(j) * G_PER_ENTRY;
    for (uint32_t k = 0; k < GD; k++) st_field(e + k, (d >> k) & 1u ? one : zero);
    for (uint32_t k = 0; k < GU; k++) st_field(e + GD + k, (u >> k) & 1ull ? one : zero);
    const int32_t beta = uint64_t(d) <= GT ? (1 << GF) - int32_t(d >> GM) : 0;
    Fr p = f_from_int<FrCfg>(beta);
    st_field(e + GD + GU, p);
    for (uint32_t t = 0; t < GM; t++) {
      p = f_mul(p, p);
      st_field(e + GD + GU + 1 + t, p);
    }
  }
  if (nprod == 0) return;
  // prefix products of d_0 .. d_(b-2) (P_j for j = 1 .. b-2)
  const uint32_t len = b - 1, chunk = (len + SM_THREADS - 1) / SM_THREADS;
  const uint32_t lo = min(len, tid * chunk), hi = min(len, lo + chunk);
  auto dfr = [&](uint32_t j) { return fr_from_u32((uint32_t)(int64_t(m) - int64_t(y[j]))); };
  Fr acc = one;
  for (uint32_t j = lo; j < hi; j++) acc = f_mul(acc, dfr(j));
  st_field(&scan[tid], acc);
  __syncthreads();
  for (uint32_t off = 1; off < SM_THREADS; off <<= 1) {  // inclusive scan of the chunk products
    Fr v = ld_field(&scan[tid]);
    if (tid >= off) v = f_mul(ld_field(&scan[tid - off]), v);
    __syncthreads();
    st_field(&scan[tid], v);
    __syncthreads();
  }
  Fr pre = tid ? ld_field(&scan[tid - 1]) : one;
  for (uint32_t j = lo; j < hi; j++) {
    pre = f_mul(pre, dfr(j));
    if (j >= 1) st_field(out + 1 + (j - 1), pre);
  }
}

struct WSrc {
  const int8_t* X;
  const int32_t* Y;
  const int8_t* W;
  const void* aux;
  int aux_kind;
  uint64_t first[G_COUNT];
};

// w[v] in Montgomery form for every variable
__global__ void k_gen_wfull(WSrc s, uint64_t n_vars, Fr* w) {
  uint64_t v = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= n_vars) return;
  Fr x;
  if (v == 0) {
    x = Fr::one();
  } else if (v < s.first[G_Y]) {
    x = f_from_int<FrCfg>(s.X[v - s.first[G_X]]);
  } else if (v < s.first[G_W]) {
    x = f_from_int<FrCfg>(s.Y[v - s.first[G_Y]]);
  } else if (v < s.first[G_AUX]) {
    x = f_from_int<FrCfg>(s.W[v - s.first[G_W]]);
  } else {
    uint64_t t = v - s.first[G_AUX];
    if (s.aux_kind == SK_FR_MONT)
      x = ld_field(reinterpret_cast<const Fr*>(s.aux) + t);
    else if (s.aux_kind == SK_I32)
      x = f_from_int<FrCfg>(reinterpret_cast<const int32_t*>(s.aux)[t]);
    else
      x = f_from_int<FrCfg>((int32_t)reinterpret_cast<const int16_t*>(s.aux)[t]);
  }
  st_field(w + v, x);
}

struct CsrView {
  const uint64_t* rowptr[3];
  const uint32_t* col[3];
  const uint32_t* coef[3];
};

__device__ __forceinline__ Fr coef_times(uint32_t c, const Fr& x, const Fr* tab) {
  if (c == COEF_ONE) return x;
  if (c == COEF_NEG) return f_neg(x);
  return f_mul(ld_field(tab + c), x);
}

// Aev/Bev/Cev[r] = <row r, w> for rows whose three parts have at most LONG_ROW entries;
// rows r in [n_rows, N) are zero.
__global__ void k_gen_spmv(CsrView m, const Fr* __restrict__ tab, const Fr* __restrict__ w, uint64_t n_rows, size_t N,
                           Fr* Aev, Fr* Bev, Fr* Cev) {
  uint64_t r = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= N) return;
  Fr* out[3] = {Aev, Bev, Cev};
  if (r >= n_rows) {
    for (int mi = 0; mi < 3; mi++) st_field(out[mi] + r, Fr::zero());
    return;
  }
  for (int mi = 0; mi < 3; mi++)
    if (m.rowptr[mi][r + 1] - m.rowptr[mi][r] > LONG_ROW) return;
  for (int mi = 0; mi < 3; mi++) {
    Fr acc = Fr::zero();
    for (uint64_t e = m.rowptr[mi][r]; e < m.rowptr[mi][r + 1]; e++)
      acc = f_add(acc, coef_times(m.coef[mi][e], ld_field(w + m.col[mi][e]), tab));
    st_field(out[mi] + r, acc);
  }
}

// a block (256 threads) per long row
__global__ void __launch_bounds__(256) k_gen_spmv_long(CsrView m, const uint32_t* __restrict__ rows,
                                                       const Fr* __restrict__ tab, const Fr* __restrict__ w, Fr* Aev,
                                                       Fr* Bev, Fr* Cev) {
  __shared__ Fr sh[256];
  const uint32_t r = rows[blockIdx.x];
  Fr* out[3] = {Aev, Bev, Cev};
  for (int mi = 0; mi < 3; mi++) {
    Fr acc = Fr::zero();
    for (uint64_t e = m.rowptr[mi][r] + threadIdx.x; e < m.rowptr[mi][r + 1]; e += blockDim.x)
      acc = f_add(acc, coef_times(m.coef[mi][e], ld_field(w + m.col[mi][e]), tab));
    Fr tot = block_sum(acc, sh);
    if (threadIdx.x == 0) st_field(out[mi] + r, tot);
  }
}

// A = pre[0]; C = pre[1] + h[0] + s A + r B1; B = g2[0]
__global__ void k_gen_encode(const G1J* pre, const G1J* hq, const G1J* chain, const G2J* g2, uint8_t* proof) {
  if (threadIdx.x == 0) {
    G1J A = ld_field(pre);
    G1J C = p_add(p_add(ld_field(pre + 1), ld_field(hq)), p_add(ld_field(chain), ld_field(chain + 1)));
    encode_a_c(A, C, proof);
  } else if (threadIdx.x == 32) {
    encode_b(ld_field(g2), proof);
  }
}

// ------------------------------------------------------------------ prover
struct GenBufs {
  Fr *ak, *bk, *yz, *S, *w, *ev, *rs;
  void* aux;
  int* flags;
  G1J *pre, *hres, *chain;
  GlvScalar* glv;
  G2J* g2res;
  uint8_t* proof;
  void *ws_pre, *ws_h, *ws_g2;
  size_t ws_pre_bytes, ws_h_bytes, ws_g2_bytes;
};

struct GenPlans {
  MsmPlan pre, h, g2;
};

static MsmSeg gseg(const GRegion& r, uint64_t count, uint32_t out, int kind, const void* sc, uint32_t skip = 0xffffffffu) {
  MsmSeg s{};
  s.base_off = r.off;
  s.count = (uint32_t)count;
  s.nwin = r.nwin;
  s.out = out;
  s.kind = kind;
  s.scalars = sc;
  s.skip = skip;
  return s;
}

static void gen_plans(const GenericKey& G, const void* src[G_COUNT], const Fr* h, const Fr* rs, GenPlans* P) {
  const GShape& sh = G.sh;
  P->pre.outs = {{C1, 1, 0, 0}, {C1, 1, 0, 0}, {C1, 1, 0, 0}};
  auto& s = P->pre.segs;
  s.clear();
  for (int g = 0; g < G_COUNT; g++) {
    const int kd = sh.kind[g];
    if (G.g1q[GQ_A][g].count) s.push_back(gseg(G.g1q[GQ_A][g], sh.count[g], 0, kd, src[g]));
    if (G.g1q[GQ_L][g].count) s.push_back(gseg(G.g1q[GQ_L][g], sh.count[g], 1, kd, src[g]));
    if (G.g1q[GQ_B1][g].count) s.push_back(gseg(G.g1q[GQ_B1][g], sh.count[g], 2, kd, src[g]));
  }
  s.push_back(gseg(G.ALPHA, 1, 0, SK_ONE, nullptr));
  s.push_back(gseg(G.DELTA, 1, 0, SK_FR_CANON, rs + 0));
  s.push_back(gseg(G.BETA, 1, 2, SK_ONE, nullptr));
  s.push_back(gseg(G.DELTA, 1, 2, SK_FR_CANON, rs + 1));
  P->h.outs = {{C1, 1, 0, 0}};
  P->h.segs = {gseg(G.H, sh.N, 0, SK_FR_MONT, h, (uint32_t)sh.N - 1), gseg(G.DELTA, 1, 0, SK_FR_CANON, rs + 3)};
  P->g2.outs = {{C2, 1, 0, 0}};
  P->g2.segs.clear();
  for (int g = 0; g < G_COUNT; g++)
    if (G.B2[g].count) P->g2.segs.push_back(gseg(G.B2[g], sh.count[g], 0, sh.kind[g], src[g]));
  P->g2.segs.push_back(gseg(G.BETA2, 1, 0, SK_ONE, nullptr));
  P->g2.segs.push_back(gseg(G.DELTA2, 1, 0, SK_FR_CANON, rs + 1));
  msm_plan_finalize(P->pre);
  msm_plan_finalize(P->h);
  msm_plan_finalize(P->g2);
}

static size_t aux_bytes(const GShape& sh) {
  size_t e = sh.kind[G_AUX] == SK_FR_MONT ? 32 : sh.kind[G_AUX] == SK_I32 ? 4 : 2;
  return std::max<size_t>(1, sh.n_aux) * e;
}

static size_t gen_carve(const zkvc_pk* pk, void* base, size_t cap, GenBufs* B, bool measuring) {
  const GenericKey& G = *pk->gen;
  const GShape& sh = G.sh;
  Arena a;
  a.base = reinterpret_cast<uint8_t*>(base);
  a.cap = cap;
  a.measuring = measuring;
  B->ak = a.take<Fr>(sh.n);
  B->bk = a.take<Fr>(sh.n);
  B->yz = a.take<Fr>(sh.a);
  B->S = a.take<Fr>(sh.n);
  B->aux = a.take<uint8_t>(aux_bytes(sh));
  B->w = a.take<Fr>(sh.n_vars);
  B->ev = a.take<Fr>(4 * sh.N);
  B->rs = a.take<Fr>(4);
  B->flags = a.take<int>(4);
  B->pre = a.take<G1J>(3);
  B->hres = a.take<G1J>(1);
  B->chain = a.take<G1J>(2);
  B->glv = a.take<GlvScalar>(2);
  B->g2res = a.take<G2J>(1);
  B->proof = a.take<uint8_t>(256);
  GenPlans P;
  const void* src[G_COUNT] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  gen_plans(G, src, nullptr, nullptr, &P);
  B->ws_pre_bytes = msm_workspace_bytes<Fp>(P.pre);
  B->ws_h_bytes = msm_workspace_bytes<Fp>(P.h);
  B->ws_g2_bytes = msm_workspace_bytes<Fp2>(P.g2);
  B->ws_pre = a.take<uint8_t>(B->ws_pre_bytes);
  B->ws_h = a.take<uint8_t>(B->ws_h_bytes);
  B->ws_g2 = a.take<uint8_t>(B->ws_g2_bytes);
  return a.off;
}

size_t prove_generic_workspace_bytes(const zkvc_pk* pk) {
  GenBufs B;
  return gen_carve(pk, nullptr, 0, &B, true);
}

struct GenStreams {
  int dev = -1;
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
static thread_local GenStreams t_gen;

int prove_generic(const zkvc_pk* pk, const int8_t* dX, const int8_t* dW, const uint8_t* rs_host, int32_t* dY, void* ws,
                  size_t ws_bytes, uint8_t* proof_host, cudaStream_t st, bool y_given) {
  ZK_CHECK(pk && pk->gen && dX && dW && rs_host && dY && ws && proof_host, ZKVC_EINVAL, "prove: null argument");
  const GenericKey& G = *pk->gen;
  const GShape& sh = G.sh;
  size_t need = prove_generic_workspace_bytes(pk);
  ZK_CHECK(ws_bytes >= need, ZKVC_EINVAL, "prove: workspace %zu < %zu bytes", ws_bytes, need);
  GenBufs B;
  gen_carve(pk, ws, ws_bytes, &B, false);
  const size_t N = sh.N;
  Fr* Aev = B.ev;
  Fr* Bev = B.ev + N;
  Fr* Cev = B.ev + 2 * N;
  Fr* Hev = B.ev + 3 * N;
  int dev = 0;
  ZK_CUDA(cudaGetDevice(&dev));
  if (t_gen.side == nullptr || t_gen.dev != dev) {
    t_gen.dev = dev;
    ZK_CUDA(cudaStreamCreateWithFlags(&t_gen.side, cudaStreamNonBlocking));
    ZK_CUDA(cudaEventCreateWithFlags(&t_gen.fork, cudaEventDisableTiming));
    ZK_CUDA(cudaEventCreateWithFlags(&t_gen.join, cudaEventDisableTiming));
  }

  ZK_CUDA(cudaMemsetAsync(B.flags, 0, 4 * sizeof(int), st));
  ZK_CUDA(cudaMemcpyAsync(B.rs, rs_host, 64, cudaMemcpyHostToDevice, st));
  {
    // s and r split by the GLV endomorphism for s A and r B1
    const GlvScalar g[2] = {glv_split(rs_host + 32), glv_split(rs_host)};
    ZK_CUDA(cudaMemcpyAsync(B.glv, g, sizeof(g), cudaMemcpyHostToDevice, st));
  }
  k_randomness<<<1, 1, 0, st>>>(B.rs, B.flags); ZK_COUNT_LAUNCH();
  // witness: Y (X W, or the caller's claimed Y), then the auxiliary variables
  if (!y_given) ZK_TRY(matmul_i8(dX, dW, dY, sh.a, sh.n, sh.b, B.flags, st));
  switch (sh.circuit) {
    case ZKVC_CIRCUIT_CRPC_PSQ:
    case ZKVC_CIRCUIT_CRPC:
    case ZKVC_CIRCUIT_SOFTMAX:
    case ZKVC_CIRCUIT_GELU:
      k_crpc_ab<<<sh.n, 256, 0, st>>>(dX, dW, pk->zA, pk->zB, sh.a, sh.n, sh.b, B.ak, B.bk); ZK_COUNT_LAUNCH();
      if (sh.circuit != ZKVC_CIRCUIT_CRPC) {
        k_crpc_y<<<sh.a, 256, 0, st>>>(dY, pk->zA, pk->zB, sh.b, B.yz); ZK_COUNT_LAUNCH();
        // prefix sums into the auxiliary array; the first n evaluations land in ev and are
        // rewritten identically by the matrix product below
        k_psq<<<1, 1024, 0, st>>>(B.ak, B.bk, B.yz, sh.a, sh.n, reinterpret_cast<Fr*>(B.aux), Aev, Bev, Cev, B.flags); ZK_COUNT_LAUNCH();
      } else {
        k_gen_crpc_products<<<(sh.n + 255) / 256, 256, 0, st>>>(B.ak, B.bk, sh.n, reinterpret_cast<Fr*>(B.aux)); ZK_COUNT_LAUNCH();
      }
      if (sh.circuit == ZKVC_CIRCUIT_SOFTMAX) {  // the gadget block follows the n - 1 prefix sums
        k_gen_softmax<<<sh.a, SM_THREADS, 0, st>>>(dY, (uint32_t)sh.b, reinterpret_cast<Fr*>(B.aux) + (sh.n - 1)); ZK_COUNT_LAUNCH();
      } else if (sh.circuit == ZKVC_CIRCUIT_GELU) {
        const uint64_t t = uint64_t(sh.a) * sh.b;
        k_gen_gelu<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(dY, t, reinterpret_cast<Fr*>(B.aux) + (sh.n - 1)); ZK_COUNT_LAUNCH();
      }
      break;
    case ZKVC_CIRCUIT_PSQ: {
      uint64_t t = uint64_t(sh.a) * sh.b;
      k_gen_psq_chains<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(dX, dW, sh.a, sh.n, sh.b, reinterpret_cast<int32_t*>(B.aux)); ZK_COUNT_LAUNCH();
      break;
    }
    default: {
      uint64_t t = uint64_t(sh.a) * sh.b * sh.n;
      k_gen_products<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(dX, dW, sh.a, sh.n, sh.b, reinterpret_cast<int16_t*>(B.aux)); ZK_COUNT_LAUNCH();
      break;
    }
  }
  ZK_CUDA(cudaGetLastError());
  WSrc src{dX, dY, dW, B.aux, sh.kind[G_AUX], {}};
  for (int g = 0; g < G_COUNT; g++) src.first[g] = sh.first[g];
  k_gen_wfull<<<(unsigned)((sh.n_vars + 255) / 256), 256, 0, st>>>(src, sh.n_vars, B.w); ZK_COUNT_LAUNCH();
  const void* msrc[G_COUNT] = {nullptr, dX, dY, dW, B.aux};
  GenPlans P;
  gen_plans(G, msrc, Hev, B.rs, &P);
  // G2 MSM on the side stream (needs W and s)
  ZK_CUDA(cudaEventRecord(t_gen.fork, st));
  ZK_CUDA(cudaStreamWaitEvent(t_gen.side, t_gen.fork, 0));
  ZK_TRY(msm_run<Fp2>(P.g2, pk->g2, B.ws_g2, B.ws_g2_bytes, B.g2res, t_gen.side));
  ZK_CUDA(cudaEventRecord(t_gen.join, t_gen.side));
  // domain evaluations
  CsrView cv;
  for (int mi = 0; mi < 3; mi++) {
    cv.rowptr[mi] = G.csr[mi].rowptr;
    cv.col[mi] = G.csr[mi].col;
    cv.coef[mi] = G.csr[mi].coef;
  }
  k_gen_spmv<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(cv, G.coef_tab, B.w, sh.n_rows, N, Aev, Bev, Cev); ZK_COUNT_LAUNCH();
  if (G.n_long) {
    k_gen_spmv_long<<<G.n_long, 256, 0, st>>>(cv, G.long_rows, G.coef_tab, B.w, Aev, Bev, Cev); ZK_COUNT_LAUNCH();
  }
  ZK_CUDA(cudaGetLastError());
  // A, the private part of C and B1 (all witness scalars known now)
  ZK_TRY(msm_run<Fp>(P.pre, pk->g1, B.ws_pre, B.ws_pre_bytes, B.pre, st));
  k_chains<<<1, 160, 0, st>>>(B.glv, B.pre, B.chain, nullptr, nullptr); ZK_COUNT_LAUNCH();
  // quotient and H
  const NttDomain* d = pk->dom;
  ZK_TRY(ntt_quotient_chain(Aev, 1, N, d, st));
  k_check_h<<<1, 32, 0, st>>>(Hev, N, B.flags); ZK_COUNT_LAUNCH();
  ZK_TRY(msm_run<Fp>(P.h, pk->g1, B.ws_h, B.ws_h_bytes, B.hres, st));
  ZK_CUDA(cudaStreamWaitEvent(st, t_gen.join, 0));
  k_gen_encode<<<1, 64, 0, st>>>(B.pre, B.hres, B.chain, B.g2res, B.proof); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  int flags = 0;
  ZK_CUDA(cudaMemcpyAsync(proof_host, B.proof, 256, cudaMemcpyDeviceToHost, st));
  ZK_CUDA(cudaMemcpyAsync(&flags, B.flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  ZK_CUDA(cudaStreamSynchronize(st));
  ZK_CHECK(!(flags & 4), ZKVC_EINVAL, "prove: r or s is not a canonical Fr element");
  ZK_CHECK(!(flags & 1), ZKVC_EUNSAT, "prove: the PSQ chain does not close against Y(z)");
  ZK_CHECK(!(flags & 2), ZKVC_EUNSAT, "prove: the quotient has degree N - 1 (QAP not satisfied)");
  return ZKVC_OK;
}

// ------------------------------------------------------------------ export
int export_generic(const zkvc_pk* pk, int query, size_t first, size_t count, uint8_t* out) {
  const GenericKey& G = *pk->gen;
  const GShape& sh = G.sh;
  const bool g2 = query == ZKVC_Q_B2 || query == ZKVC_Q_BETA2 || query == ZKVC_Q_DELTA2;
  const size_t width = g2 ? 128 : 64;
  uint64_t total = 0;
  switch (query) {
    case ZKVC_Q_A: case ZKVC_Q_B1: case ZKVC_Q_B2: case ZKVC_Q_L: total = sh.n_vars; break;
    case ZKVC_Q_H: total = sh.N - 1; break;
    case ZKVC_Q_ALPHA1: case ZKVC_Q_BETA1: case ZKVC_Q_BETA2: case ZKVC_Q_DELTA1: case ZKVC_Q_DELTA2: total = 1; break;
    default: ZK_CHECK(false, ZKVC_EINVAL, "pk_export: unknown query %d", query);
  }
  ZK_CHECK(first <= total && count <= total - first, ZKVC_EINVAL, "pk_export: range [%zu, %zu) outside %llu entries",
           first, first + count, (unsigned long long)total);
  std::vector<uint64_t> idx;
  std::vector<size_t> where;
  for (size_t q = 0; q < count; q++) {
    uint64_t e = first + q;
    const GRegion* r = nullptr;
    uint64_t at = 0;
    switch (query) {
      case ZKVC_Q_A: case ZKVC_Q_B1: case ZKVC_Q_B2: case ZKVC_Q_L: {
        int g = G_COUNT - 1;
        while (g > 0 && e < sh.first[g]) g--;
        r = query == ZKVC_Q_A ? &G.g1q[GQ_A][g] : query == ZKVC_Q_B1 ? &G.g1q[GQ_B1][g]
            : query == ZKVC_Q_L ? &G.g1q[GQ_L][g] : &G.B2[g];
        at = e - sh.first[g];
        break;
      }
      case ZKVC_Q_H: {
        uint32_t p = 0;
        for (uint32_t bit = 0; bit < sh.logN; bit++) p |= ((uint32_t)(e >> bit) & 1u) << (sh.logN - 1 - bit);
        r = &G.H;
        at = p;
        break;
      }
      case ZKVC_Q_ALPHA1: r = &G.ALPHA; break;
      case ZKVC_Q_BETA1: r = &G.BETA; break;
      case ZKVC_Q_DELTA1: r = &G.DELTA; break;
      case ZKVC_Q_BETA2: r = &G.BETA2; break;
      default: r = &G.DELTA2; break;
    }
    if (r->count == 0) continue;  // no entry: infinity (zero bytes)
    idx.push_back(r->off + at * r->nwin);
    where.push_back(q);
  }
  std::memset(out, 0, count * width);
  std::vector<uint8_t> tmpb(idx.size() * width);
  if (g2)
    ZK_TRY(export_points<Fp2>(pk->g2, idx, tmpb.data(), 0));
  else
    ZK_TRY(export_points<Fp>(pk->g1, idx, tmpb.data(), 0));
  for (size_t i = 0; i < where.size(); i++) std::memcpy(out + where[i] * width, tmpb.data() + i * width, width);
  return ZKVC_OK;
}

}  // namespace zkvc
