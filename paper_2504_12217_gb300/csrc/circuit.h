// Generic sparse-R1CS Groth16 keys and prover (internal): the circuit variants of the
// paper's ablation (Sec. V, Table II) and the private-input mode, on one set of kernels.
#pragma once
#include "groth16.h"

namespace zkvc {

// Variable groups, in variable order: one | X | Y | W | auxiliary.
enum GroupId : int { G_ONE = 0, G_X, G_Y, G_W, G_AUX, G_COUNT };

struct GShape {
  int a = 0, n = 0, b = 0;
  int circuit = 0;      // ZKVC_CIRCUIT_*
  int pub = 0;          // ZKVC_PUBLIC_*
  uint64_t n_io = 0;    // entries of X and Y
  uint64_t l = 0;       // public inputs
  uint64_t n_aux = 0, n_vars = 0;
  uint64_t n_crows = 0; // circuit rows (before the input-consistency rows)
  uint64_t n_rows = 0;  // n_crows + l + 1
  uint32_t logN = 0;
  size_t N = 0;
  uint64_t first[G_COUNT] = {}, count[G_COUNT] = {};
  int kind[G_COUNT] = {};  // ScalarKind of each group's witness values
};

int make_gshape(int a, int n, int b, int circuit, int pub, GShape* s);

// A dense run of bases over the variables of one group (count = 0: absent).
struct GRegion {
  uint64_t off = 0;
  uint64_t count = 0;
  uint32_t nwin = 0;
  uint32_t c = 0;
};

enum GQuery : int { GQ_A = 0, GQ_B1, GQ_L, GQ_COUNT };

struct Csr {  // device, one matrix of the R1CS by rows
  uint64_t* rowptr = nullptr;
  uint32_t* col = nullptr;
  uint32_t* coef = nullptr;  // index into the coefficient table
  uint64_t nnz = 0;
};

struct GenericKey {
  GShape sh;
  GRegion g1q[GQ_COUNT][G_COUNT];  // G1, c = 16
  GRegion H, ALPHA, BETA, DELTA;    // G1, c = 16 (DELTA stores 16 windows)
  GRegion B2[G_COUNT];              // G2, c = 8
  GRegion BETA2, DELTA2, GAMMA2;    // G2, c = 8 (DELTA2 stores 32 windows)
  uint64_t n_g1 = 0, n_g2 = 0;
  Csr csr[3];                       // A, B, C
  Fr* coef_tab = nullptr;           // 1, -1, z^0, z^1, ... (Montgomery)
  uint32_t n_coef = 0;
  uint32_t* long_rows = nullptr;    // rows reduced by a whole block
  uint32_t n_long = 0;
  ~GenericKey();
};

int setup_generic(int a, int n, int b, int circuit, int pub, const uint8_t* toxic, cudaStream_t st, zkvc_pk** pk,
                  zkvc_vk** vk);
size_t prove_generic_workspace_bytes(const zkvc_pk* pk);
// y_given: dY holds a claimed Y to prove instead of receiving X W (ZKVC_EUNSAT if the
// circuit's rows then fail).
int prove_generic(const zkvc_pk* pk, const int8_t* dX, const int8_t* dW, const uint8_t* rs_host, int32_t* dY, void* ws,
                  size_t ws_bytes, uint8_t* proof_host, cudaStream_t st, bool y_given = false);
// Canonical encodings of query entries by variable index (infinity where the query has
// no entry); H by position (bit-reversed storage undone), constants at index 0.
int export_generic(const zkvc_pk* pk, int query, size_t first, size_t count, uint8_t* out);

}  // namespace zkvc
