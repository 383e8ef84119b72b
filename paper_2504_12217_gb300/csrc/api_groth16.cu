// C-ABI entry points of the Groth16 layer: setup, prove, key export and release.
#include <algorithm>
#include <tuple>
#include <string>
#include <mutex>
#include <map>
#include <array>
#include <cstdio>
#include <cstring>

#include "circuit.h"
#include "groth16.h"

namespace zkvc {
int setup_impl(int a, int n, int b, const uint8_t* toxic, cudaStream_t st, zkvc_pk** pk, zkvc_vk** vk);
size_t prove_workspace_bytes(const zkvc_pk* pk, int mode);
int prove_autotune(zkvc_pk* pk, int mode, const int8_t* dX, const int8_t* dW, const uint8_t* rs, cudaStream_t st,
                   uint32_t* chosen);
int prove_impl(const zkvc_pk* pk, int mode, const int8_t* dX, const int8_t* dW, const uint8_t* rs, int32_t* dY,
               void* ws, size_t ws_bytes, uint8_t* proof, cudaStream_t st);
int prove_graph(const zkvc_pk* pk, int mode, const int8_t* dX, const int8_t* dW, const uint8_t* rs, int32_t* dY,
                void* ws, size_t ws_bytes, uint8_t* proof, cudaStream_t st);
int prove_claimed(const zkvc_pk* pk, int mode, const int8_t* dX, const int8_t* dW, const uint8_t* rs,
                  const int32_t* dY, void* ws, size_t ws_bytes, uint8_t* proof, cudaStream_t st);
template <class F>
int export_points(const Affine<F>* src, const std::vector<uint64_t>& idx, uint8_t* host_out, cudaStream_t st);

template <class F>
size_t generator_mul_ws(size_t n);
template <class F>
int generator_mul(const uint8_t* d_scalars, size_t n, uint8_t* d_out, void* ws, size_t ws_bytes, cudaStream_t st);

int verify_impl(const zkvc_vk* vk, const int8_t* X, const int32_t* Y, const uint8_t* proof, int* ok);

// ------------------------------------------------------------------ tuning cache
// Results of the one-proof autotuner, keyed by the matmul shape, the requested mode and
// the GPU (name and SM count): later keys of the same shape on the same kind of GPU take
// the stored launch shape without timing.  Process-wide, guarded by a mutex; saved to and
// loaded from a small text file (one entry per line: a n b mode sms tuning[0..9] name).
struct TuneKey {
  int a, n, b, mode, sms;
  std::string gpu;
  bool operator<(const TuneKey& o) const {
    return std::tie(a, n, b, mode, sms, gpu) < std::tie(o.a, o.n, o.b, o.mode, o.sms, o.gpu);
  }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, std::array<uint32_t, ZKVC_PK_TUNING_LEN>> g_tune_cache;

static int tune_key(const zkvc_pk* pk, int mode, TuneKey* k) {
  cudaDeviceProp prop;
  ZK_CUDA(cudaGetDeviceProperties(&prop, pk->device));
  k->a = (int)pk->shape.a;
  k->n = (int)pk->shape.n;
  k->b = (int)pk->shape.b;
  k->mode = mode;
  k->sms = prop.multiProcessorCount;
  k->gpu = prop.name;
  for (char& c : k->gpu)
    if (c == ' ' || c == '\t' || c == '\n') c = '_';
  return ZKVC_OK;
}

static bool tune_cache_get(const TuneKey& k, uint32_t* t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune_cache.find(k);
  if (it == g_tune_cache.end()) return false;
  for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) t[i] = it->second[i];
  return true;
}

static void tune_cache_put(const TuneKey& k, const uint32_t* t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto& v = g_tune_cache[k];
  for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) v[i] = t[i];
}

static void tune_cache_clear() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.clear();
}

static int tune_cache_save(const char* path) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  FILE* f = std::fopen(path, "w");
  ZK_CHECK(f, ZKVC_EIO, "tune_cache_save: cannot open %s", path);
  std::fprintf(f, "zkvc-tune-cache 1\n");
  for (const auto& e : g_tune_cache) {
    const TuneKey& k = e.first;
    std::fprintf(f, "%d %d %d %d %d", k.a, k.n, k.b, k.mode, k.sms);
    for (uint32_t v : e.second) std::fprintf(f, " %u", v);
    std::fprintf(f, " %s\n", k.gpu.c_str());
  }
  const bool ok = std::fclose(f) == 0;
  ZK_CHECK(ok, ZKVC_EIO, "tune_cache_save: write to %s failed", path);
  return ZKVC_OK;
}

// Entries are validated as zkvc_pk_set_tuning would; a malformed line rejects the file
// (ZKVC_EIO) and leaves the cache as it was.
static int tune_cache_load(const char* path) {
  FILE* f = std::fopen(path, "r");
  ZK_CHECK(f, ZKVC_EIO, "tune_cache_load: cannot open %s", path);
  char line[1024];
  std::map<TuneKey, std::array<uint32_t, ZKVC_PK_TUNING_LEN>> got;
  int rc = ZKVC_OK;
  if (!std::fgets(line, sizeof(line), f) || std::strncmp(line, "zkvc-tune-cache 1", 17) != 0) {
    set_error("tune_cache_load: %s is not a tuning cache", path);
    rc = ZKVC_EIO;
  }
  while (rc == ZKVC_OK && std::fgets(line, sizeof(line), f)) {
    if (line[0] == '\n' || line[0] == 0) continue;
    TuneKey k;
    unsigned t[ZKVC_PK_TUNING_LEN];
    char name[512];
    const int nf = std::sscanf(line, "%d %d %d %d %d %u %u %u %u %u %u %u %u %u %u %511s", &k.a, &k.n, &k.b, &k.mode,
                               &k.sms, &t[0], &t[1], &t[2], &t[3], &t[4], &t[5], &t[6], &t[7], &t[8], &t[9], name);
    bool ok = nf == 16 && k.a >= 1 && k.n >= 1 && k.b >= 1 && k.mode >= ZKVC_PROVE_FOLD && k.mode <= ZKVC_PROVE_AUTO &&
              k.sms >= 1;
    for (int i = 0; ok && i < 4; i++) ok = t[i] <= 1024;
    ok = ok && (t[4] == 0 || (t[4] >= 8 && t[4] <= 11)) && t[5] <= 2 && t[6] <= 1 && t[7] <= 1 && t[8] <= 1 &&
         t[9] <= 1;
    if (!ok) {
      set_error("tune_cache_load: malformed entry in %s: %s", path, line);
      rc = ZKVC_EIO;
      break;
    }
    k.gpu = name;
    auto& v = got[k];
    for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) v[i] = t[i];
  }
  std::fclose(f);
  if (rc != ZKVC_OK) return rc;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& e : got) g_tune_cache[e.first] = e.second;
  return ZKVC_OK;
}

int vk_get(const zkvc_vk* vk, int* a, int* n, int* b, const uint8_t** alpha1, const uint8_t** beta2,
           const uint8_t** gamma2, const uint8_t** delta2, const uint8_t** ic, size_t* n_ic) {
  ZK_CHECK(vk && vk->alpha1.size() == 64 && vk->beta2.size() == 128 && vk->gamma2.size() == 128 &&
               vk->delta2.size() == 128 && vk->ic.size() % 64 == 0,
           ZKVC_EIO, "verify: malformed verifying key");
  *a = vk->shape.a;
  *n = vk->shape.n;
  *b = vk->shape.b;
  *alpha1 = vk->alpha1.data();
  *beta2 = vk->beta2.data();
  *gamma2 = vk->gamma2.data();
  *delta2 = vk->delta2.data();
  *ic = vk->ic.data();
  *n_ic = vk->ic.size() / 64;
  return ZKVC_OK;
}

// ------------------------------------------------------------------ key files
// Layout: 8-byte magic, u32 version, u32 header words, then i32 a, n, b, u32 log N,
// u64 counts, the payload, and a trailing FNV-1a-64 checksum of the payload.
static const char PK_MAGIC[8] = {'Z', 'K', 'V', 'C', 'P', 'K', '\0', '\1'};
static const char VK_MAGIC[8] = {'Z', 'K', 'V', 'C', 'V', 'K', '\0', '\1'};
static const uint32_t KEY_VERSION = 2;  // 2: per-row Lagrange regions of the CRPC W side

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const uint8_t* b = reinterpret_cast<const uint8_t*>(p);
    for (size_t i = 0; i < n; i++) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  }
};

struct FileGuard {
  FILE* f = nullptr;
  ~FileGuard() {
    if (f) fclose(f);
  }
};

static bool wr(FILE* f, const void* p, size_t n, Fnv* h) {
  if (h) h->add(p, n);
  return fwrite(p, 1, n, f) == n;
}

static bool rd(FILE* f, void* p, size_t n, Fnv* h) {
  if (fread(p, 1, n, f) != n) return false;
  if (h) h->add(p, n);
  return true;
}

// device array <-> file in 64 MiB pieces through a host buffer
static int dev_to_file(FILE* f, const void* d, size_t bytes, Fnv* h) {
  std::vector<uint8_t> buf(std::min<size_t>(bytes, size_t(64) << 20));
  for (size_t off = 0; off < bytes; off += buf.size()) {
    size_t m = std::min(buf.size(), bytes - off);
    ZK_CUDA(cudaMemcpy(buf.data(), reinterpret_cast<const uint8_t*>(d) + off, m, cudaMemcpyDeviceToHost));
    ZK_CHECK(wr(f, buf.data(), m, h), ZKVC_EIO, "key file: write failed");
  }
  return ZKVC_OK;
}

static int file_to_dev(FILE* f, void* d, size_t bytes, Fnv* h) {
  std::vector<uint8_t> buf(std::min<size_t>(bytes, size_t(64) << 20));
  for (size_t off = 0; off < bytes; off += buf.size()) {
    size_t m = std::min(buf.size(), bytes - off);
    ZK_CHECK(rd(f, buf.data(), m, h), ZKVC_EIO, "key file: truncated payload");
    ZK_CUDA(cudaMemcpy(reinterpret_cast<uint8_t*>(d) + off, buf.data(), m, cudaMemcpyHostToDevice));
  }
  return ZKVC_OK;
}

static int device_guard(int dev) {
  int cur = -1;
  ZK_CUDA(cudaGetDevice(&cur));
  ZK_CHECK(cur == dev, ZKVC_EINVAL, "key was built on device %d but device %d is current", dev, cur);
  return ZKVC_OK;
}
}  // namespace zkvc

using namespace zkvc;

extern "C" {

size_t zkvc_generator_mul_workspace_bytes(size_t n, int group) {
  return group == 2 ? generator_mul_ws<Fp2>(n) : generator_mul_ws<Fp>(n);
}

int zkvc_g1_generator_mul(const uint8_t* d_scalars, size_t n, uint8_t* d_points, void* d_ws, size_t ws_bytes,
                          void* stream) {
  set_error("%s", "");
  return generator_mul<Fp>(d_scalars, n, d_points, d_ws, ws_bytes, (cudaStream_t)stream);
}

int zkvc_g2_generator_mul(const uint8_t* d_scalars, size_t n, uint8_t* d_points, void* d_ws, size_t ws_bytes,
                          void* stream) {
  set_error("%s", "");
  return generator_mul<Fp2>(d_scalars, n, d_points, d_ws, ws_bytes, (cudaStream_t)stream);
}

int zkvc_setup(int a, int n, int b, const uint8_t toxic[192], void* stream, zkvc_pk** pk, zkvc_vk** vk) {
  set_error("%s", "");
  ZK_CHECK(toxic && pk && vk, ZKVC_EINVAL, "setup: null argument");
  *pk = nullptr;
  *vk = nullptr;
  return setup_impl(a, n, b, toxic, (cudaStream_t)stream, pk, vk);
}

void zkvc_pk_free(zkvc_pk* pk) {
  if (!pk) return;
  cudaFree(pk->g1);
  cudaFree(pk->g2);
  cudaFree(pk->zA);
  cudaFree(pk->zB);
  zkvc::prove_graph_free(pk->graph);
  delete pk->gen;
  delete pk;
}

int zkvc_setup_circuit(int a, int n, int b, int circuit, int public_io, const uint8_t toxic[192], void* stream,
                       zkvc_pk** pk, zkvc_vk** vk) {
  set_error("%s", "");
  ZK_CHECK(toxic && pk && vk, ZKVC_EINVAL, "setup: null argument");
  *pk = nullptr;
  *vk = nullptr;
  return setup_generic(a, n, b, circuit, public_io, toxic, (cudaStream_t)stream, pk, vk);
}

int zkvc_pk_autotune(zkvc_pk* pk, int mode, const int8_t* dX, const int8_t* dW, const uint8_t rs[64], void* stream,
                     uint32_t tuning[ZKVC_PK_TUNING_LEN]) {
  set_error("%s", "");
  ZK_CHECK(pk && dX && dW && rs, ZKVC_EINVAL, "autotune: null argument");
  ZK_CHECK(!pk->gen, ZKVC_EINVAL, "autotune: keys of zkvc_setup_circuit are not tuned");
  const bool fresh = (mode & ZKVC_TUNE_FRESH) != 0;
  mode &= ~ZKVC_TUNE_FRESH;
  ZK_CHECK(mode == ZKVC_PROVE_FOLD || mode == ZKVC_PROVE_CHAIN || mode == ZKVC_PROVE_AUTO, ZKVC_EINVAL,
           "autotune: mode %d", mode);
  ZK_TRY(device_guard(pk->device));
  TuneKey key;
  ZK_TRY(tune_key(pk, mode, &key));
  uint32_t t[ZKVC_PK_TUNING_LEN];
  if (!fresh && tune_cache_get(key, t)) {
    for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) pk->prove_tune[i] = t[i];
    if (tuning)
      for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) tuning[i] = t[i];
    return ZKVC_OK;
  }
  ZK_TRY(prove_autotune(pk, mode, dX, dW, rs, (cudaStream_t)stream, t));
  tune_cache_put(key, t);
  if (tuning)
    for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) tuning[i] = t[i];
  return ZKVC_OK;
}

int zkvc_tune_cache_save(const char* path) {
  set_error("%s", "");
  ZK_CHECK(path, ZKVC_EINVAL, "tune_cache_save: null path");
  return tune_cache_save(path);
}

int zkvc_tune_cache_load(const char* path) {
  set_error("%s", "");
  ZK_CHECK(path, ZKVC_EINVAL, "tune_cache_load: null path");
  return tune_cache_load(path);
}

int zkvc_tune_cache_clear(void) {
  set_error("%s", "");
  tune_cache_clear();
  return ZKVC_OK;
}

int zkvc_pk_set_tuning(zkvc_pk* pk, const uint32_t tuning[ZKVC_PK_TUNING_LEN]) {
  set_error("%s", "");
  ZK_CHECK(pk && tuning, ZKVC_EINVAL, "set_tuning: null argument");
  for (int i = 0; i < 4; i++)
    ZK_CHECK(tuning[i] <= 1024, ZKVC_EINVAL, "set_tuning: chunk %u above 1024", tuning[i]);
  ZK_CHECK(tuning[4] == 0 || (tuning[4] >= 8 && tuning[4] <= 11), ZKVC_EINVAL,
           "set_tuning: 2^%u NTT elements per block outside [2^8, 2^11]", tuning[4]);
  ZK_CHECK(tuning[5] <= 2, ZKVC_EINVAL, "set_tuning: rest-MSM start %u outside 0..2", tuning[5]);
  ZK_CHECK(tuning[6] <= 1, ZKVC_EINVAL, "set_tuning: prover mode %u is neither fold (0) nor chain (1)", tuning[6]);
  ZK_CHECK(tuning[7] <= 1, ZKVC_EINVAL, "set_tuning: G2 start %u outside 0..1", tuning[7]);
  ZK_CHECK(tuning[8] <= 1 && tuning[9] <= 1, ZKVC_EINVAL, "set_tuning: quad flags %u, %u outside 0..1", tuning[8],
           tuning[9]);
  for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) pk->prove_tune[i] = tuning[i];
  return ZKVC_OK;
}

int zkvc_pk_get_tuning(const zkvc_pk* pk, uint32_t tuning[ZKVC_PK_TUNING_LEN]) {
  set_error("%s", "");
  ZK_CHECK(pk && tuning, ZKVC_EINVAL, "get_tuning: null argument");
  for (int i = 0; i < ZKVC_PK_TUNING_LEN; i++) tuning[i] = pk->prove_tune[i];
  return ZKVC_OK;
}

int zkvc_pk_circuit(const zkvc_pk* pk, int* circuit, int* public_io, uint64_t* rows, uint64_t* vars) {
  set_error("%s", "");
  ZK_CHECK(pk, ZKVC_EINVAL, "pk_circuit: null key");
  if (pk->gen) {
    const GShape& g = pk->gen->sh;
    if (circuit) *circuit = g.circuit;
    if (public_io) *public_io = g.pub;
    if (rows) *rows = g.n_rows;
    if (vars) *vars = g.n_vars;
  } else {
    if (circuit) *circuit = ZKVC_CIRCUIT_CRPC_PSQ;
    if (public_io) *public_io = ZKVC_PUBLIC_XY;
    if (rows) *rows = pk->shape.rows;
    if (vars) *vars = pk->shape.n_vars;
  }
  return ZKVC_OK;
}

void zkvc_vk_free(zkvc_vk* vk) { delete vk; }

int zkvc_pk_info(const zkvc_pk* pk, int* a, int* n, int* b, uint32_t* log_domain, size_t* g1_bases,
                 size_t* g2_bases) {
  set_error("%s", "");
  ZK_CHECK(pk, ZKVC_EINVAL, "pk_info: null key");
  if (a) *a = pk->shape.a;
  if (n) *n = pk->shape.n;
  if (b) *b = pk->shape.b;
  if (log_domain) *log_domain = pk->shape.logN;
  if (g1_bases) *g1_bases = pk->lay.n_g1;
  if (g2_bases) *g2_bases = pk->lay.n_g2;
  return ZKVC_OK;
}

int zkvc_pk_export(const zkvc_pk* pk, int query, size_t start, size_t count, uint8_t* out) {
  set_error("%s", "");
  ZK_CHECK(pk && (out || count == 0), ZKVC_EINVAL, "pk_export: null argument");
  ZK_TRY(device_guard(pk->device));
  if (pk->gen) return export_generic(pk, query, start, count, out);
  const Shape& sh = pk->shape;
  const Region* g = pk->lay.g1;
  const Region* g2 = pk->lay.g2;
  const uint64_t nb = uint64_t(sh.n) * sh.b;
  uint64_t total = 0;
  switch (query) {
    case ZKVC_Q_A: total = sh.l + 1; break;
    case ZKVC_Q_B1:
    case ZKVC_Q_B2: total = nb; break;
    case ZKVC_Q_L: total = nb + sh.n - 1; break;
    case ZKVC_Q_H: total = sh.N - 1; break;
    case ZKVC_Q_ALPHA1: case ZKVC_Q_BETA1: case ZKVC_Q_BETA2: case ZKVC_Q_DELTA1: case ZKVC_Q_DELTA2: total = 1; break;
    default: ZK_CHECK(false, ZKVC_EINVAL, "pk_export: unknown query %d", query);
  }
  ZK_CHECK(start <= total && count <= total - start, ZKVC_EINVAL, "pk_export: range [%zu, %zu) outside %llu entries",
           start, start + count, (unsigned long long)total);
  std::vector<uint64_t> idx(count);
  for (size_t q = 0; q < count; q++) {
    uint64_t e = start + q;
    uint64_t o = 0;
    switch (query) {
      case ZKVC_Q_A: o = g[R1_A].off + e * g[R1_A].nwin; break;
      case ZKVC_Q_B1: o = g[R1_B].off + e * g[R1_B].nwin; break;
      case ZKVC_Q_B2: o = g2[R2_B].off + e; break;
      case ZKVC_Q_L: o = e < nb ? g[R1_LW].off + e : g[R1_LS].off + (e - nb) * g[R1_LS].nwin; break;
      case ZKVC_Q_H: {
        uint32_t p = 0;
        for (uint32_t bit = 0; bit < sh.logN; bit++) p |= ((uint32_t)(e >> bit) & 1u) << (sh.logN - 1 - bit);
        o = g[R1_H].off + uint64_t(p) * g[R1_H].nwin;
        break;
      }
      case ZKVC_Q_ALPHA1: o = g[R1_ALPHA].off; break;
      case ZKVC_Q_BETA1: o = g[R1_BETA].off; break;
      case ZKVC_Q_DELTA1: o = g[R1_DELTA].off; break;
      case ZKVC_Q_BETA2: o = g2[R2_BETA].off; break;
      case ZKVC_Q_DELTA2: o = g2[R2_DELTA].off; break;
    }
    idx[q] = o;
  }
  bool is_g2 = query == ZKVC_Q_B2 || query == ZKVC_Q_BETA2 || query == ZKVC_Q_DELTA2;
  if (is_g2) return export_points<Fp2>(pk->g2, idx, out, 0);
  return export_points<Fp>(pk->g1, idx, out, 0);
}

int zkvc_vk_info(const zkvc_vk* vk, int* a, int* n, int* b) {
  set_error("%s", "");
  ZK_CHECK(vk, ZKVC_EINVAL, "vk_info: null key");
  if (a) *a = vk->shape.a;
  if (n) *n = vk->shape.n;
  if (b) *b = vk->shape.b;
  return ZKVC_OK;
}

int zkvc_vk_export(const zkvc_vk* vk, int query, size_t start, size_t count, uint8_t* out) {
  set_error("%s", "");
  ZK_CHECK(vk && (out || count == 0), ZKVC_EINVAL, "vk_export: null argument");
  const std::vector<uint8_t>* src = nullptr;
  size_t width = 64;
  switch (query) {
    case ZKVC_VK_IC: src = &vk->ic; break;
    case ZKVC_VK_ALPHA1: src = &vk->alpha1; break;
    case ZKVC_VK_BETA2: src = &vk->beta2; width = 128; break;
    case ZKVC_VK_GAMMA2: src = &vk->gamma2; width = 128; break;
    case ZKVC_VK_DELTA2: src = &vk->delta2; width = 128; break;
    default: ZK_CHECK(false, ZKVC_EINVAL, "vk_export: unknown query %d", query);
  }
  size_t total = src->size() / width;
  ZK_CHECK(start <= total && count <= total - start, ZKVC_EINVAL, "vk_export: range outside %zu entries", total);
  memcpy(out, src->data() + start * width, count * width);
  return ZKVC_OK;
}

int zkvc_vk_import(int a, int n, int b, const uint8_t alpha1[64], const uint8_t beta2[128], const uint8_t gamma2[128],
                   const uint8_t delta2[128], const uint8_t* ic, size_t n_ic, zkvc_vk** vk) {
  set_error("%s", "");
  ZK_CHECK(alpha1 && beta2 && gamma2 && delta2 && ic && vk, ZKVC_EINVAL, "vk_import: null argument");
  Shape sh;
  ZK_TRY(make_shape(a, n, b, &sh));
  ZK_CHECK(n_ic == size_t(sh.l) + 1, ZKVC_EINVAL, "vk_import: %zu IC points for %u public inputs", n_ic, sh.l);
  zkvc_vk* v = new zkvc_vk();
  v->shape = sh;
  v->alpha1.assign(alpha1, alpha1 + 64);
  v->beta2.assign(beta2, beta2 + 128);
  v->gamma2.assign(gamma2, gamma2 + 128);
  v->delta2.assign(delta2, delta2 + 128);
  v->ic.assign(ic, ic + 64 * n_ic);
  *vk = v;
  return ZKVC_OK;
}

int zkvc_verify(const zkvc_vk* vk, const int8_t* X, const int32_t* Y, const uint8_t proof[256], int* ok) {
  set_error("%s", "");
  ZK_CHECK(vk && proof && ok, ZKVC_EINVAL, "verify: null argument");
  ZK_CHECK((X && Y) || vk->ic.size() == 64, ZKVC_EINVAL, "verify: X and Y are public inputs of this key");
  return verify_impl(vk, X, Y, proof, ok);
}

int zkvc_pk_save(const zkvc_pk* pk, const char* path) {
  set_error("%s", "");
  ZK_CHECK(pk && path, ZKVC_EINVAL, "pk_save: null argument");
  ZK_CHECK(!pk->gen, ZKVC_EINVAL, "pk_save: keys of zkvc_setup_circuit are not saved to files");
  ZK_TRY(device_guard(pk->device));
  ZK_CUDA(cudaDeviceSynchronize());
  FileGuard g;
  g.f = fopen(path, "wb");
  ZK_CHECK(g.f, ZKVC_EIO, "pk_save: cannot open %s", path);
  const Shape& sh = pk->shape;
  int32_t dims[3] = {sh.a, sh.n, sh.b};
  uint64_t counts[2] = {pk->lay.n_g1, pk->lay.n_g2};
  uint32_t hdr[2] = {KEY_VERSION, 0};
  ZK_CHECK(wr(g.f, PK_MAGIC, 8, nullptr) && wr(g.f, hdr, 8, nullptr) && wr(g.f, dims, 12, nullptr) &&
               wr(g.f, &sh.logN, 4, nullptr) && wr(g.f, counts, 16, nullptr),
           ZKVC_EIO, "pk_save: write failed");
  Fnv h;
  ZK_TRY(dev_to_file(g.f, pk->g1, pk->lay.n_g1 * sizeof(G1A), &h));
  ZK_TRY(dev_to_file(g.f, pk->g2, pk->lay.n_g2 * sizeof(G2A), &h));
  ZK_TRY(dev_to_file(g.f, pk->zA, size_t(sh.a) * sizeof(Fr), &h));
  ZK_TRY(dev_to_file(g.f, pk->zB, size_t(sh.b) * sizeof(Fr), &h));
  ZK_CHECK(wr(g.f, &h.h, 8, nullptr), ZKVC_EIO, "pk_save: write failed");
  ZK_CHECK(fflush(g.f) == 0, ZKVC_EIO, "pk_save: flush failed");
  return ZKVC_OK;
}

int zkvc_pk_load(const char* path, void* stream, zkvc_pk** out) {
  set_error("%s", "");
  ZK_CHECK(path && out, ZKVC_EINVAL, "pk_load: null argument");
  (void)stream;
  *out = nullptr;
  FileGuard g;
  g.f = fopen(path, "rb");
  ZK_CHECK(g.f, ZKVC_EIO, "pk_load: cannot open %s", path);
  char magic[8];
  uint32_t hdr[2], logN;
  int32_t dims[3];
  uint64_t counts[2];
  ZK_CHECK(rd(g.f, magic, 8, nullptr) && memcmp(magic, PK_MAGIC, 8) == 0, ZKVC_EIO, "pk_load: not a proving-key file");
  ZK_CHECK(rd(g.f, hdr, 8, nullptr) && hdr[0] == KEY_VERSION, ZKVC_EIO, "pk_load: unsupported version");
  ZK_CHECK(rd(g.f, dims, 12, nullptr) && rd(g.f, &logN, 4, nullptr) && rd(g.f, counts, 16, nullptr), ZKVC_EIO,
           "pk_load: truncated header");
  Shape sh;
  ZK_CHECK(make_shape(dims[0], dims[1], dims[2], &sh) == ZKVC_OK, ZKVC_EIO, "pk_load: bad shape in header");
  Layout lay = make_layout(sh);
  ZK_CHECK(sh.logN == logN && lay.n_g1 == counts[0] && lay.n_g2 == counts[1], ZKVC_EIO,
           "pk_load: header does not match the layout of this library version");
  zkvc_pk* pk = new zkvc_pk();
  pk->shape = sh;
  pk->lay = lay;
  int rc = ntt_domain(sh.logN, &pk->dom);
  if (rc == ZKVC_OK) rc = cudaGetDevice(&pk->device) == cudaSuccess ? ZKVC_OK : ZKVC_ECUDA;
  if (rc == ZKVC_OK && (cudaMalloc(&pk->g1, lay.n_g1 * sizeof(G1A)) != cudaSuccess ||
                        cudaMalloc(&pk->g2, lay.n_g2 * sizeof(G2A)) != cudaSuccess ||
                        cudaMalloc(&pk->zA, sh.a * sizeof(Fr)) != cudaSuccess ||
                        cudaMalloc(&pk->zB, sh.b * sizeof(Fr)) != cudaSuccess)) {
    set_error("pk_load: device allocation failed");
    rc = ZKVC_ENOMEM;
  }
  Fnv h;
  if (rc == ZKVC_OK) rc = file_to_dev(g.f, pk->g1, lay.n_g1 * sizeof(G1A), &h);
  if (rc == ZKVC_OK) rc = file_to_dev(g.f, pk->g2, lay.n_g2 * sizeof(G2A), &h);
  if (rc == ZKVC_OK) rc = file_to_dev(g.f, pk->zA, size_t(sh.a) * sizeof(Fr), &h);
  if (rc == ZKVC_OK) rc = file_to_dev(g.f, pk->zB, size_t(sh.b) * sizeof(Fr), &h);
  uint64_t sum = 0;
  if (rc == ZKVC_OK && !(rd(g.f, &sum, 8, nullptr) && sum == h.h)) {
    set_error("pk_load: checksum mismatch (corrupt file)");
    rc = ZKVC_EIO;
  }
  if (rc != ZKVC_OK) {
    zkvc_pk_free(pk);
    return rc;
  }
  *out = pk;
  return ZKVC_OK;
}

int zkvc_vk_save(const zkvc_vk* vk, const char* path) {
  set_error("%s", "");
  ZK_CHECK(vk && path, ZKVC_EINVAL, "vk_save: null argument");
  FileGuard g;
  g.f = fopen(path, "wb");
  ZK_CHECK(g.f, ZKVC_EIO, "vk_save: cannot open %s", path);
  int32_t dims[3] = {vk->shape.a, vk->shape.n, vk->shape.b};
  uint64_t n_ic = vk->ic.size() / 64;
  uint32_t hdr[2] = {KEY_VERSION, 0};
  Fnv h;
  bool ok = wr(g.f, VK_MAGIC, 8, nullptr) && wr(g.f, hdr, 8, nullptr) && wr(g.f, dims, 12, nullptr) &&
            wr(g.f, &n_ic, 8, nullptr) && wr(g.f, vk->alpha1.data(), 64, &h) && wr(g.f, vk->beta2.data(), 128, &h) &&
            wr(g.f, vk->gamma2.data(), 128, &h) && wr(g.f, vk->delta2.data(), 128, &h) &&
            wr(g.f, vk->ic.data(), vk->ic.size(), &h) && wr(g.f, &h.h, 8, nullptr);
  ZK_CHECK(ok && fflush(g.f) == 0, ZKVC_EIO, "vk_save: write failed");
  return ZKVC_OK;
}

int zkvc_vk_load(const char* path, zkvc_vk** out) {
  set_error("%s", "");
  ZK_CHECK(path && out, ZKVC_EINVAL, "vk_load: null argument");
  *out = nullptr;
  FileGuard g;
  g.f = fopen(path, "rb");
  ZK_CHECK(g.f, ZKVC_EIO, "vk_load: cannot open %s", path);
  char magic[8];
  uint32_t hdr[2];
  int32_t dims[3];
  uint64_t n_ic = 0;
  ZK_CHECK(rd(g.f, magic, 8, nullptr) && memcmp(magic, VK_MAGIC, 8) == 0, ZKVC_EIO, "vk_load: not a verifying-key file");
  ZK_CHECK(rd(g.f, hdr, 8, nullptr) && hdr[0] == KEY_VERSION, ZKVC_EIO, "vk_load: unsupported version");
  ZK_CHECK(rd(g.f, dims, 12, nullptr) && rd(g.f, &n_ic, 8, nullptr), ZKVC_EIO, "vk_load: truncated header");
  Shape sh;
  ZK_CHECK(make_shape(dims[0], dims[1], dims[2], &sh) == ZKVC_OK && n_ic == uint64_t(sh.l) + 1, ZKVC_EIO,
           "vk_load: inconsistent header");
  zkvc_vk* vk = new zkvc_vk();
  vk->shape = sh;
  vk->alpha1.resize(64);
  vk->beta2.resize(128);
  vk->gamma2.resize(128);
  vk->delta2.resize(128);
  vk->ic.resize(n_ic * 64);
  Fnv h;
  uint64_t sum = 0;
  bool ok = rd(g.f, vk->alpha1.data(), 64, &h) && rd(g.f, vk->beta2.data(), 128, &h) &&
            rd(g.f, vk->gamma2.data(), 128, &h) && rd(g.f, vk->delta2.data(), 128, &h) &&
            rd(g.f, vk->ic.data(), vk->ic.size(), &h) && rd(g.f, &sum, 8, nullptr) && sum == h.h;
  if (!ok) {
    delete vk;
    set_error("vk_load: truncated or corrupt file");
    return ZKVC_EIO;
  }
  *out = vk;
  return ZKVC_OK;
}

size_t zkvc_prove_workspace_bytes(const zkvc_pk* pk) {
  if (!pk) return 0;
  return pk->gen ? prove_generic_workspace_bytes(pk) : prove_workspace_bytes(pk, (int)pk->prove_tune[6]);
}

size_t zkvc_prove_workspace_bytes_mode(const zkvc_pk* pk, int mode) {
  if (!pk || (mode != ZKVC_PROVE_FOLD && mode != ZKVC_PROVE_CHAIN)) return 0;
  return pk->gen ? prove_generic_workspace_bytes(pk) : prove_workspace_bytes(pk, mode);
}

int zkvc_prove(const zkvc_pk* pk, const int8_t* dX, const int8_t* dW, const uint8_t rs[64], int32_t* dY, void* d_ws,
               size_t ws_bytes, uint8_t proof[256], void* stream) {
  set_error("%s", "");
  ZK_CHECK(pk, ZKVC_EINVAL, "prove: null key");
  ZK_TRY(device_guard(pk->device));
  if (pk->gen) return prove_generic(pk, dX, dW, rs, dY, d_ws, ws_bytes, proof, (cudaStream_t)stream);
  return prove_graph(pk, (int)pk->prove_tune[6], dX, dW, rs, dY, d_ws, ws_bytes, proof, (cudaStream_t)stream);
}

int zkvc_prove_claimed(const zkvc_pk* pk, const int8_t* dX, const int8_t* dW, const int32_t* dY_claimed,
                       const uint8_t rs[64], void* d_ws, size_t ws_bytes, uint8_t proof[256], void* stream) {
  set_error("%s", "");
  ZK_CHECK(pk && dY_claimed, ZKVC_EINVAL, "prove_claimed: null key or claimed Y");
  ZK_TRY(device_guard(pk->device));
  if (pk->gen)
    return prove_generic(pk, dX, dW, rs, const_cast<int32_t*>(dY_claimed), d_ws, ws_bytes, proof,
                         (cudaStream_t)stream, true);
  return prove_claimed(pk, (int)pk->prove_tune[6], dX, dW, rs, dY_claimed, d_ws, ws_bytes, proof, (cudaStream_t)stream);
}

int zkvc_prove_mode(const zkvc_pk* pk, int mode, const int8_t* dX, const int8_t* dW, const uint8_t rs[64], int32_t* dY,
                    void* d_ws, size_t ws_bytes, uint8_t proof[256], void* stream) {
  set_error("%s", "");
  ZK_CHECK(pk, ZKVC_EINVAL, "prove: null key");
  ZK_TRY(device_guard(pk->device));
  if (pk->gen) {
    ZK_CHECK(mode == ZKVC_PROVE_FOLD || mode == ZKVC_PROVE_CHAIN, ZKVC_EINVAL, "prove: mode %d", mode);
    return prove_generic(pk, dX, dW, rs, dY, d_ws, ws_bytes, proof, (cudaStream_t)stream);
  }
  return prove_graph(pk, mode, dX, dW, rs, dY, d_ws, ws_bytes, proof, (cudaStream_t)stream);
}

}  // extern "C"
