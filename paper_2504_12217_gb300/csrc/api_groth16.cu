// C-ABI entry points of the Groth16 layer: setup, prove, key export and release.
#include <cstring>

#include "groth16.h"

namespace zkvc {
int setup_impl(int a, int n, int b, const uint8_t* toxic, cudaStream_t st, zkvc_pk** pk, zkvc_vk** vk);
size_t prove_workspace_bytes(const zkvc_pk* pk);
int prove_impl(const zkvc_pk* pk, const int8_t* dX, const int8_t* dW, const uint8_t* rs, int32_t* dY, void* ws,
               size_t ws_bytes, uint8_t* proof, cudaStream_t st);
template <class F>
int export_points(const Affine<F>* src, const std::vector<uint64_t>& idx, uint8_t* host_out, cudaStream_t st);

int verify_impl(const zkvc_vk* vk, const int8_t* X, const int32_t* Y, const uint8_t* proof, int* ok);

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

static int device_guard(int dev) {
  int cur = -1;
  ZK_CUDA(cudaGetDevice(&cur));
  ZK_CHECK(cur == dev, ZKVC_EINVAL, "key was built on device %d but device %d is current", dev, cur);
  return ZKVC_OK;
}
}  // namespace zkvc

using namespace zkvc;

extern "C" {

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
  delete pk;
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
  ZK_CHECK(vk && X && Y && proof && ok, ZKVC_EINVAL, "verify: null argument");
  return verify_impl(vk, X, Y, proof, ok);
}

size_t zkvc_prove_workspace_bytes(const zkvc_pk* pk) { return pk ? prove_workspace_bytes(pk) : 0; }

int zkvc_prove(const zkvc_pk* pk, const int8_t* dX, const int8_t* dW, const uint8_t rs[64], int32_t* dY, void* d_ws,
               size_t ws_bytes, uint8_t proof[256], void* stream) {
  set_error("%s", "");
  ZK_CHECK(pk, ZKVC_EINVAL, "prove: null key");
  ZK_TRY(device_guard(pk->device));
  return prove_impl(pk, dX, dW, rs, dY, d_ws, ws_bytes, proof, (cudaStream_t)stream);
}

}  // extern "C"
