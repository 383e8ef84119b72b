// Groth16 verification on the GPU (zkVC Sec. II: Verify), batched over many proofs:
//
//   e(A, B) = e(alpha, beta) e(IC(x), gamma) e(C, delta),  IC(x) = IC_0 + sum_v x_v IC_v,
//
// checked as e(-A, B) e(alpha, beta) e(IC(x), gamma) e(C, delta) = 1 with one shared final
// exponentiation per proof.  IC(x) for every proof comes from one merged multi-output MSM
// (each output reads its own verifying key's IC points; X int8 and Y int32 scalars in 8-bit
// windows); each (proof, pair) gets a thread for its Miller loop; a last kernel multiplies a
// proof's four Miller values and runs the final exponentiation.  Proof points are checked
// as the host verifier checks them: canonical coordinates, on the curve, and B in the
// order-r subgroup ([r] B = O, a 254-bit multiplication on the twist).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "groth16.h"
#include "msm.h"
#include "pairing.cuh"

namespace zkvc {

__device__ __forceinline__ Fp2 f2_pow(Fp2 x, const uint32_t (&e)[8]) {
  Fp2 r = Fp2::one();
  for (int i = 7; i >= 0; i--)
    for (int bit = 31; bit >= 0; bit--) {
      r = f_sqr(r);
      if ((e[i] >> bit) & 1u) r = f_mul(r, x);
    }
  return r;
}

// gam[k-1][m] = xi^(m (p^k - 1)/6): xi^((p-1)/6) by exponentiation, the rest by conjugation
__global__ void k_frob_init(FrobTab* T) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t m[8], e[8];
#pragma unroll
  for (int i = 0; i < 8; i++) m[i] = mod_limb<FpCfg>(i);
  m[0] -= 1;  // p - 1 (p odd)
  uint64_t rem = 0;
  for (int i = 7; i >= 0; i--) {
    uint64_t cur = (rem << 32) | m[i];
    e[i] = (uint32_t)(cur / 6);
    rem = cur % 6;
  }
  Fp2 xi{f_from_int<FpCfg>(9), f_from_int<FpCfg>(1)};
  Fp2 g1 = f2_pow(xi, e);
  Fp2 g2 = f_mul(g1, f2_conj(g1));               // xi^((p^2 - 1)/6) = g1^(p + 1)
  Fp2 g3 = f_mul(f_mul(g1, g1), f2_conj(g1));    // xi^((p^3 - 1)/6) = g1^(p^2 + p + 1)
  const Fp2 base[3] = {g1, g2, g3};
  for (int k = 0; k < 3; k++) {
    Fp2 acc = Fp2::one();
    for (int j = 0; j < 6; j++) {
      T->g[k][j] = acc;
      acc = f_mul(acc, base[k]);
    }
  }
}

static std::mutex g_frob_mu;
static std::map<int, FrobTab*> g_frob;

static int frob_table(const FrobTab** out, cudaStream_t st) {
  int dev = 0;
  ZK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_frob_mu);
  auto it = g_frob.find(dev);
  if (it == g_frob.end()) {
    FrobTab* T = nullptr;
    ZK_CUDA(cudaMalloc(&T, sizeof(FrobTab)));
    k_frob_init<<<1, 1, 0, st>>>(T); ZK_COUNT_LAUNCH();
    ZK_CUDA(cudaGetLastError());
    ZK_CUDA(cudaStreamSynchronize(st));
    it = g_frob.emplace(dev, T).first;
  }
  *out = it->second;
  return ZKVC_OK;
}

__device__ __forceinline__ bool canon_fp(const Fp& x) {
  for (int i = 7; i >= 0; i--) {
    uint32_t m = mod_limb<FpCfg>(i);
    if (x.v[i] != m) return x.v[i] < m;
  }
  return false;
}

__device__ __forceinline__ Fp ld_canon(const uint8_t* p) {
  Fp x;
#pragma unroll
  for (int i = 0; i < 8; i++)
    x.v[i] = (uint32_t)p[4 * i] | ((uint32_t)p[4 * i + 1] << 8) | ((uint32_t)p[4 * i + 2] << 16) |
             ((uint32_t)p[4 * i + 3] << 24);
  return x;
}

__device__ __forceinline__ void st_canon(uint8_t* out, const Fp& x) {
  Fp c = f_from_mont(x);
#pragma unroll
  for (int i = 0; i < 8; i++) {
    out[4 * i] = (uint8_t)c.v[i];
    out[4 * i + 1] = (uint8_t)(c.v[i] >> 8);
    out[4 * i + 2] = (uint8_t)(c.v[i] >> 16);
    out[4 * i + 3] = (uint8_t)(c.v[i] >> 24);
  }
}

// canonical bytes -> Montgomery point; *ok = 0 for a coordinate >= p
__device__ __forceinline__ G1A ld_g1(const uint8_t* p, int* ok) {
  Fp x = ld_canon(p), y = ld_canon(p + 32);
  if (!canon_fp(x) || !canon_fp(y)) *ok = 0;
  return {f_to_mont(x), f_to_mont(y)};
}
__device__ __forceinline__ G2A ld_g2(const uint8_t* p, int* ok) {
  Fp a = ld_canon(p), b = ld_canon(p + 32), c = ld_canon(p + 64), d = ld_canon(p + 96);
  if (!canon_fp(a) || !canon_fp(b) || !canon_fp(c) || !canon_fp(d)) *ok = 0;
  return {{f_to_mont(a), f_to_mont(b)}, {f_to_mont(c), f_to_mont(d)}};
}

__device__ __forceinline__ void st_f12(uint8_t* out, const Fp12& f) {
  const Fp2* c[6] = {&f.c0.c0, &f.c0.c1, &f.c0.c2, &f.c1.c0, &f.c1.c1, &f.c1.c2};
  for (int j = 0; j < 6; j++) {
    st_canon(out + 64 * j, c[j]->c0);
    st_canon(out + 64 * j + 32, c[j]->c1);
  }
}

// e(P_i, Q_i) for canonical points; out: 12 canonical Fp coefficients per pairing in tower
// order (c0.c0, c0.c1, c0.c2, c1.c0, c1.c1, c1.c2; each Fp2 as c0 then c1)
__global__ void __launch_bounds__(64) k_pairing(const uint8_t* __restrict__ P, const uint8_t* __restrict__ Q, size_t n,
                                                const FrobTab* __restrict__ T, uint8_t* out) {
  size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int ok = 1;
  G1A p = ld_g1(P + 64 * i, &ok);
  G2A q = ld_g2(Q + 128 * i, &ok);
  FrobTab t = *T;
  st_f12(out + 384 * i, final_exp(miller_loop(p, q, t), t));
}

// ------------------------------------------------------------------ batched verification
struct VkDev {
  G1A alpha1;  // Montgomery
  G2A beta2, gamma2, delta2;
  const G1A* ic;  // l + 1 points (Montgomery)
  uint32_t l;
};

struct VfyItem {
  G1A P[4];
  G2A Q[4];
  int ok;
};

__global__ void k_vfy_load(const uint8_t* __restrict__ proofs, const int* __restrict__ vk_of, const VkDev* __restrict__ vks,
                           int count, VfyItem* items) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const uint8_t* pr = proofs + 256 * size_t(t);
  int ok = 1;
  G1A A = ld_g1(pr, &ok);
  G2A B = ld_g2(pr + 64, &ok);
  G1A C = ld_g1(pr + 192, &ok);
  if (ok && (!p_on_curve(A, g1_b()) || !p_on_curve(C, g1_b()) || !p_on_curve(B, g2_b()))) ok = 0;
  const VkDev& vk = vks[vk_of[t]];
  VfyItem it;
  it.P[0] = p_neg(A);
  it.Q[0] = B;
  it.P[1] = vk.alpha1;
  it.Q[1] = vk.beta2;
  it.P[2] = G1A::inf();  // IC(x), below
  it.Q[2] = vk.gamma2;
  it.P[3] = C;
  it.Q[3] = vk.delta2;
  it.ok = ok;
  items[t] = it;
}

// IC(x) = IC_0 + msm (msm_out null: no public inputs)
__global__ void k_vfy_ic(const int* __restrict__ vk_of, const VkDev* __restrict__ vks, const int* __restrict__ msm_slot,
                         const G1J* __restrict__ msm_out, int count, VfyItem* items) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const VkDev& vk = vks[vk_of[t]];
  G1J acc = G1J::from_affine(ld_field(vk.ic));
  if (msm_slot[t] >= 0) acc = p_add(acc, ld_field(msm_out + msm_slot[t]));
  items[t].P[2] = p_to_affine(acc);
}

// B in the order-r subgroup: [r] B = O
__global__ void __launch_bounds__(64) k_vfy_subgroup(int count, VfyItem* items) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  G2A B = items[t].Q[0];
  if (B.is_inf() || !items[t].ok) return;
  uint32_t r[8];
#pragma unroll
  for (int i = 0; i < 8; i++) r[i] = mod_limb<FrCfg>(i);
  if (!p_mul_scalar_w4(G2J::from_affine(B), r).is_inf()) items[t].ok = 0;
}

__global__ void __launch_bounds__(64) k_vfy_miller(const VfyItem* __restrict__ items, int count,
                                                   const FrobTab* __restrict__ T, Fp12* f) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * count) return;
  const int i = t >> 2, k = t & 3;
  FrobTab tab = *T;
  f[t] = items[i].ok ? miller_loop(items[i].P[k], items[i].Q[k], tab) : f12_one();
}

__global__ void __launch_bounds__(64) k_vfy_final(const VfyItem* __restrict__ items, const Fp12* __restrict__ f, int count,
                                                  const FrobTab* __restrict__ T, int* ok) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  if (!items[t].ok) {
    ok[t] = 0;
    return;
  }
  FrobTab tab = *T;
  Fp12 g = f12_mul(f12_mul(f[4 * t], f[4 * t + 1]), f12_mul(f[4 * t + 2], f[4 * t + 3]));
  ok[t] = f12_is_one(final_exp(g, tab)) ? 1 : 0;
}

__global__ void k_canon_to_mont_g1(G1A* p, size_t n) {
  size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  G1A a = ld_field(p + i);
  a.x = f_to_mont(a.x);
  a.y = f_to_mont(a.y);
  st_field(p + i, a);
}

__global__ void k_vk_points(const uint8_t* __restrict__ raw, int nvk, VkDev* vks) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nvk) return;
  const uint8_t* r = raw + size_t(t) * (64 + 3 * 128);
  int ok = 1;
  vks[t].alpha1 = ld_g1(r, &ok);
  vks[t].beta2 = ld_g2(r + 64, &ok);
  vks[t].gamma2 = ld_g2(r + 192, &ok);
  vks[t].delta2 = ld_g2(r + 320, &ok);
}

struct DevBuf {
  std::vector<void*> p;
  ~DevBuf() {
    for (void* x : p) cudaFree(x);
  }
  template <class T>
  int get(T** out, size_t count) {
    if (cudaMalloc(out, std::max<size_t>(1, count) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      set_error("verify: cannot allocate %zu bytes", count * sizeof(T));
      return ZKVC_ENOMEM;
    }
    p.push_back(*out);
    return ZKVC_OK;
  }
};

int verify_batch_impl(const zkvc_vk* const* vks, const int8_t* const* X, const int32_t* const* Y, const uint8_t* proofs,
                      int count, int* ok, cudaStream_t st) {
  ZK_CHECK(vks && proofs && ok && count >= 0, ZKVC_EINVAL, "verify_batch: null argument");
  if (count == 0) return ZKVC_OK;
  const FrobTab* T = nullptr;
  ZK_TRY(frob_table(&T, st));
  // distinct verifying keys
  std::vector<const zkvc_vk*> uniq;
  std::map<const zkvc_vk*, int> idx;
  std::vector<int> vk_of(count);
  for (int i = 0; i < count; i++) {
    const zkvc_vk* v = vks[i];
    ZK_CHECK(v && v->alpha1.size() == 64 && v->beta2.size() == 128 && v->gamma2.size() == 128 &&
                 v->delta2.size() == 128 && v->ic.size() % 64 == 0 && !v->ic.empty(),
             ZKVC_EIO, "verify_batch: malformed verifying key %d", i);
    const size_t l = v->ic.size() / 64 - 1;
    const size_t io = size_t(v->shape.a) * v->shape.n + size_t(v->shape.a) * v->shape.b;
    ZK_CHECK(l == 0 || l == io, ZKVC_EIO, "verify_batch: key %d has %zu IC points for shape (%d, %d, %d)", i, l + 1,
             v->shape.a, v->shape.n, v->shape.b);
    ZK_CHECK(l == 0 || (X && Y && X[i] && Y[i]), ZKVC_EINVAL, "verify_batch: proof %d needs X and Y", i);
    auto it = idx.find(v);
    if (it == idx.end()) {
      it = idx.emplace(v, (int)uniq.size()).first;
      uniq.push_back(v);
    }
    vk_of[i] = it->second;
  }
  DevBuf buf;
  const int nvk = (int)uniq.size();
  std::vector<uint8_t> raw(size_t(nvk) * 448);
  std::vector<VkDev> hvk(nvk);
  std::vector<G1A*> d_ic(nvk);
  for (int k = 0; k < nvk; k++) {
    const zkvc_vk* v = uniq[k];
    memcpy(raw.data() + 448 * k, v->alpha1.data(), 64);
    memcpy(raw.data() + 448 * k + 64, v->beta2.data(), 128);
    memcpy(raw.data() + 448 * k + 192, v->gamma2.data(), 128);
    memcpy(raw.data() + 448 * k + 320, v->delta2.data(), 128);
    size_t nic = v->ic.size() / 64;
    ZK_TRY(buf.get(&d_ic[k], nic));
    ZK_CUDA(cudaMemcpyAsync(d_ic[k], v->ic.data(), v->ic.size(), cudaMemcpyHostToDevice, st));
    k_canon_to_mont_g1<<<(unsigned)((nic + 255) / 256), 256, 0, st>>>(d_ic[k], nic); ZK_COUNT_LAUNCH();
  }
  uint8_t* d_raw = nullptr;
  VkDev* d_vk = nullptr;
  ZK_TRY(buf.get(&d_raw, raw.size()));
  ZK_TRY(buf.get(&d_vk, nvk));
  for (int k = 0; k < nvk; k++) {  // IC pointer and count from the host, points by the kernel below
    hvk[k] = VkDev{};
    hvk[k].ic = d_ic[k];
    hvk[k].l = (uint32_t)(uniq[k]->ic.size() / 64 - 1);
  }
  ZK_CUDA(cudaMemcpyAsync(d_vk, hvk.data(), nvk * sizeof(VkDev), cudaMemcpyHostToDevice, st));
  ZK_CUDA(cudaMemcpyAsync(d_raw, raw.data(), raw.size(), cudaMemcpyHostToDevice, st));
  k_vk_points<<<(nvk + 63) / 64, 64, 0, st>>>(d_raw, nvk, d_vk); ZK_COUNT_LAUNCH();
  // public inputs and the merged IC MSM (8-bit windows, 4 windows per output)
  MsmPlan plan;
  std::vector<int> slot(count, -1);
  size_t in_bytes = 0;
  for (int i = 0; i < count; i++)
    if (uniq[vk_of[i]]->ic.size() > 64) {
      const Shape& s = uniq[vk_of[i]]->shape;
      in_bytes += size_t(s.a) * s.n + 4 * size_t(s.a) * s.b + 512;
    }
  uint8_t* d_in = nullptr;
  ZK_TRY(buf.get(&d_in, in_bytes));
  size_t off = 0;
  for (int i = 0; i < count; i++) {
    const zkvc_vk* v = uniq[vk_of[i]];
    if (v->ic.size() == 64) continue;
    const Shape& s = v->shape;
    const size_t an = size_t(s.a) * s.n, ab = size_t(s.a) * s.b;
    int8_t* dx = reinterpret_cast<int8_t*>(d_in + off);
    off += (an + 255) & ~size_t(255);
    int32_t* dy = reinterpret_cast<int32_t*>(d_in + off);
    off += (4 * ab + 255) & ~size_t(255);
    ZK_CUDA(cudaMemcpyAsync(dx, X[i], an, cudaMemcpyHostToDevice, st));
    ZK_CUDA(cudaMemcpyAsync(dy, Y[i], 4 * ab, cudaMemcpyHostToDevice, st));
    const uint32_t o = (uint32_t)plan.outs.size();
    slot[i] = (int)o;
    plan.outs.push_back({8, 4, 0, 0, d_ic[vk_of[i]] + 1});
    MsmSeg sx{}, sy{};
    sx.base_off = 0;
    sx.count = (uint32_t)an;
    sx.nwin = 1;
    sx.out = o;
    sx.kind = SK_I8;
    sx.scalars = dx;
    sx.skip = 0xffffffffu;
    sy = sx;
    sy.base_off = an;
    sy.count = (uint32_t)ab;
    sy.kind = SK_I32;
    sy.scalars = dy;
    plan.segs.push_back(sx);
    plan.segs.push_back(sy);
  }
  G1J* d_msm = nullptr;
  if (!plan.outs.empty()) {
    ZK_TRY(msm_plan_finalize(plan));
    size_t wsb = msm_workspace_bytes<Fp>(plan);
    uint8_t* ws = nullptr;
    ZK_TRY(buf.get(&ws, wsb));
    ZK_TRY(buf.get(&d_msm, plan.outs.size()));
    ZK_TRY(msm_run<Fp>(plan, nullptr, ws, wsb, d_msm, st));
  }
  // points, IC, subgroup, Miller loops, final exponentiations
  uint8_t* d_proofs = nullptr;
  int *d_vk_of = nullptr, *d_slot = nullptr, *d_ok = nullptr;
  VfyItem* d_items = nullptr;
  Fp12* d_f = nullptr;
  ZK_TRY(buf.get(&d_proofs, size_t(count) * 256));
  ZK_TRY(buf.get(&d_vk_of, count));
  ZK_TRY(buf.get(&d_slot, count));
  ZK_TRY(buf.get(&d_ok, count));
  ZK_TRY(buf.get(&d_items, count));
  ZK_TRY(buf.get(&d_f, 4 * size_t(count)));
  ZK_CUDA(cudaMemcpyAsync(d_proofs, proofs, size_t(count) * 256, cudaMemcpyHostToDevice, st));
  ZK_CUDA(cudaMemcpyAsync(d_vk_of, vk_of.data(), count * sizeof(int), cudaMemcpyHostToDevice, st));
  ZK_CUDA(cudaMemcpyAsync(d_slot, slot.data(), count * sizeof(int), cudaMemcpyHostToDevice, st));
  const unsigned g = (unsigned)((count + 63) / 64);
  k_vfy_load<<<g, 64, 0, st>>>(d_proofs, d_vk_of, d_vk, count, d_items); ZK_COUNT_LAUNCH();
  k_vfy_ic<<<g, 64, 0, st>>>(d_vk_of, d_vk, d_slot, d_msm, count, d_items); ZK_COUNT_LAUNCH();
  k_vfy_subgroup<<<g, 64, 0, st>>>(count, d_items); ZK_COUNT_LAUNCH();
  k_vfy_miller<<<(unsigned)((4 * count + 63) / 64), 64, 0, st>>>(d_items, count, T, d_f); ZK_COUNT_LAUNCH();
  k_vfy_final<<<g, 64, 0, st>>>(d_items, d_f, count, T, d_ok); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  ZK_CUDA(cudaMemcpyAsync(ok, d_ok, count * sizeof(int), cudaMemcpyDeviceToHost, st));
  ZK_TRY(wait_stream(st, "verify_batch"));
  return ZKVC_OK;
}

int pairing_impl(const uint8_t* d_P, const uint8_t* d_Q, size_t n, uint8_t* d_out, cudaStream_t st) {
  if (n == 0) return ZKVC_OK;
  ZK_CHECK(d_P && d_Q && d_out, ZKVC_EINVAL, "pairing: null pointer");
  const FrobTab* T = nullptr;
  ZK_TRY(frob_table(&T, st));
  k_pairing<<<(unsigned)((n + 63) / 64), 64, 0, st>>>(d_P, d_Q, n, T, d_out); ZK_COUNT_LAUNCH();
  ZK_CUDA(cudaGetLastError());
  return ZKVC_OK;
}

}  // namespace zkvc

using namespace zkvc;

extern "C" {

int zkvc_pairing(const uint8_t* d_P, const uint8_t* d_Q, size_t n, uint8_t* d_out, void* stream) {
  set_error("%s", "");
  return pairing_impl(d_P, d_Q, n, d_out, (cudaStream_t)stream);
}

int zkvc_verify_batch(const zkvc_vk* const* vks, const int8_t* const* X, const int32_t* const* Y, const uint8_t* proofs,
                      int count, int* ok, void* stream) {
  set_error("%s", "");
  return verify_batch_impl(vks, X, Y, proofs, count, ok, (cudaStream_t)stream);
}

}  // extern "C"
