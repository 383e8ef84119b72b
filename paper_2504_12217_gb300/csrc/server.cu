// Proof server: continuous batching of CRPC Groth16 proof requests on one GPU.
//
// Requests (key index, X, W, r || s) arrive at any time and queue in arrival order.  A
// pool of worker threads, each with its own CUDA stream (and the prover's per-thread side
// streams), admits the head of the queue as soon as a worker is idle and the request's
// device footprint -- prove workspace plus X, W and Y -- fits in what is left of a fixed
// device-memory budget; requests in flight therefore overlap on the device (their kernels
// interleave across streams), and a finished request frees its slot and memory for the
// next one at once.  Proving keys stay resident; per-request state lives in one
// preallocated arena managed by a first-fit allocator, so serving allocates no device
// memory per request.  Every device wait is bounded (ZKVC_ETIMEOUT).
//
// Mode policy: a request admitted onto an otherwise idle GPU uses the fold prover
// (lowest latency); one admitted beside others uses the chain prover (about 2.5x less
// MSM work), which raises throughput when proofs share the GPU.  Both give the same bytes.
// The merge policy goes further: a worker that finds two or more requests waiting takes
// the longest prefix of the queue whose batch fits in the largest free block (up to
// merge_max requests) and proves it as one batch (batch.cu: one witness launch for all,
// batched NTTs, merged multi-instance MSM runs), so that the GPU runs few large kernels
// instead of many small ones; a lone request still takes the one-proof path.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "groth16.h"

namespace zkvc {
size_t prove_workspace_bytes(const zkvc_pk* pk, int mode);
int prove_enqueue(const zkvc_pk* pk, int mode, const int8_t* dX, const int8_t* dW, const uint8_t* rs_host,
                  int32_t* dY, void* ws, size_t ws_bytes, uint8_t* proof_out, int* flags_out, cudaStream_t st);
int prove_status(int flags);
int batch_serve_open(int cap, zkvc_batch** out);
size_t batch_serve_bytes(const zkvc_pk* const* pks, int count);
int batch_serve_run(zkvc_batch* B, const zkvc_pk* const* pks, int count, uint8_t* mem, size_t mem_bytes,
                    const int8_t* const* hX, const int8_t* const* hW, const uint8_t* rs, int32_t* const* hY,
                    uint8_t* proofs, int* status);
void batch_serve_drain(zkvc_batch* B);

// First-fit allocator over [0, cap) in 256-byte units, with coalescing of free blocks.
class ArenaAlloc {
 public:
  void reset(size_t cap) {
    free_.clear();
    cap_ = cap & ~size_t(255);
    if (cap_) free_[0] = cap_;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        size_t rest = it->second - bytes;
        size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t largest() const {
    size_t m = 0;
    for (const auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }
  size_t cap() const { return cap_; }

 private:
  std::map<size_t, size_t> free_;
  size_t cap_ = 0, used_ = 0;
};

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  int key = 0;
  std::vector<int8_t> X, W;
  uint8_t rs[64];
  // results
  uint8_t proof[256];
  std::vector<int32_t> Y;
  int status = ZKVC_OK;
  int mode = ZKVC_PROVE_FOLD;
  std::string err;
  bool done = false;
  Clock::time_point t_submit, t_admit, t_done;
};

}  // namespace zkvc

using namespace zkvc;

struct zkvc_server {
  int device = 0;
  std::vector<const zkvc_pk*> pks;
  int policy = ZKVC_SERVER_ADAPTIVE;
  uint8_t* arena = nullptr;
  ArenaAlloc alloc;
  size_t peak_used = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  uint64_t next_id = 1;
  int in_flight = 0;
  uint64_t completed = 0, chain_count = 0, merged_count = 0, batch_count = 0;
  int merge_max = 64;
  std::vector<size_t> fp_batch;  // device bytes of a one-request batch per key (merge policy)
  bool stop = false;
  std::vector<std::thread> workers;
  std::string fatal;  // set if a worker could not start
  std::vector<size_t> fp_fold, fp_chain;  // request footprint per key and mode
  ~zkvc_server();
};

namespace zkvc {

static size_t footprint(const zkvc_pk* pk, int mode) {
  const Shape& sh = pk->shape;
  return prove_workspace_bytes(pk, mode) + round256(size_t(sh.a) * sh.n) + round256(size_t(sh.n) * sh.b) +
         round256(size_t(sh.a) * sh.b * 4);
}

struct WorkerRes {
  cudaStream_t st = nullptr;
  uint8_t* hx = nullptr;  // pinned staging: X, W, Y, proof, flags
  size_t hx_bytes = 0;
  ~WorkerRes() {
    if (st) cudaStreamDestroy(st);
    if (hx) cudaFreeHost(hx);
  }
};

struct BatchFree {
  void operator()(zkvc_batch* b) const { zkvc_batch_free(b); }
};

// Proves the requests grp (keys kp) as one batch over [off, off + bytes) of the arena and
// completes them.
static void run_merged(zkvc_server* S, zkvc_batch* MB, std::vector<Request*>& grp,
                       const std::vector<const zkvc_pk*>& kp, size_t off, size_t bytes) {
  const int m = (int)grp.size();
  const auto t_admit = Clock::now();
  std::vector<const int8_t*> hx(m), hw(m);
  std::vector<int32_t*> hy(m);
  std::vector<uint8_t> rs(size_t(m) * 64), proofs(size_t(m) * 256);
  std::vector<int> st(m, ZKVC_OK);
  for (int i = 0; i < m; i++) {
    Request* q = grp[i];
    const Shape& sh = kp[i]->shape;
    q->t_admit = t_admit;
    q->mode = -1;
    q->Y.resize(size_t(sh.a) * sh.b);
    hx[i] = q->X.data();
    hw[i] = q->W.data();
    hy[i] = q->Y.data();
    std::memcpy(rs.data() + size_t(i) * 64, q->rs, 64);
  }
  const int rc = batch_serve_run(MB, kp.data(), m, S->arena + off, bytes, hx.data(), hw.data(), rs.data(),
                                 hy.data(), proofs.data(), st.data());
  const std::string err = rc != ZKVC_OK ? last_error_text() : std::string();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (rc != ZKVC_ETIMEOUT) S->alloc.release(off, bytes);
    S->in_flight -= m;
    S->completed += m;
    const auto t_done = Clock::now();
    for (int i = 0; i < m; i++) {
      Request* q = grp[i];
      q->status = rc != ZKVC_OK ? rc : st[i];
      if (q->status == ZKVC_OK)
        std::memcpy(q->proof, proofs.data() + size_t(i) * 256, 256);
      else
        q->err = rc != ZKVC_OK ? err
                 : q->status == ZKVC_EUNSAT ? std::string("server: the request does not satisfy its constraints")
                 : q->status == ZKVC_EINVAL ? std::string("server: r or s is not a canonical Fr element")
                                            : std::string("server: a tensor-core wait timed out");
      q->done = true;
      q->t_done = t_done;
    }
  }
  S->cv_work.notify_all();
  S->cv_done.notify_all();
  if (rc == ZKVC_ETIMEOUT) {  // the batch's streams may still run: drain before the memory is reused
    batch_serve_drain(MB);
    std::lock_guard<std::mutex> lk(S->mu);
    S->alloc.release(off, bytes);
    S->cv_work.notify_all();
  }
}

static void worker_main(zkvc_server* S) {
  WorkerRes R;
  std::unique_ptr<zkvc_batch, BatchFree> MB;
  size_t max_x = 0, max_w = 0, max_y = 0;
  for (const zkvc_pk* pk : S->pks) {
    max_x = std::max(max_x, size_t(pk->shape.a) * pk->shape.n);
    max_w = std::max(max_w, size_t(pk->shape.n) * pk->shape.b);
    max_y = std::max(max_y, size_t(pk->shape.a) * pk->shape.b * 4);
  }
  const size_t ox = 0, ow = round256(max_x), oy = ow + round256(max_w), op = oy + round256(max_y), of = op + 256;
  R.hx_bytes = of + 256;
  bool ok = cudaSetDevice(S->device) == cudaSuccess &&
            cudaStreamCreateWithFlags(&R.st, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMallocHost(&R.hx, R.hx_bytes) == cudaSuccess;
  if (ok && S->policy == ZKVC_SERVER_MERGE) {
    zkvc_batch* b = nullptr;
    ok = batch_serve_open(S->merge_max, &b) == ZKVC_OK;
    MB.reset(b);
  }
  if (!ok) {
    cudaGetLastError();
    std::lock_guard<std::mutex> lk(S->mu);
    S->fatal = "server: a worker could not create its stream or pinned staging";
    S->cv_done.notify_all();
    return;
  }
  for (;;) {
    Request* q = nullptr;
    size_t off = 0, fp = 0;
    int mode = ZKVC_PROVE_FOLD;
    std::vector<Request*> grp;
    std::vector<const zkvc_pk*> kp;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop) return;
        if (MB && S->queue.size() >= 2) {
          // the longest queue prefix (up to merge_max) whose estimate fits the largest free
          // block, then its exact size; shorter prefixes if that does not fit
          const size_t largest = S->alloc.largest();
          size_t est = 0;
          kp.clear();
          for (Request* h : S->queue) {
            if ((int)kp.size() == S->merge_max) break;
            const size_t f = S->fp_batch[h->key];
            if (est + f > largest) break;
            est += f;
            kp.push_back(S->pks[h->key]);
          }
          while (kp.size() >= 2) {
            const size_t exact = batch_serve_bytes(kp.data(), (int)kp.size());
            if (S->alloc.alloc(exact, &off)) {
              fp = exact;
              break;
            }
            kp.pop_back();
          }
          if (kp.size() >= 2) {
            for (size_t i = 0; i < kp.size(); i++) {
              grp.push_back(S->queue.front());
              S->queue.pop_front();
            }
            S->in_flight += (int)grp.size();
            S->merged_count += grp.size();
            S->batch_count++;
            S->peak_used = std::max(S->peak_used, S->alloc.used());
            break;
          }
          kp.clear();
        }
        if (!S->queue.empty()) {
          Request* h = S->queue.front();
          mode = S->policy == ZKVC_SERVER_FOLD    ? ZKVC_PROVE_FOLD
                 : S->policy == ZKVC_SERVER_CHAIN ? ZKVC_PROVE_CHAIN
                 : (S->in_flight == 0 ? ZKVC_PROVE_FOLD : ZKVC_PROVE_CHAIN);  // adaptive, merge
          fp = mode == ZKVC_PROVE_CHAIN ? S->fp_chain[h->key] : S->fp_fold[h->key];
          if (fp > S->alloc.cap() && mode == ZKVC_PROVE_FOLD) {
            mode = ZKVC_PROVE_CHAIN;  // the chain prover needs less workspace
            fp = S->fp_chain[h->key];
          }
          if (fp > S->alloc.cap()) {  // can never fit: fail it now
            S->queue.pop_front();
            h->status = ZKVC_ENOMEM;
            h->err = "server: request needs " + std::to_string(fp) + " bytes, more than the whole budget";
            h->done = true;
            h->t_admit = h->t_done = Clock::now();
            S->cv_done.notify_all();
            continue;
          }
          if (S->alloc.alloc(fp, &off)) {
            S->queue.pop_front();
            q = h;
            S->in_flight++;
            S->peak_used = std::max(S->peak_used, S->alloc.used());
            if (mode == ZKVC_PROVE_CHAIN) S->chain_count++;
            break;
          }
        }
        S->cv_work.wait(lk);
      }
    }
    if (!grp.empty()) {
      run_merged(S, MB.get(), grp, kp, off, fp);
      continue;
    }
    q->t_admit = Clock::now();
    q->mode = mode;
    const zkvc_pk* pk = S->pks[q->key];
    const Shape& sh = pk->shape;
    const size_t nx = size_t(sh.a) * sh.n, nw = size_t(sh.n) * sh.b, ny = size_t(sh.a) * sh.b;
    uint8_t* base = S->arena + off;
    int8_t* dX = reinterpret_cast<int8_t*>(base);
    int8_t* dW = reinterpret_cast<int8_t*>(base + round256(nx));
    int32_t* dY = reinterpret_cast<int32_t*>(base + round256(nx) + round256(nw));
    uint8_t* ws = base + round256(nx) + round256(nw) + round256(ny * 4);
    const size_t ws_bytes = fp - (size_t(ws - base));
    std::memcpy(R.hx + ox, q->X.data(), nx);
    std::memcpy(R.hx + ow, q->W.data(), nw);
    int* hflags = reinterpret_cast<int*>(R.hx + of);
    *hflags = 0;
    int rc = ZKVC_OK;
    if (cudaMemcpyAsync(dX, R.hx + ox, nx, cudaMemcpyHostToDevice, R.st) != cudaSuccess ||
        cudaMemcpyAsync(dW, R.hx + ow, nw, cudaMemcpyHostToDevice, R.st) != cudaSuccess) {
      set_error("server: input copy failed: %s", cudaGetErrorString(cudaGetLastError()));
      rc = ZKVC_ECUDA;
    }
    if (rc == ZKVC_OK) rc = prove_enqueue(pk, mode, dX, dW, q->rs, dY, ws, ws_bytes, R.hx + op, hflags, R.st);
    if (rc == ZKVC_OK && cudaMemcpyAsync(R.hx + oy, dY, ny * 4, cudaMemcpyDeviceToHost, R.st) != cudaSuccess) {
      set_error("server: output copy failed: %s", cudaGetErrorString(cudaGetLastError()));
      rc = ZKVC_ECUDA;
    }
    int wrc = wait_stream(R.st, "server prove");  // also drains work enqueued before a failure
    if (rc == ZKVC_OK) rc = wrc;
    if (rc == ZKVC_OK) rc = prove_status(*hflags);
    if (rc == ZKVC_OK) {
      std::memcpy(q->proof, R.hx + op, 256);
      q->Y.resize(ny);
      std::memcpy(q->Y.data(), R.hx + oy, ny * 4);
    } else {
      q->err = last_error_text();
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      // a timed-out request keeps its memory (its kernels may still run); everything
      // else returns its slot at once
      if (wrc != ZKVC_ETIMEOUT) S->alloc.release(off, fp);
      S->in_flight--;
      S->completed++;
      q->status = rc;
      q->done = true;
      q->t_done = Clock::now();
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
    if (wrc == ZKVC_ETIMEOUT) {  // this worker's stream is still busy: wait it out before reuse
      cudaStreamSynchronize(R.st);
      std::lock_guard<std::mutex> lk(S->mu);
      S->alloc.release(off, fp);
      S->cv_work.notify_all();
    }
  }
}

}  // namespace zkvc

zkvc_server::~zkvc_server() {
  {
    std::lock_guard<std::mutex> lk(mu);
    stop = true;
  }
  cv_work.notify_all();
  for (auto& t : workers) t.join();
  if (arena) {
    cudaSetDevice(device);
    cudaFree(arena);
  }
}

extern "C" {

int zkvc_server_create(const zkvc_pk* const* pks, int npk, int slots, size_t mem_budget, int policy,
                       zkvc_server** out) {
  set_error("%s", "");
  ZK_CHECK(pks && out, ZKVC_EINVAL, "server: null argument");
  *out = nullptr;
  ZK_CHECK(npk >= 1, ZKVC_EINVAL, "server: no keys");
  ZK_CHECK(slots >= 1 && slots <= 64, ZKVC_EINVAL, "server: %d slots outside [1, 64]", slots);
  ZK_CHECK(policy == ZKVC_SERVER_ADAPTIVE || policy == ZKVC_SERVER_FOLD || policy == ZKVC_SERVER_CHAIN ||
               policy == ZKVC_SERVER_MERGE,
           ZKVC_EINVAL, "server: policy %d", policy);
  ZK_CHECK(mem_budget >= (1u << 20), ZKVC_EINVAL, "server: budget of %zu bytes", mem_budget);
  int dev = 0;
  ZK_CUDA(cudaGetDevice(&dev));
  for (int i = 0; i < npk; i++) {
    ZK_CHECK(pks[i], ZKVC_EINVAL, "server: key %d is null", i);
    ZK_CHECK(!pks[i]->gen, ZKVC_EINVAL, "server: key %d is a zkvc_setup_circuit key (only CRPC + PSQ keys serve)", i);
    ZK_CHECK(pks[i]->device == dev, ZKVC_EINVAL, "server: key %d lives on device %d, current is %d", i, pks[i]->device,
             dev);
  }
  std::unique_ptr<zkvc_server> S(new zkvc_server());
  S->device = dev;
  S->pks.assign(pks, pks + npk);
  S->policy = policy;
  if (cudaMalloc(&S->arena, mem_budget) != cudaSuccess) {
    cudaGetLastError();
    S->arena = nullptr;
    set_error("server: cannot allocate the %zu-byte budget", mem_budget);
    return ZKVC_ENOMEM;
  }
  S->alloc.reset(mem_budget);
  for (const zkvc_pk* pk : S->pks) {
    S->fp_fold.push_back(footprint(pk, ZKVC_PROVE_FOLD));
    S->fp_chain.push_back(footprint(pk, ZKVC_PROVE_CHAIN));
    if (policy == ZKVC_SERVER_MERGE) S->fp_batch.push_back(batch_serve_bytes(&pk, 1));
  }
  for (int i = 0; i < slots; i++) S->workers.emplace_back(worker_main, S.get());
  *out = S.release();
  return ZKVC_OK;
}

void zkvc_server_free(zkvc_server* s) { delete s; }

int zkvc_server_submit(zkvc_server* s, int key, const int8_t* X, const int8_t* W, const uint8_t rs[64],
                       uint64_t* ticket) {
  set_error("%s", "");
  ZK_CHECK(s && X && W && rs && ticket, ZKVC_EINVAL, "server submit: null argument");
  ZK_CHECK(key >= 0 && key < (int)s->pks.size(), ZKVC_EINVAL, "server submit: key %d outside [0, %zu)", key,
           s->pks.size());
  const Shape& sh = s->pks[key]->shape;
  std::unique_ptr<Request> q(new Request());
  q->key = key;
  q->X.assign(X, X + size_t(sh.a) * sh.n);
  q->W.assign(W, W + size_t(sh.n) * sh.b);
  std::memcpy(q->rs, rs, 64);
  q->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    ZK_CHECK(s->fatal.empty(), ZKVC_ECUDA, "%s", s->fatal.c_str());
    q->id = s->next_id++;
    *ticket = q->id;
    s->queue.push_back(q.get());
    s->reqs.emplace(q->id, std::move(q));
  }
  s->cv_work.notify_one();
  return ZKVC_OK;
}

int zkvc_server_wait(zkvc_server* s, uint64_t ticket, int timeout_ms, uint8_t proof[256], int32_t* Y, double times_ms[3],
                     int* status) {
  set_error("%s", "");
  ZK_CHECK(s, ZKVC_EINVAL, "server wait: null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  ZK_CHECK(it != s->reqs.end(), ZKVC_EINVAL, "server wait: unknown ticket %llu", (unsigned long long)ticket);
  Request* q = it->second.get();
  auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
  while (!q->done) {
    ZK_CHECK(s->fatal.empty(), ZKVC_ECUDA, "%s", s->fatal.c_str());
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !q->done) {
      set_error("server wait: request %llu not finished after %d ms", (unsigned long long)ticket, timeout_ms);
      return ZKVC_ETIMEOUT;
    }
  }
  if (status) *status = q->status;
  if (times_ms) {
    using ms = std::chrono::duration<double, std::milli>;
    times_ms[0] = ms(q->t_admit - q->t_submit).count();
    times_ms[1] = ms(q->t_done - q->t_admit).count();
    times_ms[2] = ms(q->t_done - q->t_submit).count();
  }
  if (q->status == ZKVC_OK) {
    if (proof) std::memcpy(proof, q->proof, 256);
    if (Y) std::memcpy(Y, q->Y.data(), q->Y.size() * 4);
  } else {
    set_error("%s", q->err.c_str());
  }
  s->reqs.erase(it);
  return ZKVC_OK;
}

int zkvc_server_stats(zkvc_server* s, uint64_t* completed, int* in_flight, int* queued, size_t* bytes_in_use,
                      size_t* peak_bytes, uint64_t* chain_mode) {
  set_error("%s", "");
  ZK_CHECK(s, ZKVC_EINVAL, "server stats: null server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = s->completed;
  if (in_flight) *in_flight = s->in_flight;
  if (queued) *queued = (int)s->queue.size();
  if (bytes_in_use) *bytes_in_use = s->alloc.used();
  if (peak_bytes) *peak_bytes = s->peak_used;
  if (chain_mode) *chain_mode = s->chain_count;
  return ZKVC_OK;
}

int zkvc_server_merge_stats(zkvc_server* s, uint64_t* merged_requests, uint64_t* batches) {
  set_error("%s", "");
  ZK_CHECK(s, ZKVC_EINVAL, "server merge stats: null server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (merged_requests) *merged_requests = s->merged_count;
  if (batches) *batches = s->batch_count;
  return ZKVC_OK;
}

size_t zkvc_server_request_bytes(const zkvc_pk* pk, int mode) {
  if (!pk || (mode != ZKVC_PROVE_FOLD && mode != ZKVC_PROVE_CHAIN)) return 0;
  return footprint(pk, mode);
}

}  // extern "C"
