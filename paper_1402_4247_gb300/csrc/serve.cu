// Serving: continuous batching of band steps (not in the paper; the paper runs one fixed
// magnetite job).  Requests (H(R), S(R), images, k-points) of mixed basis size arrive at any
// time; a scheduler thread groups queued requests of equal (precision, s_cut) and either
// equal (n, nb) or, when they want all eigenvectors, basis sizes within a factor 1.25 of each
// other, into one nao_gen_eig launch (smaller problems padded to the batch's largest n, each
// overlap matrix with its own order), runs each batch on a free slot (a CUDA stream plus a
// context of its own, so its workspace is private and batches overlap on the GPU), and admits
// a batch only when its device bytes fit next to everything the scheduler already holds.
//
// Life of a request:
//   submit  (caller thread)   inputs copied to host memory the library owns; QUEUED
//   admit   (scheduler)       device buffers allocated stream-ordered on the slot's stream,
//                             inputs copied in, Parts 1-6 enqueued; RUNNING
//   finish  (driver thread)   a host function enqueued after the batch marks the slot done
//   reap    (scheduler)       its requests become DONE, the slot is free again
//   poll    (caller thread)   waits on a condition variable; returns device pointers
//   release (caller thread)   stream-ordered frees of the request's (and, with the last
//                             request of a batch, the batch's) device memory
//
// Locking: one mutex guards the queue, requests, slots and byte counts.  No CUDA call that
// can wait on the GPU is made while holding it (the host function takes the same mutex, so
// such a call could deadlock against the stream it waits for).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "nao_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// A stream-ordered device buffer (cudaMallocAsync / cudaFreeAsync).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

enum ReqState { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2 };

struct ServeBatch;

struct ServeReq {
  uint64_t id = 0;
  nao_request rq{};  // sizes and parameters (its pointers are not used after submit)
  int nb = 0, nprob = 0;
  std::vector<double> HR, SR, kp, wk;
  std::vector<int32_t> R;
  // device memory owned by the request: inputs and the Parts 5-6 outputs; deps / dC: its
  // eigenvalues and eigenvectors compacted to its own order when the batch padded it
  DevBuf dHR, dSR, dR, dk, dw, df, drho, dmu, deb, drst, deps, dC;
  std::shared_ptr<ServeBatch> batch;
  int prob_off = 0, s_off = 0;  // slices of the batch arrays
  int state = Q_QUEUED;
  int status = NAO_OK;
  Clock::time_point t_submit, t_start, t_done;
  int batch_requests = 0;
};

struct NaoServerCore;

// Device memory of one nao_gen_eig launch, shared by its requests' results.
struct ServeBatch {
  NaoServerCore* srv = nullptr;
  int n = 0, nb = 0;       // the launch's (largest) basis size and eigenvector columns
  DevBuf Hk, Sk, smap;     // inputs of the launch: freed when it finishes
  DevBuf ssize, tmp;       // per-S orders and a padded request's Bloch sums (uneven batches)
  DevBuf eps, C, m, st;    // results: freed with the last request of the batch
  ~ServeBatch();
};

struct ServeSlot {
  nao_ctx* sub = nullptr;
  cudaStream_t stream = nullptr;
  bool busy = false;
  bool done = false;
  Clock::time_point t_done;
  std::vector<uint64_t> reqs;
  size_t ws_counted = 0;  // workspace bytes of `sub` already in the byte count
  NaoServerCore* srv = nullptr;
};

}  // namespace

struct NaoServer {
  virtual ~NaoServer() {}
};

namespace {

struct NaoServerCore : NaoServer {
  nao_ctx* owner = nullptr;
  int device = 0;
  size_t budget = 0;
  int max_batch = 256;
  int nslots = 2;
  bool started = false, stop = false, paused = false;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, std::unique_ptr<ServeReq>> reqs;
  std::vector<std::unique_ptr<ServeSlot>> slots;
  cudaStream_t free_stream = nullptr;
  size_t used = 0, peak = 0;
  uint64_t next_id = 1;
  int running = 0;

  void add_bytes(size_t b) {
    used += b;
    if (used > peak) peak = used;
  }
  // Stream-ordered free (does not wait) and the matching decrement of the byte count
  // (the admission test counts every buffer as elems_bytes of its size).  Lock held.
  void free_buf(DevBuf& b);
  void loop();
  void launch(ServeSlot* slot, std::vector<ServeReq*> batch_reqs);
  size_t batch_bytes(const std::vector<ServeReq*>& rs, size_t* req_bytes, size_t* ws_need) const;
  // a batch's launch order n (its largest request's) and eigenvector columns nb
  static void batch_shape(const std::vector<ServeReq*>& rs, int* n, int* nb) {
    int nmax = 0;
    bool uneven = false;
    for (ServeReq* r : rs) {
      if (r->rq.n != rs[0]->rq.n) uneven = true;
      if (r->rq.n > nmax) nmax = r->rq.n;
    }
    *n = nmax;
    *nb = uneven ? nmax : rs[0]->nb;  // uneven batches hold requests that want all vectors
  }
  // whether r may join a batch whose orders span [nlo, nhi] and whose first request is head
  static bool joins(const ServeReq* head, const ServeReq* r, int nlo, int nhi) {
    if (r->rq.precision != head->rq.precision || r->rq.s_cut != head->rq.s_cut) return false;
    if (r->rq.n == head->rq.n && r->nb == head->nb && nlo == nhi) return true;
    if (r->nb != r->rq.n || head->nb != head->rq.n) return false;  // padding needs all vectors
    const int lo = r->rq.n < nlo ? r->rq.n : nlo, hi = r->rq.n > nhi ? r->rq.n : nhi;
    return (long long)hi * 4 <= (long long)lo * 5;  // orders within a factor 1.25
  }
};

size_t elems_bytes(size_t count, size_t size) { return ((count * size + 255) / 256) * 256; }

void NaoServerCore::free_buf(DevBuf& b) {
  if (b.p) {
    cudaFreeAsync(b.p, free_stream);
    used -= elems_bytes(b.bytes, 1);
  }
  b.p = nullptr;
  b.bytes = 0;
}

ServeBatch::~ServeBatch() {
  if (!srv) return;
  for (DevBuf* b : {&Hk, &Sk, &smap, &ssize, &tmp, &eps, &C, &m, &st}) srv->free_buf(*b);
}

void CUDART_CB slot_done_cb(void* arg) {
  ServeSlot* s = (ServeSlot*)arg;
  NaoServerCore* srv = s->srv;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    s->done = true;
    s->t_done = Clock::now();
  }
  srv->cv_work.notify_all();
}

// Device bytes a batch adds: the requests' own buffers, the batch arrays, and the growth of
// the slot workspace (gen_eig of the whole batch, then Parts 5-6 per request).
size_t NaoServerCore::batch_bytes(const std::vector<ServeReq*>& rs, size_t* req_bytes, size_t* ws_need) const {
  int n = 0, nb = 0;
  batch_shape(rs, &n, &nb);
  size_t rb = 0, tmp = 0;
  int P = 0, NS = 0;
  for (ServeReq* r : rs) {
    const nao_request& q = r->rq;
    const size_t nr = (size_t)q.n;
    size_t b = elems_bytes((size_t)q.nspin * q.nR * nr * nr, 8) + elems_bytes((size_t)q.nR * nr * nr, 8) +
               elems_bytes((size_t)q.nR * 3, 4) + elems_bytes((size_t)q.nk * 3, 8) + elems_bytes(q.nk, 8);
    if (q.want_rho)
      b += elems_bytes((size_t)r->nprob * nr, 8) + elems_bytes((size_t)q.nspin * q.nR * nr * nr, 8) + 3 * 256;
    if (q.n < n) {  // compacted results and the padding copy of its Bloch sums
      b += elems_bytes((size_t)r->nprob * nr, 8) + elems_bytes((size_t)r->nprob * nr * nr, 16);
      const size_t t = elems_bytes((size_t)(r->nprob > q.nk ? r->nprob : q.nk) * nr * nr, 16);
      if (t > tmp) tmp = t;
    }
    rb += b;
    P += r->nprob;
    NS += q.nk;
  }
  size_t bb = elems_bytes((size_t)P * n * n, 16) + elems_bytes((size_t)NS * n * n, 16) + elems_bytes(P, 4) +
              elems_bytes((size_t)P * n, 8) + elems_bytes((size_t)P * n * nb, 16) + 2 * elems_bytes(P, 4) +
              elems_bytes(NS, 4) + tmp;
  size_t ws = gen_eig_ws_bytes(owner, n, P, NS);
  for (ServeReq* r : rs) {  // Parts 1 and 5-6 run per request in the same workspace
    const nao_request& q = r->rq;
    const size_t wd = density_ws_bytes(owner, q.n, q.nspin, q.nk, q.nR, q.n < n ? q.n : nb);
    const size_t wb = bloch_ws_bytes(owner, q.n, q.nR, q.nspin, q.nk);
    if (wd > ws) ws = wd;
    if (wb > ws) ws = wb;
  }
  *req_bytes = rb;
  *ws_need = ws + ws / 8;
  return rb + bb;
}

template <class T>
cudaError_t dalloc(DevBuf& b, size_t count, cudaStream_t st) {
  b.bytes = count * sizeof(T);
  const cudaError_t e = cudaMallocAsync(&b.p, b.bytes ? b.bytes : 16, st);
  if (e != cudaSuccess) {
    b.p = nullptr;
    b.bytes = 0;
  }
  return e;
}

void NaoServerCore::launch(ServeSlot* slot, std::vector<ServeReq*> rs) {
  cudaSetDevice(device);
  cudaStream_t st = slot->stream;
  const nao_request& q0 = rs[0]->rq;
  int n = 0, nb = 0;
  batch_shape(rs, &n, &nb);
  auto b = std::make_shared<ServeBatch>();
  b->srv = this;
  b->n = n;
  b->nb = nb;
  int P = 0, NS = 0;
  bool uneven = false;
  size_t ntmp = 0;  // elements of the padding buffer: the largest padded request's Bloch sums
  for (ServeReq* r : rs) {
    r->prob_off = P;
    r->s_off = NS;
    P += r->nprob;
    NS += r->rq.nk;
    if (r->rq.n < n) {
      uneven = true;
      const size_t t = (size_t)(r->nprob > r->rq.nk ? r->nprob : r->rq.nk) * r->rq.n * r->rq.n;
      if (t > ntmp) ntmp = t;
    }
  }
  int rc = NAO_OK;
  cudaError_t e = cudaSuccess;
  auto ck = [&](cudaError_t x) {
    if (x != cudaSuccess && e == cudaSuccess) e = x;
  };
  ck(dalloc<nao_c128>(b->Hk, (size_t)P * n * n, st));
  ck(dalloc<nao_c128>(b->Sk, (size_t)NS * n * n, st));
  ck(dalloc<int32_t>(b->smap, P, st));
  ck(dalloc<double>(b->eps, (size_t)P * n, st));
  ck(dalloc<nao_c128>(b->C, (size_t)P * n * nb, st));
  ck(dalloc<int32_t>(b->m, P, st));
  ck(dalloc<int32_t>(b->st, P, st));
  if (uneven) {
    ck(dalloc<int32_t>(b->ssize, NS, st));
    ck(dalloc<nao_c128>(b->tmp, ntmp, st));
  }
  std::vector<int32_t> smap(P), ssize(NS);
  for (ServeReq* r : rs) {
    const nao_request& q = r->rq;
    const int nr = q.n;
    for (int s = 0; s < q.nspin; ++s)
      for (int k = 0; k < q.nk; ++k) smap[r->prob_off + s * q.nk + k] = r->s_off + k;
    for (int k = 0; k < q.nk; ++k) ssize[r->s_off + k] = nr;
    ck(dalloc<double>(r->dHR, r->HR.size(), st));
    ck(dalloc<double>(r->dSR, r->SR.size(), st));
    ck(dalloc<int32_t>(r->dR, r->R.size(), st));
    ck(dalloc<double>(r->dk, r->kp.size(), st));
    ck(dalloc<double>(r->dw, r->wk.size(), st));
    if (nr < n) {
      ck(dalloc<double>(r->deps, (size_t)r->nprob * nr, st));
      ck(dalloc<nao_c128>(r->dC, (size_t)r->nprob * nr * nr, st));
    }
    if (q.want_rho) {
      ck(dalloc<double>(r->df, (size_t)r->nprob * nr, st));
      ck(dalloc<double>(r->drho, (size_t)q.nspin * q.nR * nr * nr, st));
      ck(dalloc<double>(r->dmu, 1, st));
      ck(dalloc<double>(r->deb, 1, st));
      ck(dalloc<int32_t>(r->drst, 1, st));
    }
  }
  if (e == cudaSuccess) {
    ck(cudaMemcpyAsync(b->smap.p, smap.data(), smap.size() * 4, cudaMemcpyHostToDevice, st));
    if (uneven) {  // the padded blocks of H(k) and S(k) stay zero
      ck(cudaMemcpyAsync(b->ssize.p, ssize.data(), ssize.size() * 4, cudaMemcpyHostToDevice, st));
      ck(cudaMemsetAsync(b->Hk.p, 0, b->Hk.bytes, st));
      ck(cudaMemsetAsync(b->Sk.p, 0, b->Sk.bytes, st));
    }
    for (ServeReq* r : rs) {
      ck(cudaMemcpyAsync(r->dHR.p, r->HR.data(), r->dHR.bytes, cudaMemcpyHostToDevice, st));
      ck(cudaMemcpyAsync(r->dSR.p, r->SR.data(), r->dSR.bytes, cudaMemcpyHostToDevice, st));
      ck(cudaMemcpyAsync(r->dR.p, r->R.data(), r->dR.bytes, cudaMemcpyHostToDevice, st));
      ck(cudaMemcpyAsync(r->dk.p, r->kp.data(), r->dk.bytes, cudaMemcpyHostToDevice, st));
      ck(cudaMemcpyAsync(r->dw.p, r->wk.data(), r->dw.bytes, cudaMemcpyHostToDevice, st));
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    rc = NAO_E_NOMEM;
  }
  nao_c128* Hk = (nao_c128*)b->Hk.p;
  nao_c128* Sk = (nao_c128*)b->Sk.p;
  // the n_r x n_r matrices at src (dense) into the leading blocks of n x n slots at dst
  auto pad_copy = [&](nao_c128* dst, const nao_c128* src, int count, int nr) {
    for (int a = 0; a < count && e == cudaSuccess; ++a)
      ck(cudaMemcpy2DAsync(dst + (size_t)a * n * n, (size_t)n * sizeof(nao_c128), src + (size_t)a * nr * nr,
                           (size_t)nr * sizeof(nao_c128), (size_t)nr * sizeof(nao_c128), nr, cudaMemcpyDeviceToDevice,
                           st));
  };
  for (ServeReq* r : rs) {  // Part 1 of every request into its slice of the batch
    if (rc) break;
    const nao_request& q = r->rq;
    const int nr = q.n;
    if (nr == n) {
      rc = nao_bloch_sum(slot->sub, n, q.nR, (const int32_t*)r->dR.p, 1, (const double*)r->dSR.p, q.nk,
                         (const double*)r->dk.p, Sk + (size_t)r->s_off * n * n, st);
      if (!rc)
        rc = nao_bloch_sum(slot->sub, n, q.nR, (const int32_t*)r->dR.p, q.nspin, (const double*)r->dHR.p, q.nk,
                           (const double*)r->dk.p, Hk + (size_t)r->prob_off * n * n, st);
    } else {  // at its own order, then padded into the batch's slots
      nao_c128* t = (nao_c128*)b->tmp.p;
      rc = nao_bloch_sum(slot->sub, nr, q.nR, (const int32_t*)r->dR.p, 1, (const double*)r->dSR.p, q.nk,
                         (const double*)r->dk.p, t, st);
      if (!rc) pad_copy(Sk + (size_t)r->s_off * n * n, t, q.nk, nr);
      if (!rc)
        rc = nao_bloch_sum(slot->sub, nr, q.nR, (const int32_t*)r->dR.p, q.nspin, (const double*)r->dHR.p, q.nk,
                           (const double*)r->dk.p, t, st);
      if (!rc) pad_copy(Hk + (size_t)r->prob_off * n * n, t, r->nprob, nr);
      if (!rc && e != cudaSuccess) rc = NAO_E_CUDA;
    }
  }
  if (!rc) {  // Parts 2-4 of the whole batch in one launch sequence
    nao_set_refinement(slot->sub, slot->srv->owner->refine_sweeps);  // the owner's refinement
    rc = nao_gen_eig_sized(slot->sub, n, P, Hk, Sk, (const int32_t*)b->smap.p, NS,
                           uneven ? (const int32_t*)b->ssize.p : nullptr, q0.s_cut, q0.precision, nb,
                           (double*)b->eps.p, (nao_c128*)b->C.p, (int32_t*)b->m.p, (int32_t*)b->st.p, st);
  }
  for (ServeReq* r : rs) {  // padded requests: eigenvalues and vectors at their own order
    if (rc) break;
    const int nr = r->rq.n;
    if (nr == n) continue;
    ck(cudaMemcpy2DAsync(r->deps.p, (size_t)nr * sizeof(double), (const double*)b->eps.p + (size_t)r->prob_off * n,
                         (size_t)n * sizeof(double), (size_t)nr * sizeof(double), r->nprob, cudaMemcpyDeviceToDevice,
                         st));
    for (int p = 0; p < r->nprob && e == cudaSuccess; ++p)
      ck(cudaMemcpy2DAsync((nao_c128*)r->dC.p + (size_t)p * nr * nr, (size_t)nr * sizeof(nao_c128),
                           (const nao_c128*)b->C.p + (size_t)(r->prob_off + p) * n * nb, (size_t)nb * sizeof(nao_c128),
                           (size_t)nr * sizeof(nao_c128), nr, cudaMemcpyDeviceToDevice, st));
    if (e != cudaSuccess) rc = NAO_E_CUDA;
  }
  for (ServeReq* r : rs) {  // Parts 5-6 per request (its own electrons, weights, images)
    if (rc) break;
    const nao_request& q = r->rq;
    if (!q.want_rho) continue;
    const int nr = q.n;
    const bool own = nr < n;  // compacted results
    const int nbr = own ? nr : nb;
    rc = nao_density_matrix(slot->sub, nr, q.nspin, q.nk, (const double*)r->dw.p, (const double*)r->dk.p,
                            own ? (const double*)r->deps.p : (const double*)b->eps.p + (size_t)r->prob_off * n,
                            own ? (const nao_c128*)r->dC.p : (const nao_c128*)b->C.p + (size_t)r->prob_off * n * nb,
                            nbr, (const int32_t*)b->m.p + r->prob_off, q.n_electrons, q.kT, q.nR,
                            (const int32_t*)r->dR.p, (double*)r->dmu.p, (double*)r->deb.p, (double*)r->df.p,
                            (double*)r->drho.p, nullptr, (int32_t*)r->drst.p, st);
  }
  const size_t ws_now = slot->sub->ws_bytes;
  bool enqueued = false;
  if (cudaLaunchHostFunc(st, slot_done_cb, slot) == cudaSuccess) enqueued = true;
  else cudaGetLastError();
  if (!enqueued) cudaStreamSynchronize(st);  // before taking the lock (see the note on locking)
  std::lock_guard<std::mutex> lk(mu);
  for (ServeReq* r : rs) {
    r->batch = b;
    r->batch_requests = (int)rs.size();
    if (rc) r->status = rc;
  }
  if (ws_now > slot->ws_counted) {  // the slot's workspace grew: count the new size
    add_bytes(ws_now - slot->ws_counted);
    slot->ws_counted = ws_now;
  }
  if (!enqueued) {  // no completion callback: the batch was finished above
    slot->done = true;
    slot->t_done = Clock::now();
    for (ServeReq* r : rs)
      if (!r->status) r->status = NAO_E_CUDA;
  }
}

void NaoServerCore::loop() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    // reap finished slots
    for (auto& sp : slots) {
      ServeSlot* s = sp.get();
      if (!s->busy || !s->done) continue;
      for (uint64_t id : s->reqs) {
        auto it = reqs.find(id);
        if (it == reqs.end()) continue;
        ServeReq* r = it->second.get();
        r->state = Q_DONE;
        r->t_done = s->t_done;
        if (r->batch)
          for (DevBuf* b : {&r->batch->Hk, &r->batch->Sk, &r->batch->smap, &r->batch->ssize, &r->batch->tmp})
            free_buf(*b);
        // the inputs are no longer needed either
        for (DevBuf* b : {&r->dHR, &r->dSR, &r->dR, &r->dk, &r->dw}) free_buf(*b);
      }
      s->reqs.clear();
      s->busy = false;
      s->done = false;
      --running;
      cv_done.notify_all();
    }
    if (stop && running == 0) break;
    // admit the next batch
    ServeSlot* slot = nullptr;
    for (auto& sp : slots)
      if (!sp->busy) {
        slot = sp.get();
        break;
      }
    bool launched = false;
    if (!stop && !paused && slot && !queue.empty()) {
      ServeReq* head = reqs[queue.front()].get();
      std::vector<ServeReq*> batch{head};
      int probs = head->nprob, nlo = head->rq.n, nhi = head->rq.n;
      for (size_t i = 1; i < queue.size(); ++i) {
        ServeReq* r = reqs[queue[i]].get();
        if (!joins(head, r, nlo, nhi)) continue;
        if (probs + r->nprob > max_batch) break;
        batch.push_back(r);
        probs += r->nprob;
        if (r->rq.n < nlo) nlo = r->rq.n;
        if (r->rq.n > nhi) nhi = r->rq.n;
      }
      size_t rb = 0, wsn = 0;
      size_t need = batch_bytes(batch, &rb, &wsn);
      size_t grow = wsn > slot->ws_counted ? wsn - slot->ws_counted : 0;
      if (batch.size() > 1 && used + need + grow > budget) {  // try the head alone
        batch.resize(1);
        need = batch_bytes(batch, &rb, &wsn);
        grow = wsn > slot->ws_counted ? wsn - slot->ws_counted : 0;
      }
      if (need + wsn > budget) {  // can never fit: fail the head
        head->status = NAO_E_NOMEM;
        head->state = Q_DONE;
        head->t_start = head->t_done = Clock::now();
        queue.pop_front();
        cv_done.notify_all();
        continue;
      }
      if (used + need + grow <= budget) {
        for (ServeReq* r : batch) {
          for (auto it = queue.begin(); it != queue.end(); ++it)
            if (*it == r->id) {
              queue.erase(it);
              break;
            }
          r->state = Q_RUNNING;
          r->t_start = Clock::now();
          slot->reqs.push_back(r->id);
        }
        add_bytes(need);  // each buffer's free subtracts its own share again
        slot->busy = true;
        slot->done = false;
        ++running;
        lk.unlock();
        launch(slot, batch);
        lk.lock();
        launched = true;
      }
    }
    if (!launched) cv_work.wait_for(lk, std::chrono::milliseconds(50));
  }
}

NaoServerCore* get_server(nao_ctx* ctx) {
  if (!ctx->server) {
    auto* s = new NaoServerCore();
    s->owner = ctx;
    s->device = ctx->device;
    ctx->server = s;
  }
  return static_cast<NaoServerCore*>(ctx->server);
}

int start_server(nao_ctx* ctx, NaoServerCore* s) {
  if (s->started) return NAO_OK;
  cudaSetDevice(s->device);
  if (s->budget == 0) s->budget = ctx->hbm_budget;  // the context's budget, when it has one
  if (s->budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return nao_fail(ctx, NAO_E_CUDA, "nao_serve: cudaMemGetInfo failed");
    s->budget = fr / 10 * 8;
  }
  // keep freed blocks in the device's stream-ordered pool instead of returning them
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (cudaStreamCreateWithFlags(&s->free_stream, cudaStreamNonBlocking) != cudaSuccess)
    return nao_fail(ctx, NAO_E_CUDA, "nao_serve: stream creation failed");
  for (int i = 0; i < s->nslots; ++i) {
    auto slot = std::make_unique<ServeSlot>();
    slot->srv = s;
    // a slot's context takes the owner's settings; its workspace is bounded by the
    // scheduler's admission test, not by a budget of its own
    int rc = nao_init(&slot->sub, s->device, 0, &ctx->cfg);
    if (rc) return nao_fail(ctx, rc, "nao_serve: slot context: %s", nao_last_error(nullptr));
    nao_set_gemm_method(slot->sub, ctx->gemm_method);
    if (cudaStreamCreateWithFlags(&slot->stream, cudaStreamNonBlocking) != cudaSuccess)
      return nao_fail(ctx, NAO_E_CUDA, "nao_serve: stream creation failed");
    s->slots.push_back(std::move(slot));
  }
  s->th = std::thread([s] { s->loop(); });
  s->started = true;
  return NAO_OK;
}

void release_request(NaoServerCore* s, ServeReq* r) {  // lock held; r is DONE
  for (DevBuf* b : {&r->dHR, &r->dSR, &r->dR, &r->dk, &r->dw, &r->df, &r->drho, &r->dmu, &r->deb, &r->drst,
                    &r->deps, &r->dC})
    s->free_buf(*b);
  r->batch.reset();  // the last holder frees the batch's result arrays
}

}  // namespace

void serve_shutdown(nao_ctx* ctx) {
  if (!ctx->server) return;
  NaoServerCore* s = static_cast<NaoServerCore*>(ctx->server);
  if (s->started) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
      s->queue.clear();
    }
    s->cv_work.notify_all();
    s->th.join();
    cudaSetDevice(s->device);
    for (auto& sl : s->slots) cudaStreamSynchronize(sl->stream);
    for (auto& kv : s->reqs) release_request(s, kv.second.get());
    s->reqs.clear();
    cudaStreamSynchronize(s->free_stream);
    for (auto& sl : s->slots) {
      cudaStreamDestroy(sl->stream);
      nao_destroy(sl->sub);
    }
    cudaStreamDestroy(s->free_stream);
  }
  delete s;
  ctx->server = nullptr;
}

int nao_serve_config(nao_ctx* ctx, size_t hbm_budget_bytes, int max_batch_problems, int slots) {
  if (!ctx) return nao_fail(nullptr, NAO_E_INVALID, "nao_serve_config: ctx is NULL");
  if (max_batch_problems < 1 || slots < 1 || slots > 16)
    return nao_fail(ctx, NAO_E_INVALID, "nao_serve_config: max_batch_problems >= 1, 1 <= slots <= 16");
  NaoServerCore* s = get_server(ctx);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->started && (s->running || !s->queue.empty()))
    return nao_fail(ctx, NAO_E_BUSY, "nao_serve_config: requests are queued or running");
  if (s->started && slots != s->nslots)
    return nao_fail(ctx, NAO_E_INVALID, "nao_serve_config: the slot count is fixed after the first submit");
  s->budget = hbm_budget_bytes;
  s->max_batch = max_batch_problems;
  s->nslots = slots;
  return NAO_OK;
}

int nao_serve_pause(nao_ctx* ctx, int on) {
  if (!ctx) return nao_fail(nullptr, NAO_E_INVALID, "nao_serve_pause: ctx is NULL");
  NaoServerCore* s = get_server(ctx);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->paused = on != 0;
  }
  s->cv_work.notify_all();
  return NAO_OK;
}

int nao_serve_submit(nao_ctx* ctx, const nao_request* q, uint64_t* ticket) {
  if (!ctx || !q || !ticket) return nao_fail(ctx, NAO_E_INVALID, "nao_serve_submit: NULL argument");
  if (q->n < 1 || q->n > 4096 || q->nR < 1 || q->nk < 1 || (q->nspin != 1 && q->nspin != 2))
    return nao_fail(ctx, NAO_E_INVALID, "nao_serve_submit: bad sizes");
  if (!q->HR || !q->SR || !q->R || !q->kpts || !q->wk)
    return nao_fail(ctx, NAO_E_INVALID, "nao_serve_submit: NULL array");
  if (q->precision != NAO_FP64 && q->precision != NAO_MIXED_BF16X3)
    return nao_fail(ctx, NAO_E_INVALID, "nao_serve_submit: precision %d not available", q->precision);
  if (q->nb < 0 || q->nb > q->n) return nao_fail(ctx, NAO_E_INVALID, "nao_serve_submit: nb must be in [0, n]");
  if (!(q->s_cut >= 0.0) || (q->want_rho && !(q->kT > 0.0)))
    return nao_fail(ctx, NAO_E_INVALID, "nao_serve_submit: s_cut >= 0 and kT > 0 required");
  if ((size_t)8 * q->nR * 2 > 200 * 1024 || (size_t)16 * q->nk * 8 > 200 * 1024)
    return nao_fail(ctx, NAO_E_INVALID, "nao_serve_submit: nR or nk too large");
  auto r = std::make_unique<ServeReq>();
  r->rq = *q;
  r->nb = q->nb ? q->nb : q->n;
  r->nprob = q->nspin * q->nk;
  const size_t nn = (size_t)q->n * q->n;
  r->HR.resize((size_t)q->nspin * q->nR * nn);
  r->SR.resize((size_t)q->nR * nn);
  r->R.resize((size_t)q->nR * 3);
  r->kp.resize((size_t)q->nk * 3);
  r->wk.resize(q->nk);
  cudaSetDevice(ctx->device);
  // copies from host or device memory (cudaMemcpyDefault infers the direction)
  struct {
    void* dst;
    const void* src;
    size_t bytes;
  } cp[5] = {{r->HR.data(), q->HR, r->HR.size() * 8}, {r->SR.data(), q->SR, r->SR.size() * 8},
             {r->R.data(), q->R, r->R.size() * 4}, {r->kp.data(), q->kpts, r->kp.size() * 8},
             {r->wk.data(), q->wk, r->wk.size() * 8}};
  for (auto& c : cp)
    if (cudaMemcpy(c.dst, c.src, c.bytes, cudaMemcpyDefault) != cudaSuccess) {
      cudaGetLastError();
      return nao_fail(ctx, NAO_E_INVALID, "nao_serve_submit: could not read an input array");
    }
  NaoServerCore* s = get_server(ctx);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->started) {
      int rc = start_server(ctx, s);
      if (rc) return rc;
    }
    r->id = s->next_id++;
    r->t_submit = Clock::now();
    *ticket = r->id;
    s->queue.push_back(r->id);
    s->reqs[r->id] = std::move(r);
  }
  s->cv_work.notify_all();
  return NAO_OK;
}

int nao_serve_poll(nao_ctx* ctx, uint64_t ticket, int timeout_us, nao_result* out) {
  if (!ctx || !out) return nao_fail(ctx, NAO_E_INVALID, "nao_serve_poll: NULL argument");
  if (!ctx->server) return nao_fail(ctx, NAO_E_INVALID, "nao_serve_poll: unknown ticket");
  NaoServerCore* s = static_cast<NaoServerCore*>(ctx->server);
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return nao_fail(ctx, NAO_E_INVALID, "nao_serve_poll: unknown ticket %llu",
                                            (unsigned long long)ticket);
  ServeReq* r = it->second.get();
  auto done = [&] { return r->state == Q_DONE; };
  if (timeout_us < 0) s->cv_done.wait(lk, done);
  else if (timeout_us > 0) s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done);
  std::memset(out, 0, sizeof(*out));
  out->n = r->rq.n;
  out->nprob = r->nprob;
  out->nb = r->nb;
  out->nspin = r->rq.nspin;
  out->nR = r->rq.nR;
  if (!done()) {
    out->status = NAO_E_BUSY;
    return NAO_E_BUSY;
  }
  out->status = r->status;
  out->queue_ms = ms_between(r->t_submit, r->t_start);
  out->latency_ms = ms_between(r->t_submit, r->t_done);
  out->batch_requests = r->batch_requests;
  if (r->batch && r->status == NAO_OK) {
    ServeBatch* b = r->batch.get();
    if (r->deps.p) {  // padded in its batch: the compacted copies
      out->eps = (const double*)r->deps.p;
      out->C = (const nao_c128*)r->dC.p;
    } else {
      out->eps = (const double*)b->eps.p + (size_t)r->prob_off * b->n;
      out->C = (const nao_c128*)b->C.p + (size_t)r->prob_off * b->n * b->nb;
    }
    out->m_kept = (const int32_t*)b->m.p + r->prob_off;
    out->prob_status = (const int32_t*)b->st.p + r->prob_off;
    if (r->rq.want_rho) {
      out->mu = (const double*)r->dmu.p;
      out->eband = (const double*)r->deb.p;
      out->f = (const double*)r->df.p;
      out->rho = (const double*)r->drho.p;
      out->rho_status = (const int32_t*)r->drst.p;
    }
  }
  return out->status;
}

int nao_serve_release(nao_ctx* ctx, uint64_t ticket) {
  if (!ctx || !ctx->server) return nao_fail(ctx, NAO_E_INVALID, "nao_serve_release: unknown ticket");
  NaoServerCore* s = static_cast<NaoServerCore*>(ctx->server);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return nao_fail(ctx, NAO_E_INVALID, "nao_serve_release: unknown ticket");
    if (it->second->state != Q_DONE) return nao_fail(ctx, NAO_E_BUSY, "nao_serve_release: request not finished");
    cudaSetDevice(s->device);
    release_request(s, it->second.get());
    s->reqs.erase(it);
  }
  s->cv_work.notify_all();
  return NAO_OK;
}

int nao_serve_stats(nao_ctx* ctx, size_t* used_bytes, size_t* peak_bytes, int* queued, int* running) {
  if (!ctx) return nao_fail(nullptr, NAO_E_INVALID, "nao_serve_stats: ctx is NULL");
  if (!ctx->server) {
    if (used_bytes) *used_bytes = 0;
    if (peak_bytes) *peak_bytes = 0;
    if (queued) *queued = 0;
    if (running) *running = 0;
    return NAO_OK;
  }
  NaoServerCore* s = static_cast<NaoServerCore*>(ctx->server);
  std::lock_guard<std::mutex> lk(s->mu);
  if (used_bytes) *used_bytes = s->used;
  if (peak_bytes) *peak_bytes = s->peak;
  if (queued) *queued = (int)s->queue.size();
  if (running) {
    int r = 0;
    for (auto& kv : s->reqs) r += kv.second->state == Q_RUNNING;
    *running = r;
  }
  return NAO_OK;
}
