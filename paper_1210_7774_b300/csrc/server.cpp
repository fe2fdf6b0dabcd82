// Serving loop: continuous batching of bytecode requests from concurrent
// clients on one device.
//
// The paper's Bridge collects a batch of instructions per program and hands
// it to the Vector Engine Manager (section "Bridge"); here many programs
// (requests) arrive concurrently. A scheduler thread owns the context. It
// admits queued requests in arrival order while a slot (a stream with its
// own reduction scratch) is free and the admitted footprints fit the
// memory cap, executes each request's batch on its slot's stream, and
// queues the results' copies: straight into the client's buffers when they
// are page-locked, else into pinned staging. A host callback after the
// copies wakes the client, which copies staged results into its own buffers
// in its own thread; the worker later sees the slot's event and releases the
// request's device memory. A request is admitted as soon as another
// completes, so work from different requests overlaps on the device.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "vbe_core.h"


namespace {

double now_ns() {
  return (double)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// pinned host buffers for results, reused; taken by the scheduler and
// given back by the clients that copied out of them
struct PinnedPool {
  std::mutex mu;
  std::multimap<size_t, void*> free_;
  void* get(size_t n) {
    std::lock_guard<std::mutex> lk(mu);
    auto it = free_.lower_bound(n);
    if (it != free_.end() && it->first <= 2 * n + 4096) {
      void* p = it->second;
      free_.erase(it);
      return p;
    }
    void* p = nullptr;
    vbe::cuda_check(cudaMallocHost(&p, n), "cudaMallocHost");
    sizes[p] = n;
    return p;
  }
  void put(void* p) {
    std::lock_guard<std::mutex> lk(mu);
    free_.insert({sizes[p], p});
  }
  std::unordered_map<void*, size_t> sizes;
  ~PinnedPool() {
    for (auto& kv : sizes) cudaFreeHost(kv.first);
  }
};

struct Req {
  vbe_server* srv = nullptr;
  const unsigned* err_word = nullptr;  // the executing context's error word (mapped host memory)
  int64_t id = 0;
  std::vector<vbe_req_base> bases;
  std::vector<vbe_req_view> views;
  std::vector<vbe_instr> instrs;
  int64_t footprint = 0;
  vbe_request_result res{};
  bool done = false;
  int slot = -1;
  std::vector<int64_t> bh;  // base handles
  std::vector<int64_t> vh;  // view handles
  std::vector<std::pair<int, void*>> staging;  // (base index, pinned buffer)
  cudaEvent_t ev = nullptr;
  bool ready = false;    // results are in host memory (set by a stream host callback)
  bool taken = false;    // a client's wait has started taking the results
  bool cb_enqueued = false;  // the results callback is on the stream (it may set ready)
  bool fetched = false;  // ... and is finished with the request (it may be deleted)
  // its client's wait: woken (under the server's lock) when the results are
  // ready or the request is done, and only its client, so a completion does
  // not wake every waiting client
  std::condition_variable cv;
};

}  // namespace

// a scheduler thread with its own context and slots
struct Worker {
  vbe_ctx* ctx = nullptr;
  bool owns_ctx = false;
  std::vector<vbe::Exec> slots;
  std::vector<Req*> slot_req;
  // one completion event per slot, created with the slot: a slot holds one
  // request at a time and takes the next only after this event completed
  std::vector<cudaEvent_t> slot_ev;
  int inflight = 0;
  std::thread th;
};

struct vbe_server {
  vbe_server_config cfg{};
  std::vector<std::unique_ptr<Worker>> workers;
  std::deque<Req*> queue;
  std::unordered_map<int64_t, std::unique_ptr<Req>> reqs;
  int64_t used = 0;
  int64_t next_id = 1;
  std::mutex m;
  std::condition_variable cv_work;
  bool stop = false;
  PinnedPool pinned;
  int inflight = 0;  // over all workers
};

namespace {

// Release a finished request's device memory and handles (scheduler
// thread). Its results stay in pinned staging until the client that waits
// for it copies them out (in its own thread, see vbe_server_wait).
void finish_request(Worker* w, Req* r) {
  vbe::Ctx& c = w->ctx->c;
  vbe::Exec* ex = &w->slots[r->slot];
  for (auto v : r->vh) c.views.erase(v);
  for (auto h : r->bh) {
    auto it = c.bases.find(h);
    if (it == c.bases.end()) continue;
    if (it->second.dptr && !it->second.external) vbe::dev_free(&c, ex, it->second.dptr, it->second.bytes());
    if (it->second.shadow) vbe::dev_free(&c, ex, it->second.shadow, it->second.bytes());
    c.bases.erase(it);
  }
  c.epoch++;
  r->ev = nullptr;  // the slot's event, kept for its next request
}

// Stream host callback after a request's result copies: its client may
// take the results now, before the worker notices the completion and
// releases the request's device memory. (No CUDA calls here.)
void CUDART_CB on_results_ready(void* arg) {
  Req* r = static_cast<Req*>(arg);
  vbe_server* s = r->srv;
  {
    std::lock_guard<std::mutex> lk(s->m);
    // a staged kernel of the context gave up a wait: the results may be
    // invalid (the word is cleared later by the worker's completion check;
    // a request finishing on the same context meanwhile is failed too)
    if (r->err_word && *(volatile const unsigned*)r->err_word) r->res.status = VBE_ERR_TIMEOUT;
    r->res.t_ready_ns = now_ns();
    r->ready = true;
    r->cv.notify_all();  // under the lock: the client cannot delete the request before this returns
  }
}

// pinned (page-locked) host memory: a result can be copied there directly
bool is_pinned(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // the query's own error, not a pending one: checked above by the caller
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

void admit(vbe_server* s, Worker* w, Req* r, int slot) {
  vbe::Ctx& c = w->ctx->c;
  vbe::Exec* ex = &w->slots[slot];
  r->slot = slot;
  r->err_word = c.err_word;
  r->res.t_admit_ns = now_ns();
  try {
    for (auto& b : r->bases) {
      vbe::BaseRec br;
      br.dtype = b.dtype;
      br.nelem = b.nelem;
      int64_t h = c.next_handle++;
      c.bases[h] = br;
      r->bh.push_back(h);
      if (b.init) {
        vbe::BaseRec& x = c.bases[h];
        x.dptr = vbe::dev_alloc(&c, ex, x.bytes());
        x.written = true;
        if (x.bytes() > 0)
          vbe::cuda_check(cudaMemcpyAsync(x.dptr, b.init, (size_t)x.bytes(), cudaMemcpyHostToDevice, ex->stream),
                          "request upload");
      }
    }
    for (auto& v : r->views) {
      if (v.base < 0 || v.base >= (int)r->bh.size()) vbe::fail(VBE_ERR_INVALID, "request view names no base");
      vbe::ViewDesc d;
      d.base = r->bh[v.base];
      d.offset = v.offset;
      d.ndim = v.ndim;
      if (v.ndim < 0 || v.ndim > VBE_MAX_NDIM) vbe::fail(VBE_ERR_INVALID, "ndim");
      for (int k = 0; k < v.ndim; ++k) {
        d.shape[k] = v.shape[k];
        d.strides[k] = v.strides[k];
      }
      d.finish();
      if (d.size() > 0 && (d.lo < 0 || d.hi >= c.bases[d.base].nelem))
        vbe::fail(VBE_ERR_OUT_OF_BOUNDS, "request view out of bounds");
      int64_t h = c.next_handle++;
      vbe::add_view(&c, h, d);
      r->vh.push_back(h);
    }
    std::vector<vbe_instr> prog = r->instrs;
    auto map = [&](vbe_view v) -> vbe_view {
      if (v == 0) return 0;
      if (v < 1 || v > (int64_t)r->vh.size()) vbe::fail(VBE_ERR_INVALID, "request instruction names no view");
      return r->vh[v - 1];
    };
    for (auto& in : prog) {
      in.out = map(in.out);
      for (int k = 0; k < 3; ++k) in.in[k] = map(in.in[k]);
    }
    vbe::exec_batch(&c, ex, prog.data(), (int64_t)prog.size(), false);
    for (size_t i = 0; i < r->bases.size(); ++i) {
      const vbe_req_base& b = r->bases[i];
      if (!b.result) continue;
      auto& br = c.bases[r->bh[i]];
      size_t n = (size_t)br.bytes();
      if (!n) continue;
      if (!br.dptr) vbe::fail(VBE_ERR_UNINIT, "request result base was never written");
      if (is_pinned(b.result)) {
        // the client's buffer is page-locked: the copy lands there directly
        vbe::cuda_check(cudaMemcpyAsync(b.result, br.dptr, n, cudaMemcpyDeviceToHost, ex->stream), "request result");
        continue;
      }
      void* p = s->pinned.get(n);
      r->staging.push_back({(int)i, p});
      vbe::cuda_check(cudaMemcpyAsync(p, br.dptr, n, cudaMemcpyDeviceToHost, ex->stream), "request result");
    }
    // the client is woken by the callback; the event (after it) tells the
    // worker that the slot's work, callback included, is finished
    r->ev = w->slot_ev[slot];
    vbe::cuda_check(cudaLaunchHostFunc(ex->stream, on_results_ready, r), "results callback");
    r->cb_enqueued = true;
    vbe::cuda_check(cudaEventRecord(r->ev, ex->stream), "event record");
    r->res.t_issued_ns = now_ns();
    r->res.status = VBE_OK;
  } catch (const vbe::Error& e) {
    r->res.status = e.code;
    c.last_error = e.msg;
    cudaStreamSynchronize(ex->stream);
    finish_request(w, r);
    if (!r->cb_enqueued) {  // else the callback may have woken the client, who returns them
      for (auto& st : r->staging) s->pinned.put(st.second);
      r->staging.clear();
    }
    return;
  }
}

// A scheduler thread. It holds the server's lock only to move requests
// between the queue, its slots and the finished state; planning, launching
// and releasing run outside it (only this thread touches its context), so
// clients submitting and waiting, and the other workers, are never held up
// behind that host work. It admits at most two requests per round, so that
// completions are noticed between plannings.
void worker_loop(vbe_server* s, Worker* w) {
  vbe::cuda_check(cudaSetDevice(w->ctx->c.device), "cudaSetDevice");
  std::vector<Req*> done, admitted;
  std::vector<int> admitted_slot, done_status;
  for (;;) {
    done.clear();
    done_status.clear();
    admitted.clear();
    admitted_slot.clear();
    // completions (their device work is finished), found outside the
    // server's lock: only this worker changes its slots, and a request in a
    // slot lives until this worker marks it done. The event queries are
    // driver calls, which can wait behind another thread's driver work
    // (a module load, the memory pool growing); under the lock such a wait
    // would also hold up the host callbacks of every stream, which take it
    // to hand results to their clients.
    for (size_t k = 0; k < w->slots.size(); ++k) {
      Req* r = w->slot_req[k];
      if (!r || !r->ev) continue;
      cudaError_t e = cudaEventQuery(r->ev);
      if (e == cudaErrorNotReady) continue;
      done.push_back(r);
      done_status.push_back(e == cudaSuccess ? VBE_OK : VBE_ERR_CUDA);
      w->slot_req[k] = nullptr;
    }
    {
      std::unique_lock<std::mutex> lk(s->m);
      for (size_t i = 0; i < done.size(); ++i) {
        // the context's error word is read by the results callbacks under
        // this lock, so it is taken (and cleared) under it too
        if (done_status[i] == VBE_OK && vbe::take_error_word(&w->ctx->c)) done_status[i] = VBE_ERR_TIMEOUT;
        if (done_status[i] != VBE_OK) done[i]->res.status = done_status[i];
        w->inflight--;
        s->inflight--;
      }
      // admissions, in arrival order, while a slot is free and memory fits
      while (!s->queue.empty() && admitted.size() < 2) {
        Req* r = s->queue.front();
        int free_slot = -1;
        for (size_t k = 0; k < w->slots.size(); ++k)
          if (!w->slot_req[k]) {
            free_slot = (int)k;
            break;
          }
        if (free_slot < 0) break;
        if (s->cfg.mem_cap_bytes && s->used + r->footprint > (int64_t)s->cfg.mem_cap_bytes) break;
        s->queue.pop_front();
        s->used += r->footprint;
        w->slot_req[free_slot] = r;  // reserved; its event is recorded by admit()
        w->inflight++;
        s->inflight++;
        admitted.push_back(r);
        admitted_slot.push_back(free_slot);
      }
      if (done.empty() && admitted.empty()) {
        if (s->stop && s->queue.empty() && w->inflight == 0) break;
        if (w->inflight > 0 || !s->queue.empty()) s->cv_work.wait_for(lk, std::chrono::microseconds(20));
        else s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        continue;
      }
    }
    for (Req* r : done) finish_request(w, r);
    for (size_t i = 0; i < admitted.size(); ++i) admit(s, w, admitted[i], admitted_slot[i]);
    {
      std::lock_guard<std::mutex> lk(s->m);
      for (Req* r : done) {
        r->done = true;
        s->used -= r->footprint;
        if (r->fetched) s->reqs.erase(r->id);  // its client is gone already
        else r->cv.notify_all();
      }
      for (size_t i = 0; i < admitted.size(); ++i) {
        Req* r = admitted[i];
        if (r->res.status != VBE_OK) {  // rejected while planning: finished already
          r->done = true;
          s->used -= r->footprint;
          w->slot_req[admitted_slot[i]] = nullptr;
          w->inflight--;
          s->inflight--;
          r->cv.notify_all();
        }
      }
    }
    if (!done.empty()) s->cv_work.notify_all();  // memory freed: other workers may admit
  }
}

}  // namespace

extern "C" {

int vbe_server_create(vbe_ctx* ctx, const vbe_server_config* cfg, vbe_server** out) {
  if (!ctx || !cfg || !out || cfg->slots <= 0 || cfg->workers < 0) return VBE_ERR_INVALID;
  if (ctx->c.host_only) return VBE_ERR_NO_DEVICE;
  const int nw = std::max(1, std::min<int>(cfg->workers, cfg->slots));
  auto* s = new vbe_server();
  s->cfg = *cfg;
  const uint32_t fl = cfg->flags & (VBE_FUSE | VBE_PACK | VBE_AUTOTUNE);
  try {
    for (int k = 0; k < nw; ++k) {
      auto w = std::make_unique<Worker>();
      if (k == 0) {
        w->ctx = ctx;
      } else {
        vbe_config wc = ctx->c.cfg;
        wc.stream = nullptr;
        wc.cache_dir = ctx->c.cfg.cache_dir;
        int rc = vbe_init(&wc, &w->ctx);
        if (rc != VBE_OK) vbe::fail(rc, "worker context");
        w->owns_ctx = true;
      }
      w->ctx->c.cfg.flags = (w->ctx->c.cfg.flags & ~(uint32_t)(VBE_FUSE | VBE_PACK | VBE_AUTOTUNE)) | fl;
      // slots dealt round robin over the workers
      const int ns = cfg->slots / nw + (k < cfg->slots % nw ? 1 : 0);
      w->slots.resize(ns);
      w->slot_req.assign(ns, nullptr);
      w->slot_ev.assign(ns, nullptr);
      for (int q = 0; q < ns; ++q) {
        vbe::Exec& e = w->slots[q];
        vbe::cuda_check(cudaStreamCreateWithFlags(&e.stream, cudaStreamNonBlocking), "cudaStreamCreate");
        vbe::cuda_check(cudaEventCreateWithFlags(&w->slot_ev[q], cudaEventDisableTiming), "event");
        vbe::ensure_scratch(&w->ctx->c, &e, 1 << 20, 1 << 16);
      }
      s->workers.push_back(std::move(w));
    }
  } catch (const vbe::Error& e) {
    ctx->c.last_error = e.msg;
    for (auto& w : s->workers) {
      for (auto& x : w->slots)
        if (x.stream) {
          vbe::release_exec(&w->ctx->c, &x);
          cudaStreamDestroy(x.stream);
        }
      for (auto ev : w->slot_ev)
        if (ev) cudaEventDestroy(ev);
      if (w->owns_ctx) vbe_finalize(w->ctx);
    }
    delete s;
    return e.code;
  }
  for (auto& w : s->workers) w->th = std::thread(worker_loop, s, w.get());
  *out = s;
  return VBE_OK;
}

int vbe_server_submit(vbe_server* s, const vbe_request* req, int64_t* id) {
  if (!s || !req || !id) return VBE_ERR_INVALID;
  if (req->nbases < 0 || req->nviews < 0 || req->ninstrs < 0) return VBE_ERR_INVALID;
  auto r = std::make_unique<Req>();
  r->bases.assign(req->bases, req->bases + req->nbases);
  r->views.assign(req->views, req->views + req->nviews);
  r->instrs.assign(req->instrs, req->instrs + req->ninstrs);
  for (auto& b : r->bases) {
    if (b.dtype < 0 || b.dtype > 3 || b.nelem < 0) return VBE_ERR_INVALID;
    r->footprint += b.nelem * vbe::itemsize(b.dtype);
  }
  // a base the program writes through some views and reads through others
  // may get a second buffer (a tile-fused group that updates it in place
  // while reading it around): counted twice
  {
    const size_t nb = r->bases.size();
    std::vector<std::vector<int64_t>> outs(nb), ins(nb);
    auto base_of = [&](int64_t v) -> int64_t {
      return (v >= 1 && v <= (int64_t)r->views.size()) ? r->views[v - 1].base : -1;
    };
    for (auto& in : r->instrs) {
      if (in.op == VBE_OP_SYNC || in.op == VBE_OP_DISCARD || in.op == VBE_OP_FREE) continue;
      int64_t b = base_of(in.out);
      if (b >= 0 && b < (int64_t)nb) outs[b].push_back(in.out);
      for (int k = 0; k < 3; ++k) {
        b = base_of(in.in[k]);
        if (b >= 0 && b < (int64_t)nb) ins[b].push_back(in.in[k]);
      }
    }
    for (size_t b = 0; b < nb; ++b) {
      if (outs[b].empty()) continue;
      bool other = false;
      for (int64_t v : ins[b])
        if (std::find(outs[b].begin(), outs[b].end(), v) == outs[b].end()) other = true;
      if (other) r->footprint += r->bases[b].nelem * vbe::itemsize(r->bases[b].dtype);
    }
  }
  std::lock_guard<std::mutex> lk(s->m);
  if (s->stop) return VBE_ERR_BUSY;
  if (s->cfg.mem_cap_bytes && r->footprint > (int64_t)s->cfg.mem_cap_bytes) return VBE_ERR_ADMISSION;
  if (s->cfg.max_queue > 0 && (int64_t)s->queue.size() >= s->cfg.max_queue) return VBE_ERR_BUSY;
  r->id = s->next_id++;
  r->srv = s;
  r->res.t_arrive_ns = now_ns();
  r->res.footprint_bytes = r->footprint;
  *id = r->id;
  s->queue.push_back(r.get());
  s->reqs[r->id] = std::move(r);
  s->cv_work.notify_one();
  return VBE_OK;
}

int vbe_server_wait(vbe_server* s, int64_t id, int64_t timeout_ns, vbe_request_result* out) {
  if (!s) return VBE_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->m);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return VBE_ERR_INVALID;
  Req* r = it->second.get();
  if (r->taken) return VBE_ERR_INVALID;
  // results in host memory (ready), or finished without them (done: an error)
  auto pred = [&] { return r->ready || r->done; };
  if (timeout_ns < 0) {
    r->cv.wait(lk, pred);
  } else if (!r->cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns), pred)) {
    return VBE_ERR_TIMEOUT;
  }
  r->taken = true;
  const bool ready = r->ready;
  vbe_request_result res = r->res;
  lk.unlock();
  // the results, from pinned staging into the client's buffers, in this
  // (the client's) thread and outside the server's lock
  for (auto& stg : r->staging) {
    const vbe_req_base& b = r->bases[stg.first];
    if (ready) memcpy(b.result, stg.second, (size_t)(b.nelem * vbe::itemsize(b.dtype)));
    s->pinned.put(stg.second);
  }
  r->staging.clear();
  res.t_done_ns = now_ns();
  if (!ready && res.status == VBE_OK) res.status = VBE_ERR_CUDA;
  lk.lock();
  r->fetched = true;
  if (r->done) s->reqs.erase(id);  // else the worker erases it when it finishes
  if (out) *out = res;
  return res.status;
}

int vbe_server_destroy(vbe_server* s) {
  if (!s) return VBE_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->m);
    s->stop = true;
    s->cv_work.notify_all();
  }
  for (auto& w : s->workers)
    if (w->th.joinable()) w->th.join();
  for (auto& w : s->workers) {
    for (auto& e : w->slots) {
      cudaStreamSynchronize(e.stream);
      vbe::release_exec(&w->ctx->c, &e);
      cudaStreamDestroy(e.stream);
    }
    for (auto ev : w->slot_ev)
      if (ev) cudaEventDestroy(ev);
    if (w->owns_ctx) vbe_finalize(w->ctx);
  }
  delete s;
  return VBE_OK;
}

}  // extern "C"
