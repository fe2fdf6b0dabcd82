// Serving loop: continuous batching of bytecode requests from concurrent
// clients on one device.
//
// The paper's Bridge collects a batch of instructions per program and hands
// it to the Vector Engine Manager (section "Bridge"); here many programs
// (requests) arrive concurrently. A scheduler thread owns the context. It
// admits queued requests in arrival order while a slot (a stream with its
// own reduction scratch) is free and the admitted footprints fit the
// memory cap, executes each request's batch on its slot's stream, copies
// the results into pinned staging memory, and on completion hands them to
// the client. A request is admitted as soon as another completes, so work
// from different requests overlaps on the device.
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

struct PinnedPool {
  std::multimap<size_t, void*> free_;
  void* get(size_t n) {
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
  void put(void* p) { free_.insert({sizes[p], p}); }
  std::unordered_map<void*, size_t> sizes;
  ~PinnedPool() {
    for (auto& kv : sizes) cudaFreeHost(kv.first);
  }
};

struct Req {
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
};

}  // namespace

struct vbe_server {
  vbe_ctx* ctx = nullptr;
  vbe_server_config cfg{};
  std::vector<vbe::Exec> slots;
  std::vector<Req*> slot_req;
  std::deque<Req*> queue;
  std::unordered_map<int64_t, std::unique_ptr<Req>> reqs;
  int64_t used = 0;
  int64_t next_id = 1;
  std::mutex m;
  std::condition_variable cv_done, cv_work;
  std::thread th;
  bool stop = false;
  PinnedPool pinned;
  int inflight = 0;
};

namespace {

void finish_request(vbe_server* s, Req* r) {
  vbe::Ctx& c = s->ctx->c;
  vbe::Exec* ex = &s->slots[r->slot];
  for (auto& st : r->staging) {
    const vbe_req_base& b = r->bases[st.first];
    memcpy(b.result, st.second, (size_t)(b.nelem * vbe::itemsize(b.dtype)));
    s->pinned.put(st.second);
  }
  r->staging.clear();
  for (auto v : r->vh) c.views.erase(v);
  for (auto h : r->bh) {
    auto it = c.bases.find(h);
    if (it == c.bases.end()) continue;
    if (it->second.dptr && !it->second.external) vbe::dev_free(&c, ex, it->second.dptr, it->second.bytes());
    if (it->second.shadow) vbe::dev_free(&c, ex, it->second.shadow, it->second.bytes());
    c.bases.erase(it);
  }
  c.epoch++;
  if (r->ev) cudaEventDestroy(r->ev);
  r->ev = nullptr;
}

void admit(vbe_server* s, Req* r, int slot) {
  vbe::Ctx& c = s->ctx->c;
  vbe::Exec* ex = &s->slots[slot];
  r->slot = slot;
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
      c.views[h] = d;
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
      void* p = s->pinned.get(n);
      r->staging.push_back({(int)i, p});
      vbe::cuda_check(cudaMemcpyAsync(p, br.dptr, n, cudaMemcpyDeviceToHost, ex->stream), "request result");
    }
    vbe::cuda_check(cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming), "event");
    vbe::cuda_check(cudaEventRecord(r->ev, ex->stream), "event record");
    r->res.status = VBE_OK;
  } catch (const vbe::Error& e) {
    r->res.status = e.code;
    c.last_error = e.msg;
    cudaStreamSynchronize(ex->stream);
    finish_request(s, r);
    r->done = true;
    r->res.t_done_ns = now_ns();
    s->used -= r->footprint;
    s->slot_req[slot] = nullptr;
    return;
  }
  s->slot_req[slot] = r;
  s->inflight++;
}

void loop(vbe_server* s) {
  vbe::cuda_check(cudaSetDevice(s->ctx->c.device), "cudaSetDevice");
  std::unique_lock<std::mutex> lk(s->m);
  for (;;) {
    bool progressed = false;
    // completions
    for (size_t k = 0; k < s->slots.size(); ++k) {
      Req* r = s->slot_req[k];
      if (!r) continue;
      cudaError_t e = cudaEventQuery(r->ev);
      if (e == cudaErrorNotReady) continue;
      if (e != cudaSuccess) r->res.status = VBE_ERR_CUDA;
      else if (vbe::take_error_word(&s->ctx->c)) r->res.status = VBE_ERR_TIMEOUT;
      finish_request(s, r);
      r->res.t_done_ns = now_ns();
      r->done = true;
      s->used -= r->footprint;
      s->slot_req[k] = nullptr;
      s->inflight--;
      progressed = true;
    }
    if (progressed) s->cv_done.notify_all();
    // admissions, in arrival order
    while (!s->queue.empty()) {
      Req* r = s->queue.front();
      int free_slot = -1;
      for (size_t k = 0; k < s->slots.size(); ++k)
        if (!s->slot_req[k]) {
          free_slot = (int)k;
          break;
        }
      if (free_slot < 0) break;
      if (s->cfg.mem_cap_bytes && s->used + r->footprint > (int64_t)s->cfg.mem_cap_bytes) break;
      s->queue.pop_front();
      s->used += r->footprint;
      admit(s, r, free_slot);
      if (r->done) s->cv_done.notify_all();
      progressed = true;
    }
    if (s->stop && s->queue.empty() && s->inflight == 0) break;
    if (!progressed) {
      if (s->inflight > 0)
        s->cv_work.wait_for(lk, std::chrono::microseconds(20));
      else
        s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

}  // namespace

extern "C" {

int vbe_server_create(vbe_ctx* ctx, const vbe_server_config* cfg, vbe_server** out) {
  if (!ctx || !cfg || !out || cfg->slots <= 0) return VBE_ERR_INVALID;
  if (ctx->c.host_only) return VBE_ERR_NO_DEVICE;
  auto* s = new vbe_server();
  s->ctx = ctx;
  s->cfg = *cfg;
  s->ctx->c.cfg.flags = (s->ctx->c.cfg.flags & ~(uint32_t)(VBE_FUSE | VBE_PACK | VBE_AUTOTUNE)) |
                        (cfg->flags & (VBE_FUSE | VBE_PACK | VBE_AUTOTUNE));
  s->slots.resize(cfg->slots);
  s->slot_req.assign(cfg->slots, nullptr);
  try {
    for (auto& e : s->slots) {
      vbe::cuda_check(cudaStreamCreateWithFlags(&e.stream, cudaStreamNonBlocking), "cudaStreamCreate");
      vbe::ensure_scratch(&ctx->c, &e, 1 << 20, 1 << 16);
    }
  } catch (const vbe::Error& e) {
    ctx->c.last_error = e.msg;
    delete s;
    return e.code;
  }
  s->th = std::thread(loop, s);
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
  auto pred = [&] { return r->done; };
  if (timeout_ns < 0) {
    s->cv_done.wait(lk, pred);
  } else if (!s->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), pred)) {
    return VBE_ERR_TIMEOUT;
  }
  if (out) *out = r->res;
  int st = r->res.status;
  s->reqs.erase(it);
  return st;
}

int vbe_server_destroy(vbe_server* s) {
  if (!s) return VBE_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->m);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  for (auto& e : s->slots) {
    cudaStreamSynchronize(e.stream);
    vbe::release_exec(&s->ctx->c, &e);
    cudaStreamDestroy(e.stream);
  }
  delete s;
  return VBE_OK;
}

}  // extern "C"
