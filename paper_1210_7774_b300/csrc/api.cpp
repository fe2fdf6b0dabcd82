// extern "C" entry points of libvbe (declared in include/vbe.h).
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <thread>

#include <cctype>

#include "vbe_core.h"

using vbe::Ctx;
using vbe::Error;


namespace {

thread_local std::string g_last_error;

int record(vbe_ctx* ctx, const Error& e) {
  if (ctx) ctx->c.last_error = e.msg;
  g_last_error = e.msg;
  return e.code;
}

}  // namespace

#define API_BEGIN try {
#define API_END                                                   \
  }                                                               \
  catch (const Error& e) {                                        \
    return record(ctx, e);                                        \
  }                                                               \
  catch (const std::exception& e) {                               \
    return record(ctx, Error{VBE_ERR_INVALID, e.what()});         \
  }                                                               \
  return VBE_OK;

namespace vbe {
std::vector<char> compile_cached(Ctx* c, const std::string& src, bool* compiled);
}

namespace {

// ---------------------------------------------------------- host mirrors
//
// The data-ownership scheme of section "Vector Engine Manager" for a base
// with a host mirror. Rule 2: a batch may write every output and read every
// input it names, so before it runs the device copy of each mirrored base
// it uses must be current (uploaded from the mirror when only the mirror
// is), and afterwards the mirror of every base it wrote is stale and the
// host holds no write access to any base it named. Rule 3: an in-batch SYNC
// copies the device copy back to the mirror; an in-batch DISCARD drops the
// device copy. Rules 1 and 4: the host asks for read access (sync) or write
// access (release, or discard when it has already updated its copy), and
// the library tracks which copy is current.

struct Ref {
  int64_t base;
  int kind;  // 0 read, 1 write, 2 SYNC, 3 DISCARD, 4 FREE
  bool covers = false;  // a write that covers every element of the base
};

// the references an instruction makes to bases, reads before its write
void instr_refs(Ctx& c, const vbe_instr& in, std::vector<Ref>* out) {
  out->clear();
  auto base_of = [&](int64_t vh) -> const vbe::ViewDesc* {
    auto it = c.views.find(vh);
    return it == c.views.end() ? nullptr : &it->second;
  };
  const int op = in.op;
  if (op == VBE_OP_SYNC || op == VBE_OP_DISCARD || op == VBE_OP_FREE) {
    if (auto v = base_of(in.out))
      out->push_back({v->base, op == VBE_OP_SYNC ? 2 : (op == VBE_OP_DISCARD ? 3 : 4)});
    return;
  }
  for (int k = 0; k < 3; ++k) {
    if (k == in.const_slot || in.in[k] == 0) continue;
    if (auto v = base_of(in.in[k])) out->push_back({v->base, 0});
  }
  if (auto v = base_of(in.out)) {
    auto b = c.bases.find(v->base);
    bool covers = b != c.bases.end() && v->size() == b->second.nelem && !v->self_overlapping();
    out->push_back({v->base, 1, covers});
  }
}

// Before a batch: upload every mirrored base whose value only the mirror
// holds and which the batch reads (or writes only in part) before writing
// it whole; decide which in-batch SYNCs copy back. A read of a mirrored base
// after its DISCARD in the same batch, while the mirror holds its value,
// would need an upload in mid-batch and is rejected.
void mirror_before(Ctx& c, vbe::Exec* ex, const vbe_instr* prog, int64_t n) {
  if (c.n_mirrors == 0 || !prog) return;
  c.mirror_syncs.clear();
  std::unordered_map<int64_t, std::pair<bool, bool>> sim;  // base -> (device valid, host valid)
  std::vector<int64_t> upload;
  std::vector<Ref> refs;
  for (int64_t i = 0; i < n; ++i) {
    instr_refs(c, prog[i], &refs);
    for (auto& r : refs) {
      auto b = c.bases.find(r.base);
      if (b == c.bases.end() || !b->second.mirror) continue;
      auto s = sim.find(r.base);
      if (s == sim.end()) {
        s = sim.emplace(r.base, std::make_pair(b->second.dev_valid, b->second.host_valid)).first;
        bool needs_old = r.kind == 0 || r.kind == 2 || (r.kind == 1 && !r.covers);
        if (!s->second.first && s->second.second && needs_old) {
          upload.push_back(r.base);
          s->second.first = true;
        }
      }
      bool& dv = s->second.first;
      bool& hv = s->second.second;
      switch (r.kind) {
        case 0:
          if (!dv && hv)
            vbe::fail(VBE_ERR_INVALID, "the batch reads mirrored base " + std::to_string(r.base) +
                                           " after discarding it while the host copy holds its value");
          if (!dv)
            vbe::fail(VBE_ERR_UNINIT, "the batch reads mirrored base " + std::to_string(r.base) +
                                          ", whose value no copy holds (it was discarded)");
          break;
        case 1: dv = true; hv = false; break;
        case 2:
          c.mirror_syncs[r.base].push_back(dv);
          if (dv) hv = true;
          break;
        case 3: dv = false; break;
        default: break;
      }
    }
  }
  for (int64_t b : upload) {
    vbe::BaseRec& br = c.bases[b];
    if (!br.dptr) br.dptr = vbe::dev_alloc(&c, ex, br.bytes());
    vbe::stream_copy(&c, ex, br.dptr, br.mirror, br.bytes(), false);
    br.dev_valid = true;
    br.written = true;
  }
}

// After a batch was enqueued: which copies are current, and host access.
void mirror_after(Ctx& c, const vbe_instr* prog, int64_t n) {
  if (c.n_mirrors == 0 || !prog) return;
  std::vector<Ref> refs;
  for (int64_t i = 0; i < n; ++i) {
    instr_refs(c, prog[i], &refs);
    for (auto& r : refs) {
      auto b = c.bases.find(r.base);
      if (b == c.bases.end() || !b->second.mirror) continue;
      vbe::BaseRec& br = b->second;
      br.host_write = false;
      if (r.kind == 1) {
        br.dev_valid = true;
        br.host_valid = false;
      } else if (r.kind == 2) {
        if (br.dev_valid) br.host_valid = true;
      } else if (r.kind == 3) {
        br.dev_valid = false;
      }
    }
  }
  c.mirror_syncs.clear();
}

vbe::BaseRec& mirrored(Ctx& c, vbe_base base) {
  auto it = c.bases.find(base);
  if (it == c.bases.end()) vbe::fail(VBE_ERR_INVALID, "unknown base");
  if (!it->second.mirror) vbe::fail(VBE_ERR_INVALID, "base has no host mirror");
  return it->second;
}

// wait for everything enqueued so far (so no copy back to a mirror or
// kernel is still in flight)
void drain(Ctx& c) {
  if (!c.record) vbe::cuda_check(cudaStreamSynchronize(c.exec.stream), "sync");
  vbe::check_error_word(&c);
}

// read access: the mirror holds the current value on return
void mirror_read(Ctx& c, vbe::BaseRec& br) {
  drain(c);
  if (br.host_valid) return;
  if (!br.dev_valid || !br.dptr)
    vbe::fail(VBE_ERR_UNINIT, "no copy of the base holds a value (it was discarded or never written)");
  if (br.bytes() > 0) {
    if (c.record) memcpy(br.mirror, br.dptr, (size_t)br.bytes());
    else vbe::cuda_check(cudaMemcpy(br.mirror, br.dptr, (size_t)br.bytes(), cudaMemcpyDeviceToHost), "mirror sync");
  }
  br.host_valid = true;
}

}  // namespace

extern "C" {

const char* vbe_strerror(int code) {
  switch (code) {
    case VBE_OK: return "ok";
    case VBE_ERR_INVALID: return "invalid argument";
    case VBE_ERR_OUT_OF_BOUNDS: return "view out of bounds";
    case VBE_ERR_DTYPE: return "dtype rule violated";
    case VBE_ERR_SHAPE: return "shape mismatch";
    case VBE_ERR_OOM: return "out of device memory";
    case VBE_ERR_ADMISSION: return "request exceeds the memory cap";
    case VBE_ERR_COMPILE: return "kernel compilation failed";
    case VBE_ERR_TIMEOUT: return "timed out";
    case VBE_ERR_CUDA: return "CUDA error";
    case VBE_ERR_UNINIT: return "read of a base that was never written";
    case VBE_ERR_NO_DEVICE: return "no device (host-only context)";
    case VBE_ERR_OVERLAP: return "output view overlaps itself";
    case VBE_ERR_BUSY: return "server busy";
  }
  return "unknown error";
}

const char* vbe_last_error(vbe_ctx* ctx) { return ctx ? ctx->c.last_error.c_str() : g_last_error.c_str(); }

int vbe_init(const vbe_config* cfg, vbe_ctx** out) {
  vbe_ctx* ctx = nullptr;
  API_BEGIN
  if (!cfg || !out) vbe::fail(VBE_ERR_INVALID, "null config or output");
  std::unique_ptr<vbe_ctx> h(new vbe_ctx());
  Ctx& c = h->c;
  c.cfg = *cfg;
  c.cfg.cache_dir = nullptr;
  c.record = (cfg->flags & VBE_RECORD) != 0;
  c.host_only = (cfg->flags & VBE_HOST_ONLY) != 0 || c.record;
  if (c.record) {
    // launch shapes of recorded runs (small, so a CPU can execute them)
    if (const char* e = getenv("VBE_RECORD_BLOCK")) c.rec_block = atoi(e);
    if (const char* e = getenv("VBE_RECORD_U")) c.rec_U = atoi(e);
    c.sm_count = 2;
    if (const char* e = getenv("VBE_RECORD_SMS")) c.sm_count = atoi(e);
  }
  if (const char* e = getenv("VBE_STAGING")) c.force_bulk = atoi(e);
  if (const char* e = getenv("VBE_TILE")) c.force_tile = e;
  c.device = cfg->device;
  if (cfg->cache_dir) {
    // the context keeps its own copy of the path
    c.cache_dir_s = cfg->cache_dir;
    c.cfg.cache_dir = c.cache_dir_s.c_str();
  }
  if (!c.host_only) {
    vbe::cuda_check(cudaSetDevice(c.device), "cudaSetDevice");
    int sms = 0;
    vbe::cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device), "device attribute");
    c.sm_count = sms;
    if (cfg->stream) {
      c.exec.stream = (cudaStream_t)cfg->stream;
    } else {
      vbe::cuda_check(cudaStreamCreateWithFlags(&c.exec.stream, cudaStreamNonBlocking), "cudaStreamCreate");
      c.own_stream = true;
    }
    vbe::cuda_check(cudaDeviceGetDefaultMemPool(&c.pool, c.device), "default mem pool");
    uint64_t thr = UINT64_MAX;  // keep freed blocks cached in the pool
    cudaMemPoolSetAttribute(c.pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (!c.host_only || c.record) vbe::init_error_word(&c);
  vbe::load_tune(&c);
  *out = h.release();
  API_END
}

int vbe_finalize(vbe_ctx* ctx) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  Ctx& c = ctx->c;
  if (c.record) {
    vbe::release_exec(&c, &c.exec);
    vbe::release_error_word(&c);
    for (auto& kv : c.host_allocs) free((void*)kv.first);
    c.host_allocs.clear();
  }
  if (!c.host_only) {
    cudaStreamSynchronize(c.exec.stream);
    for (auto& kv : c.bases) {
      if (kv.second.dptr && !kv.second.external) cudaFreeAsync(kv.second.dptr, c.exec.stream);
      if (kv.second.shadow) cudaFreeAsync(kv.second.shadow, c.exec.stream);
    }
    for (auto& kv : c.batches)
      for (auto& v : kv.second.v) vbe::release_variant(v);
    for (auto ev : c.ticket_ring)
      if (ev) cudaEventDestroy(ev);
    cudaStreamSynchronize(c.exec.stream);
    vbe::release_exec(&c, &c.exec);
    vbe::release_error_word(&c);
    c.kernels.clear();  // modules no other context holds are unloaded
    if (c.own_stream) cudaStreamDestroy(c.exec.stream);
  }
  delete ctx;
  ctx = nullptr;
  API_END
}

int vbe_base_create(vbe_ctx* ctx, int32_t dtype, int64_t nelem, vbe_base* out) {
  API_BEGIN
  if (!ctx || !out) vbe::fail(VBE_ERR_INVALID, "null argument");
  vbe::itemsize(dtype);
  if (nelem < 0) vbe::fail(VBE_ERR_INVALID, "negative size");
  vbe::BaseRec b;
  b.dtype = dtype;
  b.nelem = nelem;
  int64_t h = ctx->c.next_handle++;
  ctx->c.bases[h] = b;
  *out = h;
  API_END
}

int vbe_base_register(vbe_ctx* ctx, int32_t dtype, int64_t nelem, void* device_ptr, vbe_base* out) {
  API_BEGIN
  if (!ctx || !out) vbe::fail(VBE_ERR_INVALID, "null argument");
  vbe::itemsize(dtype);
  if (nelem < 0) vbe::fail(VBE_ERR_INVALID, "negative size");
  if (!device_ptr && nelem > 0) vbe::fail(VBE_ERR_INVALID, "null device pointer");
  vbe::BaseRec b;
  b.dtype = dtype;
  b.nelem = nelem;
  b.dptr = device_ptr;
  b.external = true;
  b.written = true;
  int64_t h = ctx->c.next_handle++;
  ctx->c.bases[h] = b;
  *out = h;
  API_END
}

int vbe_base_upload(vbe_ctx* ctx, vbe_base base, const void* host, int64_t nbytes) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  Ctx& c = ctx->c;
  if (c.host_only && !c.record) vbe::fail(VBE_ERR_NO_DEVICE, "host-only context");
  auto it = c.bases.find(base);
  if (it == c.bases.end()) vbe::fail(VBE_ERR_INVALID, "unknown base");
  if (nbytes != it->second.bytes()) vbe::fail(VBE_ERR_INVALID, "upload size must equal the base size");
  if (nbytes > 0 && !host) vbe::fail(VBE_ERR_INVALID, "null host pointer");
  if (!it->second.dptr) it->second.dptr = vbe::dev_alloc(&c, &c.exec, it->second.bytes());
  it->second.written = true;
  if (it->second.mirror) {
    drain(c);  // no copy back to the mirror may still be in flight
    it->second.dev_valid = true;
    it->second.host_valid = false;
    it->second.host_write = false;
  }
  if (c.record) {
    if (nbytes > 0) memcpy(it->second.dptr, host, (size_t)nbytes);
    return VBE_OK;
  }
  if (nbytes > 0)
    vbe::cuda_check(cudaMemcpyAsync(it->second.dptr, host, (size_t)nbytes, cudaMemcpyHostToDevice, c.exec.stream),
                    "upload");
  vbe::cuda_check(cudaStreamSynchronize(c.exec.stream), "upload sync");
  API_END
}

int vbe_base_device_ptr(vbe_ctx* ctx, vbe_base base, void** out) {
  API_BEGIN
  if (!ctx || !out) vbe::fail(VBE_ERR_INVALID, "null argument");
  auto it = ctx->c.bases.find(base);
  if (it == ctx->c.bases.end()) vbe::fail(VBE_ERR_INVALID, "unknown base");
  *out = it->second.dptr;
  API_END
}

int vbe_view_create(vbe_ctx* ctx, vbe_base base, int64_t offset, int32_t ndim, const int64_t* shape,
                    const int64_t* strides, vbe_view* out) {
  API_BEGIN
  if (!ctx || !out) vbe::fail(VBE_ERR_INVALID, "null argument");
  if (ndim < 0 || ndim > VBE_MAX_NDIM) vbe::fail(VBE_ERR_INVALID, "ndim out of range");
  if (ndim > 0 && (!shape || !strides)) vbe::fail(VBE_ERR_INVALID, "null shape or strides");
  auto it = ctx->c.bases.find(base);
  if (it == ctx->c.bases.end()) vbe::fail(VBE_ERR_INVALID, "unknown base");
  vbe::ViewDesc v;
  v.base = base;
  v.offset = offset;
  v.ndim = ndim;
  for (int k = 0; k < ndim; ++k) {
    if (shape[k] < 0) vbe::fail(VBE_ERR_INVALID, "negative extent");
    v.shape[k] = shape[k];
    v.strides[k] = strides[k];
  }
  v.finish();
  if (v.size() > 0 && (v.lo < 0 || v.hi >= it->second.nelem))
    vbe::fail(VBE_ERR_OUT_OF_BOUNDS, "view reaches [" + std::to_string(v.lo) + ", " + std::to_string(v.hi) +
                                         "] outside a base of " + std::to_string(it->second.nelem) + " elements");
  int64_t h = ctx->c.next_handle++;
  vbe::add_view(&ctx->c, h, v);
  *out = h;
  API_END
}

int vbe_view_destroy(vbe_ctx* ctx, vbe_view view) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  auto it = ctx->c.views.find(view);
  if (it == ctx->c.views.end()) vbe::fail(VBE_ERR_INVALID, "unknown view");
  auto bt = ctx->c.bases.find(it->second.base);
  if (bt != ctx->c.bases.end()) {
    auto& vs = bt->second.views;
    vs.erase(std::remove(vs.begin(), vs.end(), view), vs.end());
  }
  ctx->c.views.erase(it);
  ctx->c.epoch++;
  API_END
}

int vbe_submit(vbe_ctx* ctx, const vbe_instr* prog, int64_t n, vbe_ticket* ticket) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  Ctx& c = ctx->c;
  if (c.host_only && !c.record) vbe::fail(VBE_ERR_NO_DEVICE, "host-only context");
  mirror_before(c, &c.exec, prog, n);
  vbe::exec_batch(&c, &c.exec, prog, n, true);
  mirror_after(c, prog, n);
  if (ticket && c.record) *ticket = 0;
  if (ticket && !c.record) {
    if (c.ticket_ring.empty()) c.ticket_ring.assign(Ctx::kTicketRing, nullptr);
    int64_t t = c.next_ticket++;
    cudaEvent_t& ev = c.ticket_ring[t % Ctx::kTicketRing];
    if (!ev) vbe::cuda_check(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    vbe::cuda_check(cudaEventRecord(ev, c.exec.stream), "event record");
    *ticket = t;
  }
  API_END
}

int vbe_wait(vbe_ctx* ctx, vbe_ticket ticket, int64_t timeout_ns) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  Ctx& c = ctx->c;
  if (c.record && ticket == 0) {
    vbe::check_error_word(&c);  // a recorded kernel's bounded wait may have run out
    return VBE_OK;
  }
  if (ticket <= 0 || ticket >= c.next_ticket || c.ticket_ring.empty()) vbe::fail(VBE_ERR_INVALID, "unknown ticket");
  cudaEvent_t ev = c.ticket_ring[ticket % Ctx::kTicketRing];
  if (timeout_ns < 0) {
    vbe::cuda_check(cudaEventSynchronize(ev), "wait");
  } else {
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      cudaError_t e = cudaEventQuery(ev);
      if (e == cudaSuccess) break;
      if (e != cudaErrorNotReady) vbe::cuda_check(e, "wait");
      auto el = std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count();
      if (el >= timeout_ns) vbe::fail(VBE_ERR_TIMEOUT, "ticket not complete within the limit");
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
  vbe::check_error_word(&c);
  API_END
}

int vbe_sync(vbe_ctx* ctx, vbe_base base, void* host_dst, int64_t nbytes) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  Ctx& c = ctx->c;
  if (c.host_only && !c.record) vbe::fail(VBE_ERR_NO_DEVICE, "host-only context");
  auto it = c.bases.find(base);
  if (it == c.bases.end()) vbe::fail(VBE_ERR_INVALID, "unknown base");
  if (nbytes < 0 || nbytes > it->second.bytes()) vbe::fail(VBE_ERR_INVALID, "bad size");
  if (it->second.mirror && !it->second.dev_valid) {
    // only the host mirror holds the value
    drain(c);
    if (!it->second.host_valid) vbe::fail(VBE_ERR_UNINIT, "no copy of the base holds a value");
    if (nbytes > 0) {
      if (!host_dst) vbe::fail(VBE_ERR_INVALID, "null host pointer");
      memcpy(host_dst, it->second.mirror, (size_t)nbytes);
    }
    return VBE_OK;
  }
  if (nbytes > 0 && !it->second.dptr) vbe::fail(VBE_ERR_UNINIT, "base was never written");
  if (c.record) {
    if (nbytes > 0) memcpy(host_dst, it->second.dptr, (size_t)nbytes);
    vbe::check_error_word(&c);
    return VBE_OK;
  }
  if (nbytes > 0) {
    if (!host_dst) vbe::fail(VBE_ERR_INVALID, "null host pointer");
    vbe::cuda_check(cudaMemcpyAsync(host_dst, it->second.dptr, (size_t)nbytes, cudaMemcpyDeviceToHost, c.exec.stream),
                    "sync copy");
  }
  vbe::cuda_check(cudaStreamSynchronize(c.exec.stream), "sync");
  vbe::check_error_word(&c);
  API_END
}

int vbe_discard(vbe_ctx* ctx, vbe_base base) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  auto it = ctx->c.bases.find(base);
  if (it == ctx->c.bases.end()) vbe::fail(VBE_ERR_INVALID, "unknown base");
  it->second.written = false;
  it->second.dev_valid = false;
  API_END
}

int vbe_mirror_attach(vbe_ctx* ctx, vbe_base base, void* host, int64_t nbytes) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  Ctx& c = ctx->c;
  auto it = c.bases.find(base);
  if (it == c.bases.end()) vbe::fail(VBE_ERR_INVALID, "unknown base");
  if (nbytes != it->second.bytes()) vbe::fail(VBE_ERR_INVALID, "mirror size must equal the base size");
  if (!host && nbytes > 0) vbe::fail(VBE_ERR_INVALID, "null host pointer");
  if (it->second.external) vbe::fail(VBE_ERR_INVALID, "a registered base cannot have a host mirror");
  if (it->second.mirror) vbe::fail(VBE_ERR_INVALID, "base already has a host mirror");
  drain(c);  // work already enqueued on the base is finished
  it->second.mirror = host ? host : (void*)&it->second;  // an empty base needs no memory
  c.n_mirrors++;
  it->second.host_valid = true;
  it->second.dev_valid = false;
  it->second.host_write = true;
  API_END
}

int vbe_mirror_sync(vbe_ctx* ctx, vbe_base base) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  Ctx& c = ctx->c;
  mirror_read(c, mirrored(c, base));
  API_END
}

int vbe_mirror_release(vbe_ctx* ctx, vbe_base base) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  Ctx& c = ctx->c;
  vbe::BaseRec& br = mirrored(c, base);
  mirror_read(c, br);
  br.dev_valid = false;
  br.host_write = true;
  API_END
}

int vbe_mirror_discard(vbe_ctx* ctx, vbe_base base) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  Ctx& c = ctx->c;
  vbe::BaseRec& br = mirrored(c, base);
  drain(c);
  br.host_valid = true;
  br.dev_valid = false;
  br.host_write = true;
  API_END
}

int vbe_mirror_state(vbe_ctx* ctx, vbe_base base, int32_t* state) {
  API_BEGIN
  if (!ctx || !state) vbe::fail(VBE_ERR_INVALID, "null argument");
  vbe::BaseRec& br = mirrored(ctx->c, base);
  *state = (br.dev_valid ? VBE_MIRROR_DEVICE : 0) | (br.host_valid ? VBE_MIRROR_HOST : 0) |
           (br.host_write ? VBE_MIRROR_HOST_WRITE : 0);
  API_END
}

int vbe_free(vbe_ctx* ctx, vbe_base base) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  Ctx& c = ctx->c;
  auto it = c.bases.find(base);
  if (it == c.bases.end()) vbe::fail(VBE_ERR_INVALID, "unknown base");
  if (it->second.dptr && !it->second.external) vbe::dev_free(&c, &c.exec, it->second.dptr, it->second.bytes());
  if (it->second.shadow) vbe::dev_free(&c, &c.exec, it->second.shadow, it->second.bytes());
  vbe::erase_views_of(&c, it->second);
  c.bases.erase(it);
  c.epoch++;
  API_END
}

int vbe_plan(vbe_ctx* ctx, const vbe_instr* prog, int64_t n, int32_t want_source, char* buf, int64_t cap,
             int64_t* needed) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  Ctx& c = ctx->c;
  std::vector<vbe::RInstr> rp = vbe::resolve_batch(&c, prog, n);
  size_t nb = c.bases.size();
  (void)nb;
  std::vector<int64_t> before;
  for (auto& kv : c.bases) before.push_back(kv.first);
  vbe::Plan p = vbe::make_plan(&c, rp, (c.cfg.flags & VBE_FUSE) != 0, (c.cfg.flags & VBE_PACK) != 0);
  std::string js = vbe::plan_json(&c, rp, p, want_source != 0);
  for (auto& st : p.staging) c.bases.erase(st.first);
  if (needed) *needed = (int64_t)js.size() + 1;
  if (buf && cap > 0) {
    size_t k = std::min<size_t>((size_t)cap - 1, js.size());
    memcpy(buf, js.data(), k);
    buf[k] = '\0';
  }
  API_END
}

// Compile (without loading) the kernels a batch would use: a host-side
// check that the generated sources are valid CUDA for sm_103a.
int vbe_plan_compile(vbe_ctx* ctx, const vbe_instr* prog, int64_t n, int64_t* nkernels) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  Ctx& c = ctx->c;
  std::vector<vbe::RInstr> rp = vbe::resolve_batch(&c, prog, n);
  vbe::Plan p = vbe::make_plan(&c, rp, (c.cfg.flags & VBE_FUSE) != 0, (c.cfg.flags & VBE_PACK) != 0);
  int64_t k = 0;
  std::vector<std::string> srcs;
  for (auto& it : p.items) {
    if (it.kind == 2) {
      srcs.push_back(vbe::generate_group_source(*it.group, nullptr, nullptr));
      ++k;
      continue;
    }
    if (it.kind != 0) continue;
    std::vector<uintptr_t> lp(it.run.loads.size(), 0), sp(it.run.stores.size(), 0);
    vbe::Canon cn = vbe::canonicalize(it.run, true, lp, sp, 0);
    srcs.push_back(vbe::generate_source(it.run, cn, nullptr));
    ++k;
  }
  if (srcs.size() == 1) vbe::compile_cached(&c, srcs[0], nullptr);
  else vbe::precompile(&c, srcs);
  for (auto& st : p.staging) c.bases.erase(st.first);
  if (nkernels) *nkernels = k;
  API_END
}

int vbe_op_register(vbe_ctx* ctx, const char* name, const char* body, int32_t nin, int32_t dtype,
                    int32_t* opcode) {
  API_BEGIN
  if (!ctx || !name || !body || !opcode) vbe::fail(VBE_ERR_INVALID, "null argument");
  Ctx& c = ctx->c;
  if (nin < 1 || nin > 3 || (dtype != VBE_FLOAT32 && dtype != VBE_FLOAT64 && dtype != VBE_INT64))
    vbe::fail(VBE_ERR_INVALID, "a user operation takes 1 to 3 inputs of float32, float64 or int64");
  // the body must compile for the target before the opcode exists
  const std::string T = vbe::ctype(dtype), nm = name;
  std::string src = "typedef long long i64;\n__device__ __forceinline__ " + T + " vbe_user_" + nm + "(" + T + " a";
  if (nin > 1) src += ", " + T + " b";
  if (nin > 2) src += ", " + T + " c";
  src += ") {\n" + std::string(body) + "\n}\nextern \"C\" __global__ void vbe_user_probe(" + T + "* o, const " + T +
         "* x) { o[0] = vbe_user_" + nm + "(x[0]";
  if (nin > 1) src += ", x[1]";
  if (nin > 2) src += ", x[2]";
  src += "); }\n";
  for (char ch : nm)
    if (!(isalnum((unsigned char)ch) || ch == '_')) vbe::fail(VBE_ERR_INVALID, "operation name must be an identifier");
  vbe::compile_cached(&c, src, nullptr);
  *opcode = vbe::register_user_op(nm, body, nin, dtype);
  API_END
}

int vbe_views_may_overlap(vbe_ctx* ctx, vbe_view a, vbe_view b, int32_t* out) {
  API_BEGIN
  if (!ctx || !out) vbe::fail(VBE_ERR_INVALID, "null argument");
  auto ia = ctx->c.views.find(a), ib = ctx->c.views.find(b);
  if (ia == ctx->c.views.end() || ib == ctx->c.views.end()) vbe::fail(VBE_ERR_INVALID, "unknown view");
  *out = vbe::may_overlap(ia->second, ib->second) ? 1 : 0;
  API_END
}

int vbe_debug_take_launches(vbe_ctx* ctx, char* buf, int64_t cap, int64_t* needed) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  Ctx& c = ctx->c;
  if (!c.record) vbe::fail(VBE_ERR_INVALID, "not a recording context");
  std::string js = "{\"allocs\":[";
  bool first = true;
  for (auto& kv : c.host_allocs) {
    js += (first ? "[" : ",[") + std::to_string(kv.first) + "," + std::to_string(kv.second) + "]";
    first = false;
  }
  js += "],\"launches\":[";
  for (size_t i = 0; i < c.rec_launches.size(); ++i) js += (i ? "," : "") + c.rec_launches[i];
  js += "],\"sources\":{";
  first = true;
  for (auto& kv : c.rec_sources) {
    std::string esc;
    for (char ch : kv.second) {
      if (ch == '"') esc += "\\\"";
      else if (ch == '\\') esc += "\\\\";
      else if (ch == '\n') esc += "\\n";
      else esc += ch;
    }
    js += (first ? "\"" : ",\"") + kv.first + "\":\"" + esc + "\"";
    first = false;
  }
  js += "}}";
  if (needed) *needed = (int64_t)js.size() + 1;
  if (buf && cap >= (int64_t)js.size() + 1) {
    memcpy(buf, js.data(), js.size());
    buf[js.size()] = '\0';
    c.rec_launches.clear();
  }
  API_END
}

int vbe_debug_set_wait_polls(vbe_ctx* ctx, int64_t polls) {
  API_BEGIN
  if (!ctx) vbe::fail(VBE_ERR_INVALID, "null context");
  Ctx& c = ctx->c;
  if (polls > (int64_t)(1u << 24)) vbe::fail(VBE_ERR_INVALID, "at most 2^24 polls");
  if (!c.host_only) vbe::cuda_check(cudaStreamSynchronize(c.exec.stream), "sync");
  c.cwait = polls < 0 ? -1 : polls;
  // cached launches hold kernels compiled with the previous limit
  for (auto& kv : c.batches)
    for (auto& v : kv.second.v) vbe::release_variant(v);
  c.batches.clear();
  API_END
}

int vbe_get_stats(vbe_ctx* ctx, vbe_stats* out) {
  API_BEGIN
  if (!ctx || !out) vbe::fail(VBE_ERR_INVALID, "null argument");
  *out = ctx->c.stats;
  API_END
}

}  // extern "C"
