// Runtime: NVRTC compilation and module cache, device memory, launch
// shapes and their autotuning, batch execution, CUDA-graph replay of
// repeated batches and packing of independent runs into one launch.
#include <cuda.h>  // tensor-map types; the encoder comes from the driver entry point
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <set>
#include <unordered_set>
#include <sstream>

#include "vbe_core.h"

namespace vbe {

// ------------------------------------------------------------------ NVRTC

static std::vector<char> nvrtc_compile(const std::string& src, std::string* log) {
  nvrtcProgram prog;
  static const auto headers = nvrtc_headers();
  std::vector<const char*> htext, hname;
  for (auto& h : headers) {
    hname.push_back(h.first);
    htext.push_back(h.second);
  }
  if (nvrtcCreateProgram(&prog, src.c_str(), "vbe_run.cu", (int)headers.size(), htext.data(), hname.data()) !=
      NVRTC_SUCCESS)
    fail(VBE_ERR_COMPILE, "nvrtcCreateProgram failed");
  // IEEE arithmetic: no contraction into FMA, no flush to zero, correctly
  // rounded division and square root
  const char* opts[] = {"-arch=sm_103a", "--fmad=false", "-ftz=false", "-prec-div=true",
                        "-prec-sqrt=true", "-std=c++17", "-lineinfo"};
  nvrtcResult res = nvrtcCompileProgram(prog, (int)(sizeof(opts) / sizeof(opts[0])), opts);
  size_t ls = 0;
  nvrtcGetProgramLogSize(prog, &ls);
  std::string lg(ls, '\0');
  if (ls) nvrtcGetProgramLog(prog, &lg[0]);
  if (log) *log = lg;
  if (res != NVRTC_SUCCESS) {
    nvrtcDestroyProgram(&prog);
    fail(VBE_ERR_COMPILE, "NVRTC: " + std::string(nvrtcGetErrorString(res)) + "\n" + lg);
  }
  size_t n = 0;
  nvrtcGetCUBINSize(prog, &n);
  std::vector<char> cubin(n);
  nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  return cubin;
}

std::string src_key(const std::string& src) {
  return hex64(hash64(src.data(), src.size(), 1)) + hex64(hash64(src.data(), src.size(), 0x5bd1e995ull));
}

std::vector<char> compile_cached(Ctx* c, const std::string& src, bool* compiled) {
  std::string key = src_key(src);
  std::string path;
  if (c->cfg.cache_dir && *c->cfg.cache_dir) {
    path = std::string(c->cfg.cache_dir) + "/" + key + ".cubin";
    std::ifstream f(path, std::ios::binary);
    if (f) {
      std::vector<char> b((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
      if (!b.empty()) {
        if (compiled) *compiled = false;
        return b;
      }
    }
  }
  std::vector<char> cubin = nvrtc_compile(src, nullptr);
  c->stats.compiles++;
  if (compiled) *compiled = true;
  if (!path.empty()) {
    mkdir(c->cfg.cache_dir, 0755);
    std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
    std::ofstream f(tmp, std::ios::binary);
    f.write(cubin.data(), (std::streamsize)cubin.size());
    f.close();
    rename(tmp.c_str(), path.c_str());
  }
  return cubin;
}

// Tuning choices across processes: "<key> <block> <U> <maxreg> <bulk_chunk>
// <grid_mult>" lines in <cache_dir>/tune_<device model>_<SMs>.txt, appended
// as choices are made (later lines win), so a process that meets a kernel
// signature and size class tuned before skips the timing and launches what
// was chosen then. Keys hold no spaces (source hashes, size classes).
// Contexts of one process share their choices too (a serving process runs
// one context per scheduler thread): a choice made by one is found by the
// others, keyed by the device model and SM count.
namespace {
std::mutex g_tune_mu;
std::unordered_map<std::string, TuneChoice> g_tune;
}  // namespace

void load_tune(Ctx* c) {
  if (c->host_only) return;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const std::string name(prop.name);
  c->tune_device = hex64(hash64(name.data(), name.size(), 7)) + "_" + std::to_string(c->sm_count);
  if (!c->cfg.cache_dir || !*c->cfg.cache_dir) return;
  c->tune_file = std::string(c->cfg.cache_dir) + "/tune_" + c->tune_device + ".txt";
  std::ifstream f(c->tune_file);
  std::string line;
  while (std::getline(f, line)) {
    std::istringstream ls(line);
    std::string key;
    TuneChoice tc;
    // a line that does not parse, or whose values lie outside what the
    // tuner ever writes (a damaged or foreign file), is ignored: its key is
    // tuned afresh
    std::string extra;
    if (ls >> key >> tc.block >> tc.U >> tc.maxreg >> tc.bulk_chunk >> tc.grid_mult && !(ls >> extra) &&
        tc.block >= 1 && tc.block <= 1024 && tc.U >= 1 && tc.U <= 1024 &&
        (tc.maxreg == 0 || std::find(std::begin(kRegCaps), std::end(kRegCaps), tc.maxreg) != std::end(kRegCaps)) &&
        tc.bulk_chunk >= 0 && tc.bulk_chunk <= (1 << 24) && tc.grid_mult >= 0 && tc.grid_mult <= 64) {
      c->tune[key] = tc;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune.emplace(c->tune_device + ":" + key, tc);
    }
  }
}

bool recall_tune(Ctx* c, const std::string& key, TuneChoice* out) {
  auto it = c->tune.find(key);
  if (it != c->tune.end()) {
    *out = it->second;
    return true;
  }
  if (c->tune_device.empty()) return false;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto g = g_tune.find(c->tune_device + ":" + key);
  if (g == g_tune.end()) return false;
  c->tune[key] = *out = g->second;
  return true;
}

void remember_tune(Ctx* c, const std::string& key, const TuneChoice& tc) {
  c->tune[key] = tc;
  if (c->tune_device.empty()) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);  // one line at a time from the contexts of this process
  g_tune[c->tune_device + ":" + key] = tc;
  if (c->tune_file.empty()) return;
  mkdir(c->cfg.cache_dir, 0755);
  std::ofstream f(c->tune_file, std::ios::app);
  f << key << ' ' << tc.block << ' ' << tc.U << ' ' << tc.maxreg << ' ' << tc.bulk_chunk << ' ' << tc.grid_mult
    << '\n';
}

// the source a context compiles: with a wait limit set for tests, the
// limit is defined ahead of the text (and so is part of the cache key)
static bool with_wait_limit(const Ctx* c, const std::string& src, std::string* src2, std::string* key2) {
  if (c->cwait < 0) return false;
  *src2 = "#define VBE_CWAIT " + std::to_string(c->cwait) + "u\n" + src;
  *key2 = src_key(*src2);
  return true;
}

Kernel::~Kernel() {
  if (lib) cudaLibraryUnload(lib);
}

namespace {
std::mutex g_lib_mu;
std::unordered_map<std::string, std::weak_ptr<Kernel>> g_libs;  // by source key

// the module of this source key if some context of the process holds it
std::shared_ptr<Kernel> find_library(const std::string& key) {
  std::lock_guard<std::mutex> lk(g_lib_mu);
  auto it = g_libs.find(key);
  return it == g_libs.end() ? nullptr : it->second.lock();
}

// load a compiled module, unless another thread loaded it meanwhile
std::shared_ptr<Kernel> load_library(const std::string& key, const std::vector<char>& cubin) {
  std::lock_guard<std::mutex> lk(g_lib_mu);
  auto& slot = g_libs[key];
  if (auto k = slot.lock()) return k;
  auto k = std::make_shared<Kernel>();
  cuda_check(cudaLibraryLoadData(&k->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0),
             "cudaLibraryLoadData");
  slot = k;
  return k;
}
}  // namespace

// Compile, in parallel threads, every source not loaded yet (first sight
// of a batch), then load the modules.
void precompile(Ctx* c, const std::vector<std::string>& srcs, const std::vector<std::string>* keys) {
  std::vector<std::string> todo, todo_keys;
  std::set<std::string> seen;
  for (size_t i = 0; i < srcs.size(); ++i) {
    std::string src2, key2;
    const bool adj = with_wait_limit(c, srcs[i], &src2, &key2);
    const std::string k = adj ? key2 : (keys ? (*keys)[i] : src_key(srcs[i]));
    if (c->kernels.count(k) || seen.count(k)) continue;
    if (!c->host_only) {
      if (auto shared = find_library(k)) {  // another context of the process loaded it
        c->kernels[k] = shared;
        continue;
      }
    }
    seen.insert(k);
    todo.push_back(adj ? src2 : srcs[i]);
    todo_keys.push_back(k);
  }
  if (todo.size() <= 1) return;
  std::vector<std::vector<char>> bins(todo.size());
  std::vector<std::string> errs(todo.size());
  std::atomic<size_t> next{0};
  int nt = (int)std::min<size_t>(todo.size(), std::max(1u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  std::mutex mu;
  for (int t = 0; t < nt; ++t) {
    th.emplace_back([&]() {
      for (;;) {
        size_t i = next++;
        if (i >= todo.size()) return;
        try {
          bool compiled = false;
          Ctx tmp_view;  // only cfg.cache_dir is read
          tmp_view.cfg.cache_dir = c->cfg.cache_dir;
          bins[i] = compile_cached(&tmp_view, todo[i], &compiled);
          if (compiled) {
            std::lock_guard<std::mutex> lk(mu);
            c->stats.compiles++;
          }
        } catch (const Error& e) {
          errs[i] = e.msg;
        }
      }
    });
  }
  for (auto& t : th) t.join();
  for (size_t i = 0; i < todo.size(); ++i) {
    if (!errs[i].empty()) fail(VBE_ERR_COMPILE, errs[i]);
    if (c->host_only) continue;
    c->kernels[todo_keys[i]] = load_library(todo_keys[i], bins[i]);
  }
}

std::shared_ptr<Kernel> get_kernel(Ctx* c, const std::string& src_in, const std::string* key_in) {
  std::string src2, key2;
  const bool adj = with_wait_limit(c, src_in, &src2, &key2);
  const std::string& src = adj ? src2 : src_in;
  const std::string key = adj ? key2 : (key_in ? *key_in : src_key(src_in));
  auto it = c->kernels.find(key);
  if (it != c->kernels.end()) return it->second;
  if (c->record) {
    c->rec_sources[key] = src;
    // with a wait limit set, launches of this source are recorded under the
    // key of the text actually compiled
    if (adj) c->rec_alias[key_in ? *key_in : src_key(src_in)] = key;
    auto k = std::make_shared<Kernel>();
    c->kernels[key] = k;
    return k;
  }
  if (c->host_only) fail(VBE_ERR_NO_DEVICE, "host-only context cannot load kernels");
  if (auto k = find_library(key)) return c->kernels[key] = k;
  std::vector<char> cubin = compile_cached(c, src, nullptr);
  return c->kernels[key] = load_library(key, cubin);
}

static cudaKernel_t kernel_fn(Kernel* k, const std::string& name) {
  if (!k->lib) return (cudaKernel_t)(uintptr_t)1;  // recording: never launched
  std::lock_guard<std::mutex> lk(k->mu);
  auto it = k->fn.find(name);
  if (it != k->fn.end()) return it->second;
  cudaKernel_t f;
  cuda_check(cudaLibraryGetKernel(&f, k->lib, name.c_str()), "cudaLibraryGetKernel");
  k->fn[name] = f;
  return f;
}

// ----------------------------------------------------------------- memory

static void* host_alloc(Ctx* c, int64_t bytes) {
  size_t n = ((size_t)bytes + 255) / 256 * 256;
  void* p = aligned_alloc(256, n);
  if (!p) fail(VBE_ERR_OOM, "host allocation failed");
  memset(p, 0, n);
  c->host_allocs[(uintptr_t)p] = (size_t)bytes;
  return p;
}

static void host_free(Ctx* c, void* p) {
  c->host_allocs.erase((uintptr_t)p);
  free(p);
}

// The error word: staged kernels whose bounded waits ran out set it. It
// lives in mapped host memory, so the host reads it after a synchronisation
// without a copy.
void init_error_word(Ctx* c) {
  if (c->record) {
    c->err_word = c->err_word_dev = (unsigned*)host_alloc(c, 64);
    return;
  }
  void* p = nullptr;
  cuda_check(cudaHostAlloc(&p, 64, cudaHostAllocMapped | cudaHostAllocPortable), "cudaHostAlloc(error word)");
  memset(p, 0, 64);
  void* d = nullptr;
  cuda_check(cudaHostGetDevicePointer(&d, p, 0), "cudaHostGetDevicePointer(error word)");
  c->err_word = (unsigned*)p;
  c->err_word_dev = (unsigned*)d;
}

void release_error_word(Ctx* c) {
  if (!c->err_word) return;
  if (c->record) host_free(c, c->err_word);
  else cudaFreeHost(c->err_word);
  c->err_word = c->err_word_dev = nullptr;
}

bool take_error_word(Ctx* c) {
  if (!c->err_word) return false;
  volatile unsigned* w = c->err_word;
  if (*w == 0) return false;
  *w = 0;
  return true;
}

void check_error_word(Ctx* c) {
  if (take_error_word(c))
    fail(VBE_ERR_TIMEOUT, "a staged kernel's bulk-copy wait ran out; the results of its batch are invalid");
}

void* dev_alloc(Ctx* c, Exec* ex, int64_t bytes) {
  if (bytes <= 0) bytes = 16;
  if (c->record) {
    void* p = host_alloc(c, bytes);
    c->stats.bytes_allocated += bytes;
    c->stats.peak_bytes = std::max(c->stats.peak_bytes, c->stats.bytes_allocated);
    return p;
  }
  if (c->cfg.mem_cap_bytes && c->stats.bytes_allocated + bytes > (int64_t)c->cfg.mem_cap_bytes)
    fail(VBE_ERR_OOM, "allocation of " + std::to_string(bytes) + " bytes exceeds the memory cap");
  void* p = nullptr;
  cuda_check(cudaMallocAsync(&p, (size_t)bytes, ex->stream), "cudaMallocAsync");
  c->stats.bytes_allocated += bytes;
  c->stats.peak_bytes = std::max(c->stats.peak_bytes, c->stats.bytes_allocated);
  return p;
}

void dev_free(Ctx* c, Exec* ex, void* p, int64_t bytes) {
  if (!p) return;
  if (bytes <= 0) bytes = 16;
  c->stats.bytes_allocated -= bytes;
  if (c->record) {
    // recorded launches run later, so a freed block stays allocated (and
    // addressable) until the context ends, like a stream-ordered free
    return;
  }
  cudaFreeAsync(p, ex->stream);
}

void ensure_scratch(Ctx* c, Exec* ex, int64_t partials, int64_t counters) {
  Scratch& s = ex->scratch;
  if (s.n_partials >= partials && s.n_counters >= counters) return;
  if (c->record) {
    s.n_partials = std::max<int64_t>(partials, 1 << 20);
    s.n_counters = std::max<int64_t>(counters, 1 << 16);
    s.partials = host_alloc(c, s.n_partials * 8);
    s.counters = (unsigned int*)host_alloc(c, s.n_counters * 4);
    return;
  }
  // grow: wait for users of the old buffers, then replace them
  cuda_check(cudaStreamSynchronize(ex->stream), "cudaStreamSynchronize");
  if (s.partials) cudaFree(s.partials);
  if (s.counters) cudaFree(s.counters);
  // cached graphs may reference the old buffers
  for (auto& kv : c->batches)
    for (auto& v : kv.second.v) release_variant(v);
  s.n_partials = std::max<int64_t>(partials, 1 << 20);
  s.n_counters = std::max<int64_t>(counters, 1 << 16);
  cuda_check(cudaMalloc(&s.partials, (size_t)s.n_partials * 8), "cudaMalloc(partials)");
  cuda_check(cudaMalloc((void**)&s.counters, (size_t)s.n_counters * 4), "cudaMalloc(counters)");
  cuda_check(cudaMemset(s.counters, 0, (size_t)s.n_counters * 4), "cudaMemset(counters)");
}

void release_variant(CachedVariant& v) {
  if (v.exec) cudaGraphExecDestroy(v.exec);
  if (v.graph) cudaGraphDestroy(v.graph);
  for (void* p : v.keep) cudaFree(p);
  v.exec = nullptr;
  v.graph = nullptr;
  v.keep.clear();
  v.launches = 0;
}

void release_exec(Ctx* c, Exec* ex) {
  if (c->record) {
    if (ex->scratch.partials) host_free(c, ex->scratch.partials);
    if (ex->scratch.counters) host_free(c, ex->scratch.counters);
    ex->scratch = Scratch();
    return;
  }
  if (ex->scratch.partials) cudaFree(ex->scratch.partials);
  if (ex->scratch.counters) cudaFree(ex->scratch.counters);
  ex->scratch = Scratch();
  if (ex->ev0) cudaEventDestroy(ex->ev0);
  if (ex->ev1) cudaEventDestroy(ex->ev1);
  ex->ev0 = ex->ev1 = nullptr;
}

// --------------------------------------------------------------- launches

struct Launch {
  cudaKernel_t fn = nullptr;
  std::string key, entry;          // module and kernel name (recorded launches)
  unsigned grid = 1, block = 256;
  unsigned smem = 0;               // dynamic shared memory bytes (staged kernels)
  std::vector<int64_t> words;      // by-value parameter block (single runs)
  bool packed = false;
  std::vector<int64_t> descs;      // packed: words of every instance
  std::vector<int64_t> prefix;     // packed: chunk prefix sums
  int ninst = 0;
  int64_t total = 0, chunk = 0;
  void* d_descs = nullptr;         // device copies (packed)
  void* d_prefix = nullptr;
  int64_t d_bytes = 0;
  bool tma = false;                // a tile-fused group in the tensor-copy form
  bool sweep = false;              // a tile-fused group in the row-sweep form
};

namespace {

int occupancy(cudaKernel_t fn, int block, size_t smem = 0) {
  int n = 0;
  if (fn == (cudaKernel_t)(uintptr_t)1) return 2;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, (const void*)fn, block, smem) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    n = std::max(1, 2048 / block);
  }
  return n;
}

uintptr_t base_ptr(Ctx* c, int64_t b) {
  auto it = c->bases.find(b);
  if (it == c->bases.end()) fail(VBE_ERR_INVALID, "base vanished during execution");
  return (uintptr_t)it->second.dptr;
}

std::string words_json(const std::vector<int64_t>& w) {
  std::string s = "[";
  for (size_t i = 0; i < w.size(); ++i) s += (i ? "," : "") + std::to_string(w[i]);
  return s + "]";
}

}  // namespace

void stream_copy(Ctx* c, Exec* ex, void* dst, const void* src, int64_t bytes, bool to_host) {
  if (bytes <= 0) return;
  if (c->record) {
    // executed by whoever runs the recorded launches, in order with them
    c->rec_launches.push_back("{\"copy\":true,\"dst\":" + std::to_string((uintptr_t)dst) + ",\"src\":" +
                              std::to_string((uintptr_t)src) + ",\"bytes\":" + std::to_string(bytes) + "}");
    return;
  }
  cuda_check(cudaMemcpyAsync(dst, src, (size_t)bytes, to_host ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice,
                             ex->stream),
             to_host ? "copy to the host mirror" : "copy from the host mirror");
}

namespace {

void record_launch(Ctx* c, Exec* ex, Launch& L) {
  std::string key = L.key;
  if (c->cwait >= 0) {
    auto a = c->rec_alias.find(L.key);
    if (a != c->rec_alias.end()) key = a->second;
  }
  std::string j = "{\"key\":\"" + key + "\",\"entry\":\"" + L.entry + "\",\"grid\":" +
                  std::to_string(L.grid) + ",\"block\":" + std::to_string(L.block) + ",\"smem\":" +
                  std::to_string(L.smem);
  if (L.packed) {
    int64_t db = (int64_t)(L.descs.size() * 8), pb = (int64_t)(L.prefix.size() * 8);
    char* d = (char*)dev_alloc(c, ex, db + pb);  // kept until the context ends
    memcpy(d, L.descs.data(), db);
    memcpy(d + db, L.prefix.data(), pb);
    unsigned* work = ex->scratch.counters + (ex->scratch.n_counters - 1);
    j += ",\"packed\":true,\"descs\":" + std::to_string((uintptr_t)d) + ",\"prefix\":" +
         std::to_string((uintptr_t)(d + db)) + ",\"ninst\":" + std::to_string(L.ninst) + ",\"total\":" +
         std::to_string(L.total) + ",\"chunk\":" + std::to_string(L.chunk) + ",\"work\":" +
         std::to_string((uintptr_t)work);
  } else {
    j += ",\"words\":" + words_json(L.words);
  }
  c->rec_launches.push_back(j + "}");
  c->stats.kernel_launches++;
  if (L.packed) c->stats.packed_launches++;
  if (L.sweep) c->stats.sweep_group_launches++;
}

// Every generated kernel starts with griddepcontrol.wait, so it may be
// launched with programmatic stream serialization: its blocks are scheduled
// while the previous kernel on the stream drains, and wait there for it.
cudaError_t launch_pdl(cudaKernel_t fn, unsigned grid, unsigned block, void** args, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, (const void*)fn, args);
}

void issue(Ctx* c, Exec* ex, Launch& L, bool capturing) {
  if (c->record) {
    record_launch(c, ex, L);
    return;
  }
  cudaStream_t s = ex->stream;
  if (L.packed) {
    if (!capturing) {
      int64_t db = (int64_t)(L.descs.size() * 8), pb = (int64_t)(L.prefix.size() * 8);
      char* d = (char*)dev_alloc(c, ex, db + pb);
      cuda_check(cudaMemcpyAsync(d, L.descs.data(), db, cudaMemcpyHostToDevice, s), "upload descriptors");
      cuda_check(cudaMemcpyAsync(d + db, L.prefix.data(), pb, cudaMemcpyHostToDevice, s), "upload prefix");
      L.d_descs = d;
      L.d_prefix = d + db;
      L.d_bytes = db + pb;
    }
    unsigned* work = ex->scratch.counters + (ex->scratch.n_counters - 1);
    cuda_check(cudaMemsetAsync(work, 0, 4, s), "cudaMemsetAsync(work)");
    void* a0 = L.d_descs;
    void* a1 = L.d_prefix;
    int a2 = L.ninst;
    long long a3 = L.total, a4 = L.chunk;
    void* a5 = work;
    void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5};
    cuda_check(launch_pdl(L.fn, L.grid, L.block, args, 0, s), "launch (packed)");
    if (!capturing) {
      dev_free(c, ex, L.d_descs, L.d_bytes);
      L.d_descs = L.d_prefix = nullptr;
    }
  } else {
    void* args[] = {(void*)L.words.data()};
    cuda_check(launch_pdl(L.fn, L.grid, L.block, args, L.smem, s), "launch");
  }
  if (!capturing) c->stats.kernel_launches++;
  if (!capturing && L.packed) c->stats.packed_launches++;
  if (L.tma) c->stats.tma_group_launches++;
  if (L.sweep) c->stats.sweep_group_launches++;
}

struct RunPtrs {
  std::vector<uintptr_t> lp, sp;
  uintptr_t rp = 0, rp2 = 0;  // reduction output, paired index output
};

RunPtrs run_ptrs(Ctx* c, const Run& r) {
  RunPtrs p;
  for (auto& s : r.loads) p.lp.push_back(base_ptr(c, s.base));
  for (auto& s : r.stores) p.sp.push_back(base_ptr(c, s.base));
  if (r.has_red) p.rp = base_ptr(c, r.red_out.base);
  if (r.has_red2) p.rp2 = base_ptr(c, r.red2_out.base);
  return p;
}

// late allocation (section "Vector Engine Manager"): a base gets memory
// when a run first stores into it
void allocate_outputs(Ctx* c, Exec* ex, const Run& r) {
  auto need = [&](int64_t b) {
    BaseRec& br = c->bases[b];
    if (!br.dptr) br.dptr = dev_alloc(c, ex, br.bytes());
    br.written = true;
  };
  for (auto& s : r.stores) need(s.base);
  if (r.has_red) need(r.red_out.base);
  if (r.has_red2) need(r.red2_out.base);
  for (auto& s : r.loads) {
    BaseRec& br = c->bases[s.base];
    if (!br.dptr) fail(VBE_ERR_UNINIT, "a run reads base " + std::to_string(s.base) + " which was never written");
  }
}

// bytes of shared memory one element of a staged run occupies in one stage
int64_t bulk_bytes_per_elem(const Run& r, const Canon& cn) {
  int64_t b = 0;
  for (size_t s = 0; s < r.loads.size(); ++s)
    if (cn.spec.load_cls[s] == 1) b += itemsize(r.loads[s].dtype);
  return b;
}

constexpr int64_t kBulkSmemMax = 200 * 1024;

// a staged launch needs the vector form, at least one unit-stride input,
// room for two stages and 16-byte aligned sources for the bulk copies
bool bulk_ok(const Run& r, const Canon& cn, const RunPtrs& ptr, int64_t CH) {
  if (!cn.spec.vec || CH <= 0 || CH % 16 != 0) return false;
  if (cn.spec.mode != Mode::ELEM && cn.spec.mode != Mode::FULL) return false;
  int64_t bpe = bulk_bytes_per_elem(r, cn);
  if (bpe == 0 || 2 * CH * bpe + 64 > kBulkSmemMax || cn.dims[0] < CH) return false;
  for (size_t s = 0; s < r.loads.size(); ++s) {
    if (cn.spec.load_cls[s] != 1) continue;
    uintptr_t a = ptr.lp[s] + (uintptr_t)(r.loads[s].offset * itemsize(r.loads[s].dtype));
    if (a % 16) return false;
  }
  return true;
}

int64_t tiles_of(const Canon& cn, int block, int U) {
  int64_t bsu = (int64_t)block * U;
  if (cn.spec.vec) {
    int64_t nvec = cn.dims[0] / cn.spec.E;
    return std::max<int64_t>(1, (nvec + bsu - 1) / bsu);
  }
  int64_t inner = cn.dims.back(), outer = 1;
  for (int k = 0; k + 1 < cn.spec.nd; ++k) outer *= cn.dims[k];
  return std::max<int64_t>(1, outer * ((inner + bsu - 1) / bsu));
}

struct Prepared {
  Run* run = nullptr;
  Canon canon;
  std::shared_ptr<const RunSource> rs;  // source, key, kernel name prefix
  std::shared_ptr<Kernel> kern;
};

std::string tune_key(const std::string& key, const Canon& cn) {
  // tuned per signature and per size class (log2 of the element count)
  int lg = 0;
  int64_t n = std::max<int64_t>(1, cn.total);
  while (n > 1) {
    n >>= 1;
    ++lg;
  }
  return key + ":" + std::to_string(lg);
}

Launch build_single(Ctx* c, Exec* ex, Prepared& P, const TuneChoice& tc, const RunPtrs& ptr) {
  Launch L;
  const Run& r = *P.run;
  const Canon& cn = P.canon;
  LaunchArgs a;
  if (tc.bulk_chunk > 0 && bulk_ok(r, cn, ptr, tc.bulk_chunk)) {
    // inputs staged through shared memory: two stages of CH elements per unit-stride input
    const int64_t CH = tc.bulk_chunk;
    L.entry = P.rs->prefix + "_bulk";
    L.key = P.rs->key;
    L.fn = kernel_fn(P.kern.get(), L.entry);
    L.block = tc.block;
    L.smem = (unsigned)(2 * CH * bulk_bytes_per_elem(r, cn) + 64);
    if (!c->record)
      cuda_check(cudaKernelSetAttributeForDevice(L.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem,
                                                 c->device),
                 "dynamic shared memory attribute");
    int64_t chunks = std::max<int64_t>(1, cn.dims[0] / CH);
    int64_t cap = (int64_t)occupancy(L.fn, tc.block, L.smem) * c->sm_count;
    int64_t g = std::min(chunks, cap);
    if (cn.spec.mode == Mode::FULL) g = std::min<int64_t>(g, ex->scratch.n_partials);
    L.grid = (unsigned)std::max<int64_t>(1, g);
    fill_words(r, cn, ptr.lp, ptr.sp, ptr.rp, (uintptr_t)ex->scratch.partials, (uintptr_t)ex->scratch.counters,
               tc.block, 1, &a, CH, (uintptr_t)c->err_word_dev);
  } else if (cn.spec.mode == Mode::ELEM || cn.spec.mode == Mode::FULL) {
    L.entry = P.rs->prefix + "_u" + std::to_string(tc.U) + (tc.maxreg ? "r" + std::to_string(tc.maxreg) : std::string());
    L.key = P.rs->key;
    L.fn = kernel_fn(P.kern.get(), L.entry);
    L.block = tc.block;
    int64_t tiles = tiles_of(cn, tc.block, tc.U);
    int64_t cap = (int64_t)occupancy(L.fn, tc.block) * c->sm_count;
    if (tc.grid_mult > 0) cap = std::min<int64_t>(cap, (int64_t)tc.grid_mult * c->sm_count);
    int64_t g = std::min(tiles, cap);
    if (cn.spec.mode == Mode::FULL) g = std::min<int64_t>(g, ex->scratch.n_partials);
    L.grid = (unsigned)std::max<int64_t>(1, g);
    fill_words(r, cn, ptr.lp, ptr.sp, ptr.rp, (uintptr_t)ex->scratch.partials, (uintptr_t)ex->scratch.counters,
               tc.block, tc.U, &a, 0, (uintptr_t)c->err_word_dev);
  } else {
    L.entry = P.rs->prefix + "_axis";
    L.key = P.rs->key;
    L.fn = kernel_fn(P.kern.get(), L.entry);
    int64_t nout = 1, nred = 1;
    for (int k = 0; k < cn.spec.ndk; ++k) nout *= cn.dims[k];
    for (int k = 0; k < cn.spec.ndr; ++k) nred *= cn.dims[cn.spec.ndk + k];
    if (cn.spec.mode == Mode::AXIS_BLOCK) {
      int b = 32;
      while (b < 256 && b * 8 < nred) b *= 2;
      L.block = b;
      int64_t cap = (int64_t)occupancy(L.fn, b) * c->sm_count;
      L.grid = (unsigned)std::max<int64_t>(1, std::min(nout, cap));
    } else {
      L.block = 128;
      int64_t cap = (int64_t)occupancy(L.fn, 128) * c->sm_count;
      L.grid = (unsigned)std::max<int64_t>(1, std::min((nout + 127) / 128, cap));
    }
    fill_words(r, cn, ptr.lp, ptr.sp, ptr.rp, 0, 0, L.block, 1, &a, 0, 0, ptr.rp2);
  }
  L.words = std::move(a.w);
  return L;
}

// time the launch shapes of a tile kernel with its outputs redirected to
// scratch buffers (so in-place runs are not disturbed) and keep the fastest
TuneChoice autotune(Ctx* c, Exec* ex, Prepared& P, const RunPtrs& real) {
  const Run& r = *P.run;
  RunPtrs ptr = real;
  std::vector<std::pair<void*, int64_t>> bufs;
  auto redirect = [&](const Slot& s, const std::vector<int64_t>& shape_st, int64_t nshape_dims,
                      const std::vector<int64_t>& shape, uintptr_t* p) {
    (void)shape_st;
    (void)nshape_dims;
    int isz = itemsize(s.dtype);
    int64_t lo = s.offset, hi = s.offset;
    for (size_t k = 0; k < s.st.size() && k < shape.size(); ++k) {
      int64_t e = (shape[k] - 1) * s.st[k];
      if (e < 0) lo += e; else hi += e;
    }
    int64_t bytes = (hi - lo + 1) * isz;
    void* b = dev_alloc(c, ex, bytes);
    bufs.push_back({b, bytes});
    *p = (uintptr_t)b - (uintptr_t)(lo * isz);
  };
  for (size_t s = 0; s < r.stores.size(); ++s) redirect(r.stores[s], {}, 0, r.shape, &ptr.sp[s]);
  if (r.has_red) {
    std::vector<int64_t> kshape;
    for (int d = 0; d < (int)r.shape.size(); ++d)
      if (!std::binary_search(r.red_axes.begin(), r.red_axes.end(), d)) kshape.push_back(r.shape[d]);
    redirect(r.red_out, {}, 0, kshape, &ptr.rp);
  }
  TuneChoice best;
  float best_ms = 1e30f;
  if (!ex->ev0) {
    cudaEventCreate(&ex->ev0);
    cudaEventCreate(&ex->ev1);
  }
  std::vector<TuneChoice> cands;
  for (int block : {128, 256, 512})
    for (int U : {1, 2, 4}) {
      TuneChoice tc;
      tc.block = block;
      tc.U = U;
      cands.push_back(tc);
    }
  if (reg_cap_variants(r))
    for (int block : {256, 512})
      for (int U : {1, 2})
        for (int cap : kRegCaps) {
          TuneChoice tc;
          tc.block = block;
          tc.U = U;
          tc.maxreg = cap;
          cands.push_back(tc);
        }
  for (int block : {256, 512})
    for (int ch : {1024, 2048, 4096}) {
      TuneChoice tc;
      tc.block = block;
      tc.bulk_chunk = ch;
      if (bulk_ok(r, P.canon, real, ch)) cands.push_back(tc);
    }
  for (const TuneChoice& tc : cands) {
    {
      Launch L = build_single(c, ex, P, tc, ptr);
      issue(c, ex, L, false);  // warm
      c->stats.kernel_launches--;
      cuda_check(cudaEventRecord(ex->ev0, ex->stream), "event");
      for (int rep = 0; rep < 3; ++rep) {
        issue(c, ex, L, false);
        c->stats.kernel_launches--;
      }
      cuda_check(cudaEventRecord(ex->ev1, ex->stream), "event");
      cuda_check(cudaEventSynchronize(ex->ev1), "event sync");
      float ms = 0;
      cudaEventElapsedTime(&ms, ex->ev0, ex->ev1);
      if (ms < best_ms) {
        best_ms = ms;
        best = tc;
      }
    }
  }
  for (auto& b : bufs) dev_free(c, ex, b.first, b.second);
  c->stats.autotunes++;
  return best;
}

TuneChoice choose(Ctx* c, Exec* ex, Prepared& P, const RunPtrs& ptr, bool may_tune) {
  bool tile = P.canon.spec.mode == Mode::ELEM || P.canon.spec.mode == Mode::FULL;
  if (c->record) {
    TuneChoice tc;
    tc.block = c->rec_block;
    tc.U = c->rec_U;
    tc.bulk_chunk = c->force_bulk;
    return tc;
  }
  if (c->force_bulk > 0 && bulk_ok(*P.run, P.canon, ptr, c->force_bulk)) {
    TuneChoice tc;
    tc.block = 512;
    tc.bulk_chunk = c->force_bulk;
    return tc;
  }
  std::string tk = tune_key(P.rs->key, P.canon);
  TuneChoice known;
  if (recall_tune(c, tk, &known)) return known;
  TuneChoice tc;
  tc.block = 256;
  tc.U = P.canon.total >= (1 << 16) ? 2 : 1;
  if (c->record) {
    tc.block = c->rec_block;
    tc.U = c->rec_U;
    return tc;
  }
  if (tile && may_tune && (c->cfg.flags & VBE_AUTOTUNE) && P.canon.total >= (1 << 20)) {
    tc = autotune(c, ex, P, ptr);
    remember_tune(c, tk, tc);
  }
  return tc;
}

bool independent(const Run& a, const Run& b, Ctx* c) {
  auto view_of = [&](const Slot& s, const std::vector<int64_t>& shape) {
    ViewDesc v;
    v.base = s.base;
    v.offset = s.offset;
    v.ndim = (int)shape.size();
    for (int k = 0; k < v.ndim; ++k) {
      v.shape[k] = shape[k];
      v.strides[k] = s.st[k];
    }
    v.finish();
    return v;
  };
  (void)c;
  std::vector<ViewDesc> ra, wa, rb, wb;
  for (auto& s : a.loads) ra.push_back(view_of(s, a.shape));
  for (auto& s : a.stores) wa.push_back(view_of(s, a.shape));
  for (auto& s : b.loads) rb.push_back(view_of(s, b.shape));
  for (auto& s : b.stores) wb.push_back(view_of(s, b.shape));
  auto kept = [](const Run& r) {
    std::vector<int64_t> k;
    for (int d = 0; d < (int)r.shape.size(); ++d)
      if (!std::binary_search(r.red_axes.begin(), r.red_axes.end(), d)) k.push_back(r.shape[d]);
    return k;
  };
  if (a.has_red) wa.push_back(view_of(a.red_out, kept(a)));
  if (b.has_red) wb.push_back(view_of(b.red_out, kept(b)));
  if (a.has_red2) wa.push_back(view_of(a.red2_out, kept(a)));
  if (b.has_red2) wb.push_back(view_of(b.red2_out, kept(b)));
  for (auto& x : wb) {
    for (auto& y : ra) if (may_overlap(x, y)) return false;
    for (auto& y : wa) if (may_overlap(x, y)) return false;
  }
  for (auto& x : rb)
    for (auto& y : wa) if (may_overlap(x, y)) return false;
  return true;
}

// ------------------------------------------------------ tile-fused groups

struct GroupPrepared {
  Group* g = nullptr;
  std::shared_ptr<const GroupSource> gs;  // source, entry prefix, key, tile shapes
  std::shared_ptr<Kernel> kern;
};

struct GroupPtrs {
  std::vector<std::vector<uintptr_t>> lp, sp;
  std::vector<std::pair<uintptr_t, uintptr_t>> ren;  // (current buffer, second buffer)
  std::vector<uintptr_t> red;                        // per run: reduction output (0: none)
};

// memory the group reads must exist; the anchor's targets are allocated,
// renamed bases get their second buffer
void allocate_group(Ctx* c, Exec* ex, const Group& g) {
  const int anchor = (int)g.runs.size() - 1;
  for (size_t k = 0; k < g.runs.size(); ++k)
    for (size_t s = 0; s < g.runs[k].loads.size(); ++s) {
      if (g.lds[k][s].prod >= 0) continue;
      BaseRec& br = c->bases[g.runs[k].loads[s].base];
      if (!br.dptr)
        fail(VBE_ERR_UNINIT, "a run reads base " + std::to_string(g.runs[k].loads[s].base) + " which was never written");
    }
  for (auto& st : g.runs[anchor].stores) {
    BaseRec& br = c->bases[st.base];
    if (!br.dptr) br.dptr = dev_alloc(c, ex, br.bytes());
    br.written = true;
  }
  for (int64_t b : g.renamed) {
    BaseRec& br = c->bases[b];
    if (!br.shadow) br.shadow = dev_alloc(c, ex, br.bytes());
  }
  for (auto& r : g.runs) {
    if (!r.has_red) continue;
    BaseRec& br = c->bases[r.red_out.base];
    if (!br.dptr) br.dptr = dev_alloc(c, ex, br.bytes());
    br.written = true;
  }
}

GroupPtrs group_ptrs(Ctx* c, const Group& g) {
  GroupPtrs p;
  const int m = (int)g.runs.size(), anchor = m - 1;
  p.lp.resize(m);
  p.sp.resize(m);
  for (int k = 0; k < m; ++k) {
    for (size_t s = 0; s < g.runs[k].loads.size(); ++s)
      p.lp[k].push_back(g.lds[k][s].prod >= 0 ? 0 : base_ptr(c, g.runs[k].loads[s].base));
    for (size_t s = 0; s < g.runs[k].stores.size(); ++s) {
      uintptr_t a = 0;
      if (k == anchor) {
        int64_t b = g.runs[k].stores[s].base;
        a = base_ptr(c, b);
        for (size_t r = 0; r < g.renamed.size(); ++r)
          if (g.renamed[r] == b) a = (uintptr_t)c->bases[b].shadow;
      }
      p.sp[k].push_back(a);
    }
  }
  for (int64_t b : g.renamed) p.ren.push_back({base_ptr(c, b), (uintptr_t)c->bases[b].shadow});
  for (auto& r : g.runs) p.red.push_back(r.has_red ? base_ptr(c, r.red_out.base) : 0);
  return p;
}

// cuTensorMapEncodeTiled, taken from the driver at run time (no link-time
// dependency on the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return (EncodeTiledFn)p;
  }();
  return fn;
}

// The tensor maps of a tensor-copy group launch: 16 words each. A recording
// context writes its own description instead (address, row stride, rows,
// row bytes, box), which the host emulation of the copy reads.
std::vector<int64_t> group_tensor_maps(Ctx* c, const Group& g, const TileShape& ts, const GroupPtrs& ptr) {
  std::vector<int64_t> w;
  for (const TmaBox& b : group_tma_boxes(g, ts)) {
    const uintptr_t base = ptr.lp[b.ref_k][b.ref_s];
    int64_t m[16] = {0};
    if (c->record) {
      m[0] = (int64_t)base;
      m[1] = b.pitch;
      m[2] = b.rows;
      m[3] = b.pitch * b.isz;
      m[4] = b.box_cols;
      m[5] = b.box_rows;
      m[6] = b.isz;
    } else {
      EncodeTiledFn enc = encode_tiled();
      if (!enc) fail(VBE_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
      const CUtensorMapDataType dt = b.isz == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                     : (b.isz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64);
      const cuuint64_t dims[2] = {(cuuint64_t)b.pitch, (cuuint64_t)b.rows};
      const cuuint64_t strides[1] = {(cuuint64_t)(b.pitch * b.isz)};
      const cuuint32_t box[2] = {(cuuint32_t)b.box_cols, (cuuint32_t)b.box_rows};
      const cuuint32_t estr[2] = {1, 1};
      CUresult r = enc((CUtensorMap*)m, dt, 2, (void*)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) fail(VBE_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    }
    w.insert(w.end(), m, m + 16);
  }
  return w;
}

// tensor copies read whole 16-byte units from 16-byte aligned bases
bool tma_pointers_ok(const Group& g, const TileShape& ts, const GroupPtrs& ptr) {
  for (const TmaBox& b : group_tma_boxes(g, ts))
    if (ptr.lp[b.ref_k][b.ref_s] % 16 != 0) return false;
  return true;
}

Launch build_group(Ctx* c, Exec* ex, GroupPrepared& G, const TileShape& ts, const GroupPtrs& ptr) {
  Launch L;
  L.entry = G.gs->prefix + ts.suffix();
  L.key = G.gs->key;
  L.fn = kernel_fn(G.kern.get(), L.entry);
  L.block = (unsigned)(ts.block + (ts.tma ? 32 : 0));  // the tensor-copy form adds a producer warp
  L.smem = (unsigned)ts.smem;
  if (!c->record)
    cuda_check(cudaKernelSetAttributeForDevice(L.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem,
                                               c->device),
               "dynamic shared memory attribute");
  LaunchArgs a;
  int nred = 0;
  for (auto& r : G.g->runs) nred += r.has_red ? 1 : 0;
  const Run& ra = G.g->runs.back();
  const int64_t ntiles = ((ra.shape[0] + ts.th - 1) / ts.th) * ((ra.shape[1] + ts.tw - 1) / ts.tw);
  if (nred * ntiles > ex->scratch.n_partials) fail(VBE_ERR_INVALID, "tile-fused group needs more reduction partials");
  fill_group_words(*G.g, ts, ptr.lp, ptr.sp, ptr.ren, ptr.red, (uintptr_t)ex->scratch.partials,
                   (uintptr_t)ex->scratch.counters, &a, (uintptr_t)c->err_word_dev);
  L.grid = (unsigned)std::max<int64_t>(1, a.w[3]);
  if (ts.sweep) {  // one warp per strip
    const int64_t nw = ts.block / 32;
    L.grid = (unsigned)std::max<int64_t>(1, (a.w[3] + nw - 1) / nw);
    L.sweep = true;
  }
  if (ts.tma) {
    // persistent: as many blocks as fit, tensor maps ahead of the words
    const int64_t cap = (int64_t)occupancy(L.fn, (int)L.block, L.smem) * c->sm_count;
    L.grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(a.w[3], cap));
    std::vector<int64_t> w = group_tensor_maps(c, *G.g, ts, ptr);
    w.insert(w.end(), a.w.begin(), a.w.end());
    while (w.size() % 8) w.push_back(0);  // the parameter block is 64-byte aligned
    L.words = std::move(w);
    L.tma = true;
    return L;
  }
  L.words = std::move(a.w);
  return L;
}

std::string group_tune_key(const GroupPrepared& G) {
  const Group& g = *G.g;
  int64_t n = std::max<int64_t>(1, g.rows((int)g.runs.size() - 1) * g.cols((int)g.runs.size() - 1));
  int lg = 0;
  while (n > 1) {
    n >>= 1;
    ++lg;
  }
  return G.gs->key + ":" + std::to_string(lg);
}

// the tile shape: fixed in record mode (VBE_RECORD_TILE=THxTW), else timed
// per signature and size class with the anchor's in-place targets
// redirected to scratch buffers
TileShape choose_group(Ctx* c, Exec* ex, GroupPrepared& G, const GroupPtrs& real, bool may_tune) {
  const std::vector<TileShape>& shapes = G.gs->shapes;
  if (shapes.empty()) fail(VBE_ERR_INVALID, "tile-fused group without a tile shape");
  // a fixed shape: "THxTW", "sTHxTW" for the staged form, "tTHxTW" for the
  // tensor-copy form, "rR" for the row-sweep form with strips of R rows
  // (VBE_RECORD_TILE when recording, else VBE_TILE)
  const char* e = c->record ? getenv("VBE_RECORD_TILE") : (c->force_tile.empty() ? nullptr : c->force_tile.c_str());
  if (e)
    for (auto& ts : shapes) {
      const std::string name = ts.letter() + std::to_string(ts.th) + (ts.sweep ? "" : "x" + std::to_string(ts.tw));
      if (name == e && (c->record || !ts.tma || tma_pointers_ok(*G.g, ts, real))) return ts;
    }
  if (c->record) return shapes[0];
  std::string tk = group_tune_key(G);
  TuneChoice known;
  if (recall_tune(c, tk, &known))
    for (auto& ts : shapes)
      if (ts.th == known.block && ts.tw == known.U && ts.form() == known.grid_mult &&
          (!ts.tma || tma_pointers_ok(*G.g, ts, real)))
        return ts;
  TileShape def = shapes[0];
  for (auto& ts : shapes)
    if (!ts.staged && !ts.tma && !ts.sweep && ts.th * ts.tw <= 1024 && ts.th * ts.tw >= def.th * def.tw) def = ts;
  const Group& g = *G.g;
  const int anchor = (int)g.runs.size() - 1;
  if (!(may_tune && (c->cfg.flags & VBE_AUTOTUNE) && g.rows(anchor) * g.cols(anchor) >= (1 << 16))) return def;
  GroupPtrs ptr = real;
  std::vector<std::pair<void*, int64_t>> bufs;
  const Run& ra = g.runs[anchor];
  for (size_t s = 0; s < ra.stores.size(); ++s) {
    bool renamed = false;
    for (int64_t b : g.renamed)
      if (b == ra.stores[s].base) renamed = true;
    if (renamed) continue;  // writes the second buffer only
    const Slot& st = ra.stores[s];
    int64_t lo = st.offset, hi = st.offset;
    for (int k = 0; k < 2; ++k) {
      int64_t e = (ra.shape[k] - 1) * st.st[k];
      if (e < 0) lo += e; else hi += e;
    }
    int64_t bytes = (hi - lo + 1) * itemsize(st.dtype);
    void* b = dev_alloc(c, ex, bytes);
    bufs.push_back({b, bytes});
    ptr.sp[anchor][s] = (uintptr_t)b - (uintptr_t)(lo * itemsize(st.dtype));
  }
  if (!ex->ev0) {
    cudaEventCreate(&ex->ev0);
    cudaEventCreate(&ex->ev1);
  }
  TileShape best = def;
  float best_ms = 1e30f;
  for (const TileShape& ts : shapes) {
    if (ts.tma && !tma_pointers_ok(g, ts, ptr)) continue;
    Launch L = build_group(c, ex, G, ts, ptr);
    issue(c, ex, L, false);  // warm
    c->stats.kernel_launches--;
    cuda_check(cudaEventRecord(ex->ev0, ex->stream), "event");
    for (int rep = 0; rep < 3; ++rep) {
      issue(c, ex, L, false);
      c->stats.kernel_launches--;
    }
    cuda_check(cudaEventRecord(ex->ev1, ex->stream), "event");
    cuda_check(cudaEventSynchronize(ex->ev1), "event sync");
    float ms = 0;
    cudaEventElapsedTime(&ms, ex->ev0, ex->ev1);
    if (ms < best_ms) {
      best_ms = ms;
      best = ts;
    }
  }
  for (auto& b : bufs) dev_free(c, ex, b.first, b.second);
  c->stats.autotunes++;
  TuneChoice tc;  // the group's choice: tile rows, tile columns, form
  tc.block = best.th;
  tc.U = best.tw;
  tc.grid_mult = best.form();
  remember_tune(c, tk, tc);
  return best;
}

// Whether the group runs faster as its separate kernels (temporaries through
// memory, no halo recomputation). Timed once per signature and size class
// with VBE_AUTOTUNE: the group kernel writes only second buffers and
// scratch; the separate kernels write the group's temporaries (dead after
// it) and scratch in place of the anchor's targets, so nothing live changes.
bool group_split(Ctx* c, Exec* ex, GroupPrepared& G, const TileShape& ts, const GroupPtrs& real, bool may_tune) {
  if (c->record) return getenv("VBE_RECORD_SPLIT") != nullptr;
  if (!c->force_tile.empty()) return false;  // a fixed tile shape runs the group kernel
  const std::string sk = group_tune_key(G) + ":split";
  TuneChoice known;
  if (recall_tune(c, sk, &known)) return known.block == 1;
  Group& g = *G.g;
  const int anchor = (int)g.runs.size() - 1;
  if (!(may_tune && (c->cfg.flags & VBE_AUTOTUNE) && g.rows(anchor) * g.cols(anchor) >= (1 << 16))) return false;
  std::vector<std::pair<void*, int64_t>> bufs;
  auto scratch_for = [&](const Slot& st, const std::vector<int64_t>& shape) {
    int64_t lo = st.offset, hi = st.offset;
    for (int k = 0; k < 2; ++k) {
      int64_t e = (shape[k] - 1) * st.st[k];
      if (e < 0) lo += e; else hi += e;
    }
    int64_t bytes = (hi - lo + 1) * itemsize(st.dtype);
    void* b = dev_alloc(c, ex, bytes);
    bufs.push_back({b, bytes});
    return (uintptr_t)b - (uintptr_t)(lo * itemsize(st.dtype));
  };
  // the group kernel, non-renamed anchor targets redirected
  GroupPtrs gp = real;
  const Run& ra = g.runs[anchor];
  for (size_t s = 0; s < ra.stores.size(); ++s) {
    bool renamed = false;
    for (int64_t b : g.renamed)
      if (b == ra.stores[s].base) renamed = true;
    if (!renamed) gp.sp[anchor][s] = scratch_for(ra.stores[s], ra.shape);
  }
  std::vector<Launch> grp{build_group(c, ex, G, ts, gp)};
  // the separate kernels
  std::vector<Launch> sep;
  std::vector<Prepared> preps(g.runs.size());
  for (int k = 0; k <= anchor; ++k) {
    Run& r = g.runs[k];
    if (k < anchor) allocate_outputs(c, ex, r);
    Prepared& P = preps[k];
    P.run = &r;
    RunPtrs rp = run_ptrs(c, r);
    if (k == anchor)
      for (size_t s = 0; s < r.stores.size(); ++s) rp.sp[s] = scratch_for(r.stores[s], r.shape);
    P.canon = canonicalize(r, true, rp.lp, rp.sp, rp.rp);
    P.rs = run_source(r, P.canon);
    P.kern = get_kernel(c, P.rs->src, &P.rs->key);
    TuneChoice tc = choose(c, ex, P, rp, true);
    sep.push_back(build_single(c, ex, P, tc, rp));
  }
  if (!ex->ev0) {
    cudaEventCreate(&ex->ev0);
    cudaEventCreate(&ex->ev1);
  }
  auto time_of = [&](std::vector<Launch>& Ls) {
    for (auto& L : Ls) {
      issue(c, ex, L, false);
      c->stats.kernel_launches--;
    }
    cuda_check(cudaEventRecord(ex->ev0, ex->stream), "event");
    for (int rep = 0; rep < 3; ++rep)
      for (auto& L : Ls) {
        issue(c, ex, L, false);
        c->stats.kernel_launches--;
      }
    cuda_check(cudaEventRecord(ex->ev1, ex->stream), "event");
    cuda_check(cudaEventSynchronize(ex->ev1), "event sync");
    float ms = 0;
    cudaEventElapsedTime(&ms, ex->ev0, ex->ev1);
    return ms;
  };
  const float t_group = time_of(grp), t_sep = time_of(sep);
  for (auto& b : bufs) dev_free(c, ex, b.first, b.second);
  TuneChoice tc;
  tc.block = t_sep < t_group ? 1 : 0;
  remember_tune(c, sk, tc);
  return tc.block == 1;
}

uint64_t batch_key(const vbe_instr* prog, int64_t n) {
  return hash64(prog, (size_t)n * sizeof(vbe_instr), (uint64_t)n);
}

std::vector<std::pair<int64_t, uintptr_t>> fingerprint(Ctx* c, const std::vector<RInstr>& rp) {
  std::vector<int64_t> ids;
  for (auto& r : rp) {
    ids.push_back(r.out.base);
    for (int k = 0; k < r.nin; ++k)
      if (k != r.const_slot) ids.push_back(r.in[k].base);
  }
  std::sort(ids.begin(), ids.end());
  ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
  std::vector<std::pair<int64_t, uintptr_t>> f;
  for (auto b : ids) {
    auto it = c->bases.find(b);
    f.push_back({b, it == c->bases.end() ? 0 : (uintptr_t)it->second.dptr});
    if (it != c->bases.end() && it->second.shadow) f.push_back({-b, (uintptr_t)it->second.shadow});
  }
  return f;
}

}  // namespace

void add_view(Ctx* c, int64_t handle, const ViewDesc& v) {
  c->views[handle] = v;
  auto it = c->bases.find(v.base);
  if (it != c->bases.end()) it->second.views.push_back(handle);
}

void erase_views_of(Ctx* c, BaseRec& br) {
  for (int64_t h : br.views) c->views.erase(h);
  br.views.clear();
}

namespace {

void do_action(Ctx* c, Exec* ex, const HostAction& a) {
  auto it = c->bases.find(a.base);
  if (it == c->bases.end()) return;
  if (a.kind == 2 && it->second.mirror) {
    // a SYNC of a base with a host mirror copies the device copy back to
    // the mirror at this point of the batch (rule 3 of the ownership
    // scheme), unless the device copy holds no current value there
    auto q = c->mirror_syncs.find(a.base);
    bool copy = q != c->mirror_syncs.end() && !q->second.empty() && q->second.front();
    if (q != c->mirror_syncs.end() && !q->second.empty()) q->second.pop_front();
    if (copy && it->second.dptr && it->second.bytes() > 0)
      stream_copy(c, ex, it->second.mirror, it->second.dptr, it->second.bytes(), true);
    return;
  }
  if (a.kind == 0) {  // FREE
    if (it->second.dptr && !it->second.external) dev_free(c, ex, it->second.dptr, it->second.bytes());
    if (it->second.shadow) dev_free(c, ex, it->second.shadow, it->second.bytes());
    erase_views_of(c, it->second);
    c->bases.erase(it);
    c->epoch++;
  }
}

}  // namespace

// Batches of fewer launches replay their launch list even with VBE_GRAPHS:
// with programmatic dependent launch one or two stream launches cost less
// than a graph launch (measured: a one-kernel Jacobi iteration 6.5 us
// replayed from its list, 8.3 us from a graph).
constexpr size_t kGraphMinLaunches = 3;

// Execute one batch on ex's stream. Eager the first time a batch is seen;
// with VBE_GRAPHS, a batch seen again (same instructions, same views, same
// base addresses, no FREE) is captured into a CUDA graph and later replayed.
// A batch whose tile-fused groups rename bases alternates between two
// address sets; each has its own cached launches.
void exec_batch(Ctx* c, Exec* ex, const vbe_instr* prog, int64_t n, bool allow_graph) {
  if (c->host_only && !c->record) fail(VBE_ERR_NO_DEVICE, "host-only context");
  c->stats.batches++;
  // a batch without FREE that comes again unchanged (same instructions,
  // views and base addresses) skips validation, analysis and code
  // generation: its launches are replayed from a graph (VBE_GRAPHS) or one
  // by one. Never for one-shot server requests.
  const bool may_cache = allow_graph && !c->record;
  uint64_t key = may_cache ? (batch_key(prog, n) ^ (uint64_t)(uintptr_t)ex) : 0;
  CachedBatch* known = nullptr;
  if (may_cache) {
    auto kb = c->batches.find(key);
    if (kb != c->batches.end() && kb->second.rp_epoch == c->epoch) known = &kb->second;
  }
  std::vector<RInstr> rp_local;
  if (!known) rp_local = resolve_batch(c, prog, n);
  const std::vector<RInstr>& rp = known ? known->rp : rp_local;
  // a batch with FREE, or with a SYNC or DISCARD of a base that has a host
  // mirror (they act on the host copy), is executed afresh every time
  bool one_shot = false;
  for (auto& r : rp) {
    if (r.op == VBE_OP_FREE) one_shot = true;
    if ((r.op == VBE_OP_SYNC || r.op == VBE_OP_DISCARD) && c->bases.count(r.out.base) &&
        c->bases[r.out.base].mirror)
      one_shot = true;
  }
  bool graphs = allow_graph && (c->cfg.flags & VBE_GRAPHS) && !one_shot && !c->record;
  bool cacheable = may_cache && !one_shot;
  static uint64_t use_clock = 0;
  CachedBatch* cb = nullptr;
  CachedVariant* var = nullptr;
  auto apply_after = [&](const CachedVariant& v) {
    for (auto& a : v.after) {
      BaseRec& br = c->bases[a.first];
      br.dptr = a.second.first;
      br.shadow = a.second.second;
    }
  };
  if (cacheable) {
    cb = &c->batches[key];
    cb->key = key;
    if (!known) {
      cb->rp = rp_local;
      cb->rp_epoch = c->epoch;
    }
    auto fp = fingerprint(c, rp);
    for (auto& v : cb->v)
      if (v.fingerprint == fp) var = &v;
    if (var) {
      var->last_use = ++use_clock;
      if (graphs && var->exec) {
        cuda_check(cudaGraphLaunch(var->exec, ex->stream), "cudaGraphLaunch");
        c->stats.graph_launches++;
        c->stats.kernel_launches += var->launches;
        c->stats.packed_launches += var->packed_launches;
        apply_after(*var);
        return;
      }
      if ((!graphs || (var->has_eager && var->eager.size() < kGraphMinLaunches)) && var->has_eager) {
        for (auto& L : var->eager) issue(c, ex, *L, false);
        c->stats.list_replays++;
        apply_after(*var);
        return;
      }
    }
  }
  bool fuse = (c->cfg.flags & VBE_FUSE) != 0;
  bool pack = (c->cfg.flags & VBE_PACK) != 0;
  std::vector<RInstr> staged = rp;
  Plan plan = make_plan(c, staged, fuse, pack);
  {
    // reduction partials of tile-fused groups: one per tile of the smallest
    // tile shape (8 x 16) per reducing run, reserved before anything is issued
    int64_t need = 1 << 20;
    for (auto& it : plan.items) {
      if (it.kind != 2) continue;
      int64_t nred = 0;
      for (auto& r : it.group->runs) nred += r.has_red ? 1 : 0;
      const Run& ra = it.group->runs.back();
      need = std::max<int64_t>(need, nred * ((ra.shape[0] + 7) / 8) * ((ra.shape[1] + 15) / 16));
    }
    ensure_scratch(c, ex, need, 1 << 16);
  }
  bool capture = graphs && var && var->seen >= 1 && !(var->has_eager && var->eager.size() < kGraphMinLaunches);

  // compile the batch's kernels in parallel on first sight
  {
    std::vector<std::string> srcs, keys;
    for (auto& it : plan.items) {
      if (it.kind == 2) {
        auto gs = group_source(*it.group);
        if (c->cwait < 0 && c->kernels.count(gs->key)) continue;  // loaded already
        keys.push_back(gs->key);
        srcs.push_back(gs->src);
        continue;
      }
      if (it.kind != 0) continue;
      RunPtrs pp;
      for (auto& s : it.run.loads) pp.lp.push_back((uintptr_t)c->bases[s.base].dptr);
      for (auto& s : it.run.stores) pp.sp.push_back((uintptr_t)c->bases[s.base].dptr);
      Canon cn = canonicalize(it.run, true, pp.lp, pp.sp, 0);
      auto rs = run_source(it.run, cn);
      if (c->cwait < 0 && c->kernels.count(rs->key)) continue;  // loaded already
      keys.push_back(rs->key);
      srcs.push_back(rs->src);
    }
    if (!c->record) precompile(c, srcs, &keys);
  }
  // first pass: allocation order and reads of never-written bases (a base
  // is available when it has memory or an earlier item of the batch writes
  // it; only the bases the batch touches are looked at, so the cost does not
  // grow with the bases other requests keep in the context)
  {
    struct Avail {
      Ctx* c;
      std::unordered_set<int64_t> written;
      size_t count(int64_t b) const {
        if (written.count(b)) return 1;
        auto it = c->bases.find(b);
        return it != c->bases.end() && it->second.dptr ? 1 : 0;
      }
      void insert(int64_t b) { written.insert(b); }
    } avail{c, {}};
    for (auto& it : plan.items) {
      if (it.kind == 2) {
        const Group& g = *it.group;
        for (size_t k = 0; k < g.runs.size(); ++k)
          for (size_t s = 0; s < g.runs[k].loads.size(); ++s)
            if (g.lds[k][s].prod < 0 && !avail.count(g.runs[k].loads[s].base))
              fail(VBE_ERR_UNINIT, "the batch reads base " + std::to_string(g.runs[k].loads[s].base) +
                                       " before anything wrote it");
        for (auto& s : g.runs.back().stores) avail.insert(s.base);
        continue;
      }
      if (it.kind != 0) continue;
      for (auto& s : it.run.loads)
        if (!avail.count(s.base))
          fail(VBE_ERR_UNINIT, "the batch reads base " + std::to_string(s.base) + " before anything wrote it");
      for (auto& s : it.run.stores) avail.insert(s.base);
      if (it.run.has_red) avail.insert(it.run.red_out.base);
      if (it.run.has_red2) avail.insert(it.run.red2_out.base);
    }
  }
  // capture needs every store target (and second buffer) allocated already
  if (capture) {
    for (auto& it : plan.items) {
      if (it.kind == 2) {
        for (auto& s : it.group->runs.back().stores)
          if (!c->bases[s.base].dptr) capture = false;
        for (int64_t b : it.group->renamed)
          if (!c->bases[b].shadow) capture = false;
        continue;
      }
      if (it.kind != 0) continue;
      for (auto& s : it.run.stores)
        if (!c->bases[s.base].dptr) capture = false;
      if (it.run.has_red && !c->bases[it.run.red_out.base].dptr) capture = false;
      if (it.run.has_red2 && !c->bases[it.run.red2_out.base].dptr) capture = false;
    }
  }

  std::vector<Launch> recorded;
  std::vector<std::shared_ptr<Launch>> issued;
  std::vector<HostAction> deferred;
  std::map<int64_t, int> swaps;  // renamed bases: times swapped in this batch
  auto flush_deferred = [&]() {
    for (auto& a : deferred) do_action(c, ex, a);
    deferred.clear();
  };
  size_t i = 0;
  while (i < plan.items.size()) {
    PlanItem& it = plan.items[i];
    if (it.kind == 1) {
      if (capture) {
        ++i;
        continue;  // capture never has FREE; DISCARD/SYNC are no-ops on the device
      }
      deferred.push_back(it.act);
      ++i;
      if (it.act.kind == 2) flush_deferred();
      continue;
    }
    if (it.kind == 2) {
      Group& g = *it.group;
      allocate_group(c, ex, g);
      GroupPrepared G;
      G.g = &g;
      G.gs = group_source(g);
      G.kern = get_kernel(c, G.gs->src, &G.gs->key);
      GroupPtrs ptr = group_ptrs(c, g);
      TileShape ts = choose_group(c, ex, G, ptr, !capture);
      if (group_split(c, ex, G, ts, ptr, !capture)) {
        // measured faster as separate kernels (e.g. when the halo
        // recomputation costs more arithmetic than the temporaries' traffic)
        for (Run& r : g.runs) {
          if (!r.has_red && r.elements() == 0) continue;
          allocate_outputs(c, ex, r);
          Prepared P;
          P.run = &r;
          RunPtrs rp = run_ptrs(c, r);
          P.canon = canonicalize(r, true, rp.lp, rp.sp, rp.rp);
          P.rs = run_source(r, P.canon);
          P.kern = get_kernel(c, P.rs->src, &P.rs->key);
          TuneChoice tc = choose(c, ex, P, rp, !capture);
          Launch L = build_single(c, ex, P, tc, rp);
          if (capture) {
            recorded.push_back(std::move(L));
          } else {
            issue(c, ex, L, false);
            if (cacheable) issued.push_back(std::make_shared<Launch>(L));
          }
        }
        ++i;
        if (!capture) flush_deferred();
        continue;
      }
      Launch L = build_group(c, ex, G, ts, ptr);
      if (capture) {
        recorded.push_back(std::move(L));
      } else {
        issue(c, ex, L, false);
        if (cacheable) issued.push_back(std::make_shared<Launch>(L));
      }
      for (int64_t b : g.renamed) {
        BaseRec& br = c->bases[b];
        std::swap(br.dptr, br.shadow);
        swaps[b]++;
      }
      ++i;
      if (!capture) flush_deferred();
      continue;
    }
    Run& r = it.run;
    if (!r.has_red && r.elements() == 0) {
      ++i;
      continue;
    }
    allocate_outputs(c, ex, r);
    Prepared P;
    P.run = &r;
    RunPtrs ptr = run_ptrs(c, r);
    P.canon = canonicalize(r, true, ptr.lp, ptr.sp, ptr.rp);
    P.rs = run_source(r, P.canon);
    P.kern = get_kernel(c, P.rs->src, &P.rs->key);
    bool tile = P.canon.spec.mode == Mode::ELEM || P.canon.spec.mode == Mode::FULL;
    // packing: following runs with the same kernel that share no data
    std::vector<size_t> group{i};
    size_t j = i + 1;
    if (pack && tile && P.canon.spec.nd == 1) {
      std::vector<size_t> skipped;
      while (j < plan.items.size()) {
        PlanItem& nx = plan.items[j];
        if (nx.kind == 2) break;
        if (nx.kind == 1) {
          if (nx.act.kind == 2) break;  // SYNC
          ++j;
          continue;
        }
        Run& r2 = nx.run;
        if (r2.shape.size() != r.shape.size() && !(r2.shape.size() <= 1 && r.shape.size() <= 1)) break;
        bool ok = true;
        for (size_t g : group)
          if (!independent(plan.items[g].run, r2, c)) ok = false;
        if (!ok) break;
        allocate_outputs(c, ex, r2);
        RunPtrs p2 = run_ptrs(c, r2);
        Canon c2 = canonicalize(r2, true, p2.lp, p2.sp, p2.rp);
        if (c2.spec.nd != 1 || run_source(r2, c2) != P.rs) break;
        group.push_back(j);
        ++j;
      }
      if (group.size() == 1) j = i + 1;
    }
    if (group.size() > 1 && (int64_t)group.size() < ex->scratch.n_counters - 1) {
      // one persistent launch over all instances
      Launch L;
      L.packed = true;
      int U = 4;
      L.entry = P.rs->prefix + "_pack_u" + std::to_string(U);
      L.key = P.rs->key;
      L.fn = kernel_fn(P.kern.get(), L.entry);
      L.block = 256;
      int64_t total_elems = 0;
      for (size_t g : group) total_elems += plan.items[g].run.elements();
      int64_t chunk = std::max<int64_t>(L.block * U * 4, (total_elems / (ex->scratch.n_partials / 2)) + 1);
      chunk = ((chunk + 1023) / 1024) * 1024;
      L.chunk = chunk;
      L.ninst = (int)group.size();
      int64_t poff = 0;
      L.prefix.push_back(0);
      for (size_t gi = 0; gi < group.size(); ++gi) {
        Run& rg = plan.items[group[gi]].run;
        RunPtrs pg = run_ptrs(c, rg);
        Canon cg = canonicalize(rg, true, pg.lp, pg.sp, pg.rp);
        int64_t ne = rg.elements();
        int64_t nch = ne > 0 ? (ne + chunk - 1) / chunk : 1;
        LaunchArgs a;
        fill_words(rg, cg, pg.lp, pg.sp, pg.rp,
                   (uintptr_t)((char*)ex->scratch.partials + poff * 8),
                   (uintptr_t)(ex->scratch.counters + gi), L.block, U, &a);
        L.descs.insert(L.descs.end(), a.w.begin(), a.w.end());
        poff += nch;
        L.prefix.push_back(L.prefix.back() + nch);
      }
      L.total = L.prefix.back();
      if (poff > ex->scratch.n_partials) fail(VBE_ERR_INVALID, "packed launch needs too many partials");
      L.grid = (unsigned)std::min<int64_t>(L.total, (int64_t)occupancy(L.fn, L.block) * c->sm_count);
      if (capture) {
        recorded.push_back(std::move(L));
      } else {
        issue(c, ex, L, false);
        if (cacheable) issued.push_back(std::make_shared<Launch>(L));
      }
      // host actions skipped over while packing run after the pack
      for (size_t k = i + 1; k < j; ++k)
        if (plan.items[k].kind == 1) deferred.push_back(plan.items[k].act);
      i = j;
      if (!capture) flush_deferred();
      continue;
    }
    TuneChoice tc = choose(c, ex, P, ptr, !capture);
    Launch L = build_single(c, ex, P, tc, ptr);
    if (capture) {
      recorded.push_back(std::move(L));
    } else {
      issue(c, ex, L, false);
      if (cacheable) issued.push_back(std::make_shared<Launch>(L));
    }
    ++i;
    if (!capture) flush_deferred();
  }
  if (!capture) flush_deferred();

  // the address set these launches are valid for: the end state with this
  // batch's renames undone
  std::vector<std::pair<int64_t, std::pair<void*, void*>>> after;
  std::vector<std::pair<int64_t, uintptr_t>> valid_fp;
  if (cacheable) {
    for (auto& kv : swaps) {
      BaseRec& br = c->bases[kv.first];
      after.push_back({kv.first, {br.dptr, br.shadow}});
      if (kv.second % 2) std::swap(br.dptr, br.shadow);
    }
    valid_fp = fingerprint(c, rp);
    for (auto& a : after) {
      BaseRec& br = c->bases[a.first];
      br.dptr = a.second.first;
      br.shadow = a.second.second;
    }
    var = nullptr;
    for (auto& v : cb->v)
      if (v.fingerprint == valid_fp) var = &v;
    if (!var) {
      if (cb->v.size() >= 2) {
        // replace the least recently used address set
        auto lru = std::min_element(cb->v.begin(), cb->v.end(), [](const CachedVariant& a, const CachedVariant& b) {
          return a.last_use < b.last_use;
        });
        release_variant(*lru);
        cb->v.erase(lru);
      }
      cb->v.emplace_back();
      var = &cb->v.back();
      var->fingerprint = valid_fp;
    }
    var->after = after;
    var->last_use = ++use_clock;
    if (graphs) var->seen++;
  }
  if (!capture) {
    if (cacheable) {
      var->eager = std::move(issued);
      var->has_eager = true;
    }
    return;
  }
  // capture the recorded launches into a graph and replay it
  std::vector<void*> keep;
  for (auto& L : recorded) {
    if (!L.packed) continue;
    int64_t db = (int64_t)(L.descs.size() * 8), pb = (int64_t)(L.prefix.size() * 8);
    char* d = nullptr;
    cuda_check(cudaMalloc((void**)&d, db + pb), "cudaMalloc(descriptors)");
    cuda_check(cudaMemcpy(d, L.descs.data(), db, cudaMemcpyHostToDevice), "descriptors");
    cuda_check(cudaMemcpy(d + db, L.prefix.data(), pb, cudaMemcpyHostToDevice), "prefix");
    L.d_descs = d;
    L.d_prefix = d + db;
    keep.push_back(d);
  }
  static thread_local cudaStream_t cap = nullptr;
  if (!cap) cuda_check(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
  Exec cex = *ex;
  cex.stream = cap;
  cuda_check(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  try {
    for (auto& L : recorded) issue(c, &cex, L, true);
  } catch (...) {
    cudaGraph_t g;
    cudaStreamEndCapture(cap, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  cudaGraph_t graph;
  cuda_check(cudaStreamEndCapture(cap, &graph), "cudaStreamEndCapture");
  cudaGraphExec_t gexec;
  cuda_check(cudaGraphInstantiate(&gexec, graph, 0), "cudaGraphInstantiate");
  release_variant(*var);
  var->exec = gexec;
  var->graph = graph;
  var->keep = keep;
  var->launches = (int64_t)recorded.size();
  var->packed_launches = std::count_if(recorded.begin(), recorded.end(), [](const Launch& L) { return L.packed; });
  c->stats.graph_captures++;
  cuda_check(cudaGraphLaunch(gexec, ex->stream), "cudaGraphLaunch");
  c->stats.graph_launches++;
  c->stats.kernel_launches += var->launches;
  c->stats.packed_launches += var->packed_launches;
}

}  // namespace vbe
