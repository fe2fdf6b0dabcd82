// CPU emulation of the CUDA features the generated kernels use, so that
// tests can run a recorded launch on the host: every CUDA thread of a block
// is a std::thread, blocks run one after another, __syncthreads and warp
// shuffles are barriers, and every memory access goes through a checked
// pointer that rejects addresses outside the allocations the library made.
// Test infrastructure only.
#pragma once
#define VBE_EMU 1

#include <atomic>
#include <barrier>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

struct dim3 {
  unsigned x = 1, y = 1, z = 1;
};
struct uint4 {
  unsigned x, y, z, w;
};
struct uint2 {
  unsigned x, y;
};

extern thread_local dim3 threadIdx, blockIdx;
extern dim3 blockDim, gridDim;

#define __global__
#define __device__
#define __align__(x) alignas(x)
#define __grid_constant__
#define __forceinline__ inline
#define SF_CALL __attribute__((noinline))
#define __launch_bounds__(...)
#define __maxnreg__(...)
#define __shared__ static

struct EmuRange {
  uintptr_t lo, hi;
};
extern std::vector<EmuRange> g_ranges;
extern std::atomic<long long> g_bad;
extern char g_bad_msg[256];
extern std::barrier<>* g_block_bar;
extern std::vector<std::unique_ptr<std::barrier<>>> g_warp_bar;
extern unsigned long long g_xchg[1024];

inline bool emu_ok(const volatile void* p, size_t n) {
  uintptr_t a = (uintptr_t)p;
  for (auto& r : g_ranges)
    if (a >= r.lo && a + n <= r.hi) return true;
  if (g_bad.fetch_add(1) == 0)
    snprintf(g_bad_msg, sizeof g_bad_msg, "access of %zu bytes at %p outside every allocation", n, (const void*)a);
  return false;
}

template <class T>
struct CP {  // checked pointer
  T* p;
  T& operator[](long long i) const {
    static thread_local typename std::remove_cv<T>::type dummy;
    if (!emu_ok(p + i, sizeof(T))) return (T&)dummy;
    return p[i];
  }
  CP operator+(long long i) const { return CP{p + i}; }
};
template <class T>
inline CP<T> vbe_ptr(long long v) {
  return CP<T>{reinterpret_cast<T*>(v)};
}
template <class T>
inline bool vbe_aligned16(CP<T> p) {
  return ((uintptr_t)p.p & 15) == 0;
}
template <class T, int E>
inline void vbe_vload(CP<const T> p, T (&o)[E]) {
  if (((uintptr_t)p.p) % (sizeof(T) * E) != 0 && g_bad.fetch_add(1) == 0)
    snprintf(g_bad_msg, sizeof g_bad_msg, "misaligned vector load at %p", (void*)p.p);
  if (!emu_ok(p.p, sizeof(T) * E)) return;
  for (int e = 0; e < E; ++e) o[e] = p.p[e];
}
template <class T, int E>
inline void vbe_vstore(CP<T> p, const T (&o)[E]) {
  if (((uintptr_t)p.p) % (sizeof(T) * E) != 0 && g_bad.fetch_add(1) == 0)
    snprintf(g_bad_msg, sizeof g_bad_msg, "misaligned vector store at %p", (void*)p.p);
  if (!emu_ok(p.p, sizeof(T) * E)) return;
  for (int e = 0; e < E; ++e) p.p[e] = o[e];
}

template <class T, int E>
inline void vbe_vload(const T* p, T (&o)[E]) {  // shared-memory source (unchecked)
  for (int e = 0; e < E; ++e) o[e] = p[e];
}
#define VBE_DYN_SMEM static unsigned char vbe_smem[262144] __attribute__((aligned(128)))

// mbarriers, kept in a table beside the shared memory they would occupy: a
// phase completes when its expected arrivals have arrived and the bytes of
// the copies it tracks have landed (copies land when they are issued on the
// host). Waits poll with a time limit, as the device waits do with an
// iteration limit, and an arrival on a barrier nobody initialised is an error.
struct EmuBar {
  int expected = 0, pending = 0;
  long long tx = 0;
  unsigned phase = 0;
};
inline std::mutex& emu_bar_mu() {
  static std::mutex m;
  return m;
}
inline std::unordered_map<const void*, EmuBar>& emu_bars() {
  static std::unordered_map<const void*, EmuBar> t;
  return t;
}
inline EmuBar* emu_bar(const void* bar) {
  auto it = emu_bars().find(bar);
  if (it != emu_bars().end()) return &it->second;
  if (g_bad.fetch_add(1) == 0) snprintf(g_bad_msg, sizeof g_bad_msg, "mbarrier at %p used before its init", bar);
  return nullptr;
}
inline void emu_bar_settle(EmuBar* b) {
  if (b->pending < 0 && g_bad.fetch_add(1) == 0)
    snprintf(g_bad_msg, sizeof g_bad_msg, "more arrivals on an mbarrier phase than it expects");
  if (b->pending == 0 && b->tx == 0) {
    ++b->phase;
    b->pending = b->expected;
  }
}
inline void vbe_mbar_init(unsigned long long* bar, unsigned count) {
  std::lock_guard<std::mutex> g(emu_bar_mu());
  emu_bars()[bar] = EmuBar{(int)count, (int)count, 0, 0};
}
inline void vbe_fence_mbar_init() {}
inline void vbe_fence_proxy_async() {}
inline void vbe_mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  std::lock_guard<std::mutex> g(emu_bar_mu());
  if (EmuBar* b = emu_bar(bar)) {
    b->tx += bytes;
    --b->pending;
    emu_bar_settle(b);
  }
}
inline void vbe_mbar_arrive(unsigned long long* bar) {
  std::lock_guard<std::mutex> g(emu_bar_mu());
  if (EmuBar* b = emu_bar(bar)) {
    --b->pending;
    emu_bar_settle(b);
  }
}
inline void emu_bar_landed(unsigned long long* bar, long long bytes) {
  std::lock_guard<std::mutex> g(emu_bar_mu());
  if (EmuBar* b = emu_bar(bar)) {
    b->tx -= bytes;
    if (b->tx < 0 && g_bad.fetch_add(1) == 0)
      snprintf(g_bad_msg, sizeof g_bad_msg, "copies landed beyond the bytes an mbarrier phase expects");
    emu_bar_settle(b);
  }
}
// g_emu_drop: bulk and tensor copies never land (a copy that never
// completes), and every wait gives up after 50 ms instead of 60 s
extern int g_emu_drop;
inline bool vbe_mbar_wait(unsigned long long* bar, unsigned parity) {
  const auto until = std::chrono::steady_clock::now() +
                     (g_emu_drop ? std::chrono::milliseconds(50) : std::chrono::milliseconds(60000));
  for (;;) {
    {
      std::lock_guard<std::mutex> g(emu_bar_mu());
      EmuBar* b = emu_bar(bar);
      if (!b) return false;
      if ((b->phase & 1u) != (parity & 1u)) return true;
    }
    if (std::chrono::steady_clock::now() > until) return false;
    std::this_thread::yield();
  }
}
// a wait of at most `polls` polls: zero polls give up at once, as on the
// device; otherwise the time-limited wait above
inline bool vbe_mbar_wait_n(unsigned long long* bar, unsigned parity, unsigned polls) {
  if (polls == 0) return false;
  return vbe_mbar_wait(bar, parity);
}
inline void vbe_bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  if ((((uintptr_t)dst) | ((uintptr_t)src) | bytes) % 16 != 0 && g_bad.fetch_add(1) == 0)
    snprintf(g_bad_msg, sizeof g_bad_msg, "bulk copy not 16-byte aligned: %p <- %p, %u bytes", dst, src, bytes);
  if (g_emu_drop) return;
  if (emu_ok(src, bytes)) memcpy(dst, src, bytes);
  emu_bar_landed(bar, bytes);
}

// named barriers over the first n threads of a block (one per id and n,
// reused by every block), optionally or-reducing a predicate
struct EmuNamedBar {
  bool acc = false, result = false;
  std::barrier<std::function<void()>> bar;
  explicit EmuNamedBar(int n) : bar(n, std::function<void()>([this] { result = acc; acc = false; })) {}
};
inline EmuNamedBar& emu_named_bar(int id, int n) {
  static std::mutex m;
  static std::map<std::pair<int, int>, std::unique_ptr<EmuNamedBar>> t;
  std::lock_guard<std::mutex> g(m);
  auto& e = t[{id, n}];
  if (!e) e.reset(new EmuNamedBar(n));
  return *e;
}
inline bool vbe_bar_or(int id, int n, bool v) {
  if ((int)threadIdx.x >= n && g_bad.fetch_add(1) == 0)
    snprintf(g_bad_msg, sizeof g_bad_msg, "thread outside the %d threads of named barrier %d", n, id);
  EmuNamedBar& b = emu_named_bar(id, n);
  if (v) {
    static std::mutex m;
    std::lock_guard<std::mutex> g(m);
    b.acc = true;
  }
  b.bar.arrive_and_wait();
  return b.result;
}
inline void vbe_bar_sync(int id, int n) { (void)vbe_bar_or(id, n, false); }
inline void __syncwarp(unsigned = 0xffffffffu) { g_warp_bar[threadIdx.x >> 5]->arrive_and_wait(); }

inline void vbe_grid_wait() {}  // launches run one after another on the host

// a tensor copy, from the description a recording context writes into the
// map (address, row stride, rows, row bytes, box columns, box rows, element
// size); elements outside the tensor read as zeros
inline void vbe_tma_2d(void* dst, const void* tmap, int x, int y, unsigned long long* bar) {
  if (g_emu_drop) return;
  const long long* m = (const long long*)tmap;
  const char* base = (const char*)m[0];
  const long long pitch = m[1], rows = m[2], bc = m[4], br = m[5], isz = m[6];
  char* d = (char*)dst;
  for (long long r = 0; r < br; ++r)
    for (long long c = 0; c < bc; ++c) {
      const long long gx = x + c, gy = y + r;
      char* out = d + (r * bc + c) * isz;
      if (gx < 0 || gx >= pitch || gy < 0 || gy >= rows) {
        memset(out, 0, (size_t)isz);
        continue;
      }
      const char* src = base + (gy * pitch + gx) * isz;
      if (emu_ok(src, (size_t)isz)) memcpy(out, src, (size_t)isz);
    }
  emu_bar_landed(bar, br * bc * isz);
}

inline void __syncthreads() { g_block_bar->arrive_and_wait(); }
inline void __threadfence() { std::atomic_thread_fence(std::memory_order_seq_cst); }
inline unsigned atomicAdd(CP<unsigned> p, unsigned v) {
  if (!emu_ok(p.p, 4)) return 0;
  return __atomic_fetch_add(p.p, v, __ATOMIC_SEQ_CST);
}
inline unsigned atomicAdd(unsigned* p, unsigned v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }

template <class T>
inline T __shfl_down_sync(unsigned, T v, int off) {
  static_assert(sizeof(T) <= 8, "shuffle width");
  const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long bits = 0;
  memcpy(&bits, &v, sizeof(T));
  g_xchg[threadIdx.x] = bits;
  g_warp_bar[w]->arrive_and_wait();
  T r = v;
  unsigned src = lane + (unsigned)off;
  if (src < 32 && w * 32 + src < blockDim.x) memcpy(&r, &g_xchg[w * 32 + src], sizeof(T));
  g_warp_bar[w]->arrive_and_wait();
  return r;
}

template <class T>
inline T __shfl_up_sync(unsigned, T v, int off) {
  static_assert(sizeof(T) <= 8, "shuffle width");
  const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long bits = 0;
  memcpy(&bits, &v, sizeof(T));
  g_xchg[threadIdx.x] = bits;
  g_warp_bar[w]->arrive_and_wait();
  T r = v;
  if (lane >= (unsigned)off) memcpy(&r, &g_xchg[w * 32 + lane - off], sizeof(T));
  g_warp_bar[w]->arrive_and_wait();
  return r;
}

inline double __longlong_as_double(long long v) {
  double d;
  memcpy(&d, &v, 8);
  return d;
}
inline float __int_as_float(int v) {
  float f;
  memcpy(&f, &v, 4);
  return f;
}
inline long long min(long long a, long long b) { return a < b ? a : b; }
inline long long __double_as_longlong(double d) {
  long long v;
  memcpy(&v, &d, 8);
  return v;
}
inline int __float_as_int(float f) {
  int v;
  memcpy(&v, &f, 4);
  return v;
}
inline unsigned __float_as_uint(float f) {
  unsigned v;
  memcpy(&v, &f, 4);
  return v;
}
inline float __uint_as_float(unsigned v) {
  float f;
  memcpy(&f, &v, 4);
  return f;
}
inline unsigned long long vbe_umulhi(unsigned long long a, unsigned long long b) {
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
}
inline long long vbe_smulhi(long long a, long long b) { return (long long)(((__int128)a * b) >> 64); }
inline int vbe_clz64(unsigned long long x) { return x ? __builtin_clzll(x) : 64; }
inline float vbe_rcp_approx(float x) { return 1.0f / x; }
inline float vbe_rsqrt_approx(float x) { return 1.0f / std::sqrt(x); }

template <class F>
void emu_grid(unsigned grid, unsigned block, F f) {
  blockDim.x = block;
  gridDim.x = grid;
  for (unsigned b = 0; b < grid; ++b) {
    std::barrier<> bar((std::ptrdiff_t)block);
    g_block_bar = &bar;
    g_warp_bar.clear();
    for (unsigned w = 0; w * 32 < block; ++w)
      g_warp_bar.emplace_back(new std::barrier<>((std::ptrdiff_t)std::min(32u, block - w * 32)));
    std::vector<std::thread> th;
    th.reserve(block);
    for (unsigned t = 0; t < block; ++t)
      th.emplace_back([&, t, b]() {
        threadIdx.x = t;
        blockIdx.x = b;
        f();
      });
    for (auto& x : th) x.join();
  }
}
