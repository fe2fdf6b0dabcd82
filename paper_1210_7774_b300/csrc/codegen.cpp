// Code generator: one CUDA kernel per run, compiled by NVRTC for sm_103a.
//
// The paper proposes JIT compilation of instruction kernels as the remedy
// for memory-bound bytecode execution (section "Future Work"). Each run is
// rendered as straight-line CUDA: the run's instructions become a chain of
// register operations evaluated once per element; loads and stores touch
// only the run's live-in and live-out views. Iteration patterns:
//
//   elementwise / full reduction ("tile" kernels): the coalesced iteration
//     space is walked in tiles of blockDim.x * U elements of the innermost
//     dimension; a one-dimensional run whose views are unit-stride and
//     aligned uses 16-byte vector loads and stores. A full reduction keeps a
//     per-thread accumulator, reduces it in the block (warp shuffles, then
//     shared memory), writes one partial per block, and the last block to
//     finish sums the partials in block order.
//   axis reduction: one thread per output element looping over the reduced
//     dimensions (reduced dimensions outer in memory), or one block per
//     output element with the threads striding the reduced dimensions and a
//     block tree (reduced dimension inner in memory).
//   packed: many independent one-dimensional runs of one signature in one
//     persistent launch; blocks take fixed-size chunks from an atomic
//     counter, and the last chunk of an instance to finish sums that
//     instance's chunk partials in chunk order.
//
// Every reduction order depends only on the launch shape, never on timing,
// so a result is reproducible for a given signature and size.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <set>
#include <sstream>

#include "vbe_core.h"

namespace vbe {

namespace {

struct Layout {
  int nwords = 0;
  int dims0 = 0;
  int nouter = -1, inner = -1;
  int nout = -1, nred = -1;
  std::vector<int> lptr, lst, sptr, sst;
  int red_ptr = -1, red_st = -1, partials = -1, counter = -1;
  int red2_ptr = -1, red2_st = -1;  // the paired index output (axis kernels)
  int idx_st = -1;
  std::vector<int> rnd;
  int consts = -1;
  int bulk_ch = -1, err = -1;  // tile kernels: bulk-copy chunk (elements), error word
};

bool tile_mode(Mode m) { return m == Mode::ELEM || m == Mode::FULL; }

Layout layout_of(const Run& r, const Canon& c) {
  Layout L;
  int w = 0;
  int nst;  // strides per slot
  L.dims0 = w;
  if (tile_mode(c.spec.mode)) {
    w += c.spec.nd;
    L.nouter = w++;
    L.inner = w++;
    nst = c.spec.nd;
  } else {
    w += c.spec.ndk + c.spec.ndr;
    L.nout = w++;
    L.nred = w++;
    nst = c.spec.ndk + c.spec.ndr;
  }
  for (size_t s = 0; s < r.loads.size(); ++s) {
    L.lptr.push_back(w++);
    L.lst.push_back(w);
    w += nst;
  }
  for (size_t s = 0; s < r.stores.size(); ++s) {
    L.sptr.push_back(w++);
    L.sst.push_back(w);
    w += nst;
  }
  if (r.has_red) {
    L.red_ptr = w++;
    if (!tile_mode(c.spec.mode)) {
      L.red_st = w;
      w += c.spec.ndk;
      if (r.has_red2) {
        L.red2_ptr = w++;
        L.red2_st = w;
        w += c.spec.ndk;
      }
    } else {
      L.partials = w++;
      L.counter = w++;
    }
  }
  if (r.nrandom > 0 && !tile_mode(c.spec.mode)) {
    L.idx_st = w;
    w += c.spec.ndk + c.spec.ndr;
  }
  for (int k = 0; k < r.nrandom; ++k) {
    L.rnd.push_back(w);
    w += 3;
  }
  L.consts = w;
  w += (int)r.consts.size();
  if (tile_mode(c.spec.mode)) {
    L.bulk_ch = w++;
    L.err = w++;
  }
  L.nwords = std::max(w, 1);
  return L;
}

// merge consecutive dims (in the given order) when every stride list agrees
void coalesce(std::vector<int64_t>& dims, std::vector<std::vector<int64_t>*> lists) {
  std::vector<int64_t> nd;
  std::vector<std::vector<int64_t>> nl(lists.size());
  for (size_t k = 0; k < dims.size(); ++k) {
    if (dims[k] == 1) continue;
    if (!nd.empty()) {
      bool ok = true;
      for (size_t s = 0; s < lists.size(); ++s)
        if (nl[s].back() != (*lists[s])[k] * dims[k]) ok = false;
      if (ok) {
        nd.back() *= dims[k];
        for (size_t s = 0; s < lists.size(); ++s) nl[s].back() = (*lists[s])[k];
        continue;
      }
    }
    nd.push_back(dims[k]);
    for (size_t s = 0; s < lists.size(); ++s) nl[s].push_back((*lists[s])[k]);
  }
  dims = nd;
  for (size_t s = 0; s < lists.size(); ++s) *lists[s] = nl[s];
}

std::vector<int64_t> c_strides(const std::vector<int64_t>& shape) {
  std::vector<int64_t> st(shape.size());
  int64_t acc = 1;
  for (int k = (int)shape.size() - 1; k >= 0; --k) {
    st[k] = acc;
    acc *= std::max<int64_t>(1, shape[k]);
  }
  return st;
}

int cls_of(int64_t s) { return s == 0 ? 0 : (s == 1 ? 1 : 2); }

}  // namespace

Canon canonicalize(const Run& r, bool allow_vec, const std::vector<uintptr_t>& load_ptrs,
                   const std::vector<uintptr_t>& store_ptrs, uintptr_t red_ptr) {
  Canon c;
  int D = (int)r.shape.size();
  c.total = r.elements();
  // every slot must describe the run's iteration space (internal invariant)
  for (auto& s : r.loads)
    if ((int)s.st.size() != D) fail(VBE_ERR_INVALID, "internal: load slot rank differs from the run's");
  for (auto& s : r.stores)
    if ((int)s.st.size() != D) fail(VBE_ERR_INVALID, "internal: store slot rank differs from the run's");
  if (r.has_red && (int)r.red_out.st.size() != D - (int)r.red_axes.size())
    fail(VBE_ERR_INVALID, "internal: reduction output rank");
  // ARGMIN/ARGMAX keep the axis path (an index along the reduced axis)
  bool full = r.has_red && (int)r.red_axes.size() == D && r.red_op != VBE_OP_ARGMIN_REDUCE &&
              r.red_op != VBE_OP_ARGMAX_REDUCE && !r.has_red2;
  if (!r.has_red || full) {
    c.spec.mode = r.has_red ? Mode::FULL : Mode::ELEM;
    std::vector<int64_t> dims = r.shape;
    c.lst.clear();
    for (auto& s : r.loads) c.lst.push_back(s.st);
    for (auto& s : r.stores) c.sst.push_back(s.st);
    std::vector<std::vector<int64_t>*> lists;
    for (auto& v : c.lst) lists.push_back(&v);
    for (auto& v : c.sst) lists.push_back(&v);
    coalesce(dims, lists);
    if (dims.empty()) {
      dims.push_back(1);
      for (auto* l : lists) l->assign(1, 0);
    }
    c.dims = dims;
    c.spec.nd = (int)dims.size();
    for (auto& v : c.lst) c.spec.load_cls.push_back(cls_of(v.back()));
    for (auto& v : c.sst) c.spec.store_cls.push_back(cls_of(v.back()));
    // vector path: one dimension, unit or zero strides, aligned pointers
    if (allow_vec && c.spec.nd == 1) {
      int maxsz = 0;
      bool ok = true;
      for (size_t s = 0; s < r.loads.size(); ++s) {
        if (c.spec.load_cls[s] == 2) ok = false;
        if (c.spec.load_cls[s] == 1) maxsz = std::max(maxsz, itemsize(r.loads[s].dtype));
      }
      for (size_t s = 0; s < r.stores.size(); ++s) {
        if (c.spec.store_cls[s] != 1) ok = false;
        maxsz = std::max(maxsz, itemsize(r.stores[s].dtype));
      }
      if (ok && maxsz > 0) {
        int E = 16 / maxsz;
        for (size_t s = 0; s < r.loads.size(); ++s) {
          if (c.spec.load_cls[s] != 1) continue;
          int b = E * itemsize(r.loads[s].dtype);
          uintptr_t p = load_ptrs[s] + (uintptr_t)(r.loads[s].offset * itemsize(r.loads[s].dtype));
          if (p % b) ok = false;
        }
        for (size_t s = 0; s < r.stores.size(); ++s) {
          int b = E * itemsize(r.stores[s].dtype);
          uintptr_t p = store_ptrs[s] + (uintptr_t)(r.stores[s].offset * itemsize(r.stores[s].dtype));
          if (p % b) ok = false;
        }
        if (ok) {
          c.spec.vec = true;
          c.spec.E = E;
        }
      }
    }
    (void)red_ptr;
    return c;
  }
  // axis reduction: kept dims (in order) then reduced dims
  std::vector<int> kept, red = r.red_axes;
  for (int d = 0; d < D; ++d)
    if (!std::binary_search(red.begin(), red.end(), d)) kept.push_back(d);
  std::vector<int64_t> cst = c_strides(r.shape);
  auto pick = [](const std::vector<int64_t>& v, const std::vector<int>& idx) {
    std::vector<int64_t> o;
    for (int i : idx) o.push_back(v[i]);
    return o;
  };
  std::vector<int64_t> kd = pick(r.shape, kept), rd = pick(r.shape, red);
  std::vector<std::vector<int64_t>> lk, lr, sk, sr;
  for (auto& s : r.loads) {
    lk.push_back(pick(s.st, kept));
    lr.push_back(pick(s.st, red));
  }
  for (auto& s : r.stores) {
    sk.push_back(pick(s.st, kept));
    sr.push_back(pick(s.st, red));
  }
  std::vector<int64_t> outk = r.red_out.st;  // already over the kept dims
  std::vector<int64_t> outk2 = r.has_red2 ? r.red2_out.st : r.red_out.st;
  std::vector<int64_t> ik = pick(cst, kept), ir = pick(cst, red);
  {
    std::vector<std::vector<int64_t>*> L;
    for (auto& v : lk) L.push_back(&v);
    for (auto& v : sk) L.push_back(&v);
    L.push_back(&outk);
    if (r.has_red2) L.push_back(&outk2);
    if (r.nrandom) L.push_back(&ik);
    coalesce(kd, L);
  }
  {
    std::vector<std::vector<int64_t>*> L;
    for (auto& v : lr) L.push_back(&v);
    for (auto& v : sr) L.push_back(&v);
    if (r.nrandom) L.push_back(&ir);
    coalesce(rd, L);
  }
  if (rd.empty()) {  // reducing extent-1 dims only
    rd.push_back(1);
    for (auto& v : lr) v.assign(1, 0);
    for (auto& v : sr) v.assign(1, 0);
    ir.assign(1, 0);
  }
  c.spec.ndk = (int)kd.size();
  c.spec.ndr = (int)rd.size();
  c.dims = kd;
  c.dims.insert(c.dims.end(), rd.begin(), rd.end());
  for (size_t s = 0; s < lk.size(); ++s) {
    std::vector<int64_t> v = lk[s];
    v.insert(v.end(), lr[s].begin(), lr[s].end());
    c.lst.push_back(v);
    c.spec.load_cls.push_back(cls_of(lr[s].back()));
  }
  for (size_t s = 0; s < sk.size(); ++s) {
    std::vector<int64_t> v = sk[s];
    v.insert(v.end(), sr[s].begin(), sr[s].end());
    c.sst.push_back(v);
    c.spec.store_cls.push_back(cls_of(sr[s].back()));
  }
  c.red_st = outk;
  if (r.has_red2) c.red2_st = outk2;
  c.idx_st = ik;
  c.idx_st.insert(c.idx_st.end(), ir.begin(), ir.end());
  int64_t nred = 1, nout = 1;
  for (auto v : rd) nred *= v;
  for (auto v : kd) nout *= v;
  // one block per output when the reduced dimension is inner in memory
  bool inner_unit = !r.loads.empty() && lr[0].back() == 1;
  c.spec.mode = (nred >= 64 && (inner_unit || nout < 4 * 148)) ? Mode::AXIS_BLOCK : Mode::AXIS_THREAD;
  return c;
}

int words_count(const Run& r, const Canon& c) { return layout_of(r, c).nwords; }

// a constant operand as the parameter word the generated code decodes
static int64_t const_bits(const Operand& o) {
  int64_t bits = o.i;
  if (o.dtype == VBE_FLOAT64) {
    memcpy(&bits, &o.f, 8);
  } else if (o.dtype == VBE_FLOAT32) {
    float g = (float)o.f;
    uint32_t b32;
    memcpy(&b32, &g, 4);
    bits = (int64_t)b32;
  }
  return bits;
}

void fill_words(const Run& r, const Canon& c, const std::vector<uintptr_t>& load_ptrs,
                const std::vector<uintptr_t>& store_ptrs, uintptr_t red_ptr, uintptr_t partials,
                uintptr_t counter, int64_t block, int64_t U, LaunchArgs* out, int64_t chunk, uintptr_t err,
                uintptr_t red2_ptr) {
  (void)block;
  (void)U;
  Layout L = layout_of(r, c);
  std::vector<int64_t>& w = out->w;
  w.assign(L.nwords, 0);
  for (size_t k = 0; k < c.dims.size(); ++k) w[L.dims0 + k] = c.dims[k];
  if (tile_mode(c.spec.mode)) {
    int64_t no = 1;
    for (int k = 0; k + 1 < c.spec.nd; ++k) no *= c.dims[k];
    w[L.nouter] = no;
    w[L.inner] = c.dims[c.spec.nd - 1];
  } else {
    int64_t no = 1, nr = 1;
    for (int k = 0; k < c.spec.ndk; ++k) no *= c.dims[k];
    for (int k = 0; k < c.spec.ndr; ++k) nr *= c.dims[c.spec.ndk + k];
    w[L.nout] = no;
    w[L.nred] = nr;
  }
  for (size_t s = 0; s < r.loads.size(); ++s) {
    w[L.lptr[s]] = (int64_t)(load_ptrs[s] + (uintptr_t)(r.loads[s].offset * itemsize(r.loads[s].dtype)));
    for (size_t k = 0; k < c.lst[s].size(); ++k) w[L.lst[s] + k] = c.lst[s][k];
  }
  for (size_t s = 0; s < r.stores.size(); ++s) {
    w[L.sptr[s]] = (int64_t)(store_ptrs[s] + (uintptr_t)(r.stores[s].offset * itemsize(r.stores[s].dtype)));
    for (size_t k = 0; k < c.sst[s].size(); ++k) w[L.sst[s] + k] = c.sst[s][k];
  }
  if (r.has_red) {
    w[L.red_ptr] = (int64_t)(red_ptr + (uintptr_t)(r.red_out.offset * itemsize(r.red_dtype)));
    if (L.red_st >= 0)
      for (size_t k = 0; k < c.red_st.size(); ++k) w[L.red_st + k] = c.red_st[k];
    if (L.red2_ptr >= 0) {
      w[L.red2_ptr] = (int64_t)(red2_ptr + (uintptr_t)(r.red2_out.offset * 8));
      for (size_t k = 0; k < c.red2_st.size(); ++k) w[L.red2_st + k] = c.red2_st[k];
    }
    if (L.partials >= 0) {
      w[L.partials] = (int64_t)partials;
      w[L.counter] = (int64_t)counter;
    }
  }
  if (L.idx_st >= 0)
    for (size_t k = 0; k < c.idx_st.size(); ++k) w[L.idx_st + k] = c.idx_st[k];
  for (size_t k = 0; k < r.consts.size(); ++k) w[L.consts + k] = const_bits(r.consts[k]);
  if (L.bulk_ch >= 0) {
    w[L.bulk_ch] = chunk;
    w[L.err] = (int64_t)err;
  }
  int ri = 0;
  for (auto& s : r.steps) {
    if (s.op != VBE_OP_RANDOM) continue;
    w[L.rnd[ri]] = (int64_t)s.seed;
    w[L.rnd[ri] + 1] = (int64_t)s.key;
    w[L.rnd[ri] + 2] = s.rstep;
    ++ri;
  }
}

// ---------------------------------------------------------------- source

namespace {

const char* kPrelude = R"CUDA(
typedef long long i64;
typedef unsigned long long u64;
__device__ __forceinline__ i64 vbe_iadd(i64 a, i64 b) { return (i64)((u64)a + (u64)b); }
__device__ __forceinline__ i64 vbe_isub(i64 a, i64 b) { return (i64)((u64)a - (u64)b); }
__device__ __forceinline__ i64 vbe_imul(i64 a, i64 b) { return (i64)((u64)a * (u64)b); }
__device__ __forceinline__ i64 vbe_ineg(i64 a) { return (i64)(0ull - (u64)a); }
__device__ __forceinline__ i64 vbe_iabs(i64 a) { return a < 0 ? vbe_ineg(a) : a; }
template <class T> __device__ __forceinline__ T vbe_max(T a, T b) { return (a > b || a != a) ? a : b; }
// IEEE division with zero numerators kept off the hardware sequence's slow
// path (tile-fused stencil kernels: state fields such as the momenta of a
// fluid at rest are mostly zeros). For a == 0 the quotient is a * (2^-64 / b):
// 2^-64 / b is finite and non-zero for every finite non-zero b, subnormal b
// included, so the product is the zero with the sign of a / b; it is NaN
// for b = 0 (2^-64 / 0 = inf) or NaN, and a zero for an infinite b, exactly
// as a / b.
template <class T> __device__ __forceinline__ T vbe_zdiv(T a, T b) {
  const bool z = a == (T)0;
  const T q = (z ? (T)0x1p-64 : a) / b;
  return z ? a * q : q;
}
template <class T> __device__ __forceinline__ T vbe_min(T a, T b) { return (a < b || a != a) ? a : b; }
// ARGMIN/ARGMAX: keep (x, j) over (v, i) when x is better, a NaN counting
// as better than any number and equal values going to the lower index (the
// first occurrence); associative and commutative, so every combining order
// gives the same pair
template <class T> __device__ __forceinline__ void vbe_arg_upd(T& v, i64& i, T x, i64 j, bool maxi) {
  const bool xn = x != x, vn = v != v;
  const bool better = maxi ? (x > v) : (x < v);
  const bool take = (xn || vn) ? (xn && (!vn || j < i)) : (better || (x == v && j < i));
  if (take) { v = x; i = j; }
}
// float64 orderings on the integer pipes (the FP64 pipe is B300's scarcest):
// for numbers, the bit pattern with the sign folded (negatives negated)
// orders like the values and maps -0 and +0 to the same key; a NaN is a
// pattern above the infinity's once the sign is cleared
__device__ __forceinline__ bool vbe_disnan(i64 u) { return (u & 0x7fffffffffffffffll) > 0x7ff0000000000000ll; }
__device__ __forceinline__ i64 vbe_dkey(i64 u) { return u < 0 ? -(u & 0x7fffffffffffffffll) : u; }
template <> __device__ __forceinline__ double vbe_min<double>(double a, double b) {
  const i64 ua = __double_as_longlong(a), ub = __double_as_longlong(b);
  return (vbe_disnan(ua) || (!vbe_disnan(ub) && vbe_dkey(ua) < vbe_dkey(ub))) ? a : b;
}
template <> __device__ __forceinline__ double vbe_max<double>(double a, double b) {
  const i64 ua = __double_as_longlong(a), ub = __double_as_longlong(b);
  return (vbe_disnan(ua) || (!vbe_disnan(ub) && vbe_dkey(ua) > vbe_dkey(ub))) ? a : b;
}
template <> __device__ __forceinline__ void vbe_arg_upd<double>(double& v, i64& i, double x, i64 j, bool maxi) {
  const i64 ux = __double_as_longlong(x), uv = __double_as_longlong(v);
  const bool xn = vbe_disnan(ux), vn = vbe_disnan(uv);
  const i64 kx = vbe_dkey(ux), kv = vbe_dkey(uv);
  const bool better = maxi ? (kx > kv) : (kx < kv);
  const bool take = (xn || vn) ? (xn && (!vn || j < i)) : (better || (kx == kv && j < i));
  if (take) { v = x; i = j; }
}
// polls of a compute thread's wait for its staged data (the waits of a
// producer and of the final drain always allow 2^24); a context may lower it
// (vbe_debug_set_wait_polls) to make those waits run out in a test
#ifndef VBE_CWAIT
#define VBE_CWAIT (1u << 24)
#endif
// RANDOM: splitmix64 finaliser of seed + (key + step*m + 1) * golden gamma,
// top 53 bits scaled to [0, 1)
__device__ __forceinline__ double vbe_u01(u64 seed, u64 key, u64 step, u64 m) {
  u64 z = seed + (key + step * m + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * 1.1102230246251565404236316680908203125e-16;
}
#ifndef VBE_EMU
template <class T> __device__ __forceinline__ T* vbe_ptr(i64 v) { return reinterpret_cast<T*>(v); }
template <class T> __device__ __forceinline__ bool vbe_aligned16(const T* p) { return ((u64)p & 15ull) == 0; }
template <int B> struct vbe_vec;
template <> struct vbe_vec<16> { typedef uint4 t; };
template <> struct vbe_vec<8> { typedef uint2 t; };
template <> struct vbe_vec<4> { typedef unsigned int t; };
template <> struct vbe_vec<2> { typedef unsigned short t; };
template <> struct vbe_vec<1> { typedef unsigned char t; };
template <class T, int E> __device__ __forceinline__ void vbe_vload(const T* p, T (&o)[E]) {
  typedef typename vbe_vec<sizeof(T) * E>::t V;
  union { V v; T t[E]; } u;
  u.v = *reinterpret_cast<const V*>(p);
#pragma unroll
  for (int e = 0; e < E; ++e) o[e] = u.t[e];
}
template <class T, int E> __device__ __forceinline__ void vbe_vstore(T* p, const T (&o)[E]) {
  typedef typename vbe_vec<sizeof(T) * E>::t V;
  union { V v; T t[E]; } u;
#pragma unroll
  for (int e = 0; e < E; ++e) u.t[e] = o[e];
  *reinterpret_cast<V*>(p) = u.v;
}
// bulk asynchronous copies (TMA engine) into shared memory, completed on an
// mbarrier; waits are bounded and report failure instead of hanging
__device__ __forceinline__ unsigned vbe_saddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void vbe_mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(vbe_saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void vbe_fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void vbe_fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void vbe_mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(vbe_saddr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void vbe_bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(vbe_saddr(dst)), "l"(src), "r"(bytes), "r"(vbe_saddr(bar)) : "memory");
}
// at most `polls` polls: false when the phase has not completed by then
__device__ __forceinline__ bool vbe_mbar_wait_n(unsigned long long* bar, unsigned parity, unsigned polls) {
  for (unsigned it = 0; it < polls; ++it) {
    unsigned ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok) : "r"(vbe_saddr(bar)), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ bool vbe_mbar_wait(unsigned long long* bar, unsigned parity) {
  return vbe_mbar_wait_n(bar, parity, 1u << 24);
}
#define VBE_DYN_SMEM extern __shared__ __align__(128) unsigned char vbe_smem[]
// programmatic dependent launch: a kernel launched while its predecessor on
// the stream is still running waits here until that grid has completed and
// its writes are visible (a no-op for an ordinary launch). Kernels do not
// trigger their successors early: measured, that slowed the persistent
// tensor-copy kernels (the successor's blocks took resources while the
// predecessor still ran) and gained nothing elsewhere.
__device__ __forceinline__ void vbe_grid_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ unsigned long long vbe_umulhi(unsigned long long a, unsigned long long b) {
  return __umul64hi(a, b);
}
__device__ __forceinline__ long long vbe_smulhi(long long a, long long b) { return __mul64hi(a, b); }
__device__ __forceinline__ int vbe_clz64(unsigned long long x) { return __clzll((long long)x); }
__device__ __forceinline__ float vbe_rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float vbe_rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
#endif
)CUDA";

// Tensor-copy helpers, only in sources of groups with the tensor-copy form:
// a tensor map (an opaque 128-byte, 64-byte aligned descriptor) and a
// two-dimensional tiled copy of the box at (x, y) into shared memory,
// completed on an mbarrier; boxes reaching outside the tensor read zeros.
const char* kTmaPrelude = R"CUDA(
struct __align__(64) vbe_tmap { unsigned long long v[16]; };
#ifndef VBE_EMU
__device__ __forceinline__ void vbe_tma_2d(void* dst, const void* tmap, int x, int y, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(vbe_saddr(dst)), "l"(tmap), "r"(x), "r"(y), "r"(vbe_saddr(bar)) : "memory");
}
// one arrival on an mbarrier (release: this thread's earlier accesses are
// ordered before the phase completes)
__device__ __forceinline__ void vbe_mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(vbe_saddr(bar)) : "memory");
}
// barrier `id` over the first n threads of the block (n a multiple of 32)
__device__ __forceinline__ void vbe_bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
// the same barrier, returning whether v holds in any of the n threads
__device__ __forceinline__ bool vbe_bar_or(int id, int n, bool v) {
  unsigned r;
  asm volatile("{ .reg .pred p, q; setp.ne.u32 p, %1, 0; bar.red.or.pred q, %2, %3, p; selp.u32 %0, 1, 0, q; }"
               : "=r"(r) : "r"((unsigned)v), "r"(id), "r"(n) : "memory");
  return r != 0;
}
#endif
)CUDA";

// float64 divide/sqrt/exp/log on the integer pipes (sf64_tables.h + sf64.cuh)
#include "_embed_sf64.inc"

// the soft float64 library reaches generated kernels as NVRTC headers; the
// include line carries a hash of their text so that compiled-kernel caches
// keyed by the source see every change of the library
std::string sf64_include() {
  static const std::string line = [] {
    uint64_t h = fnv1a(kSf64Tables, strlen(kSf64Tables));
    h = fnv1a(kSf64Code, strlen(kSf64Code), h);
    return "#include \"sf64.cuh\"  // " + hex64(h) + "\n";
  }();
  return line;
}

// definitions of the user operations a run uses (section "Interface":
// registered user-defined operations), ahead of its element function
std::string user_op_defs(const std::vector<const Run*>& runs) {
  std::vector<int> seen;
  std::string out;
  for (const Run* r : runs)
    for (auto& s : r->steps) {
      const UserOp* u = user_op(s.op);
      if (!u || std::find(seen.begin(), seen.end(), s.op) != seen.end()) continue;
      seen.push_back(s.op);
      const std::string T = ctype(u->dtype);
      out += "__device__ __forceinline__ " + T + " vbe_user_" + u->name + "(" + T + " a";
      if (u->nin > 1) out += ", " + T + " b";
      if (u->nin > 2) out += ", " + T + " c";
      out += ") {\n" + u->body + "\n}\n";
    }
  return out;
}

bool uses_soft_f64(const Run& r) {
  if (!r.soft_f64) return false;
  for (auto& s : r.steps)
    if (s.dt_in == VBE_FLOAT64 || s.op == VBE_OP_RANDOM) return true;
  return false;
}

// a float64 constant operand equal to +-2^k, k in [-1022, 1023] (part of a
// kernel's signature: such products are generated differently)
bool pow2_const(const Operand& a) {
  if (a.kind != 1 || a.dtype != VBE_FLOAT64) return false;
  uint64_t u;
  memcpy(&u, &a.f, 8);
  const int e = (int)((u >> 52) & 0x7ff);
  return (u & 0xFFFFFFFFFFFFFull) == 0 && e != 0 && e != 0x7ff;
}

bool is_simple_f64(const Step& s) {
  if (s.dt_in != VBE_FLOAT64) return false;
  switch (s.op) {
    case VBE_OP_ADD: case VBE_OP_SUBTRACT: case VBE_OP_MULTIPLY: case VBE_OP_LESS: case VBE_OP_LESS_EQUAL:
    case VBE_OP_GREATER: case VBE_OP_GREATER_EQUAL: case VBE_OP_EQUAL: case VBE_OP_NOT_EQUAL:
      return true;
  }
  return false;
}

// Which float64 add/subtract/multiply/compare steps run on the integer
// pipes. Measured on B300 (Black-Scholes, shallow water, Monte-Carlo, all in
// float64), emulating any of them was slower than the FP64 pipe: an
// emulated add or multiply costs about as many SM cycles on the ALU and IMAD
// pipes as the native one does on the FP64 pipe, and its longer dependency
// chain hides latency worse. So by default only divide, square root, exp,
// log, the RANDOM conversion and sign operations are emulated; the
// environment variable VBE_F64_SIMPLE=cmp|mul|all moves compares,
// multiplies and compares, or every simple step, to the integer pipes for
// experiments.
// Either choice gives the same (correctly rounded) results.
std::vector<char> balance_f64(const Run& r) {
  std::vector<char> soft(r.steps.size(), 0);
  if (!r.soft_f64) return soft;
  static const char* pol = getenv("VBE_F64_SIMPLE");
  const std::string policy = pol ? pol : "none";
  for (size_t i = 0; i < r.steps.size(); ++i) {
    const Step& s = r.steps[i];
    if (!is_simple_f64(s)) continue;
    if (policy == "all") soft[i] = 1;
    if (policy == "mul" && s.op != VBE_OP_ADD && s.op != VBE_OP_SUBTRACT) soft[i] = 1;
    if (policy == "cmp" && s.op >= VBE_OP_LESS && s.op <= VBE_OP_NOT_EQUAL) soft[i] = 1;
  }
  return soft;
}

struct Gen {
  const Run& r;
  const Canon& c;
  Layout L;
  std::ostringstream o;
  const char* rt() const { return ctype(r.red_dtype); }
  bool kahan() const {
    return r.has_red && r.red_op == VBE_OP_ADD_REDUCE && r.red_dtype == VBE_FLOAT32 && !plain_sum;
  }
  // the float32 sum's plain variant (axis kernels, short reduced extents)
  bool plain_sum = false;
  // ARGMIN/ARGMAX, or MIN/MAX paired with them: (value, index) pairs
  bool arg() const {
    return r.has_red && (r.red_op == VBE_OP_ARGMIN_REDUCE || r.red_op == VBE_OP_ARGMAX_REDUCE || r.has_red2);
  }
  bool argmax() const {
    return r.has_red && (r.red_op == VBE_OP_ARGMAX_REDUCE || (r.has_red2 && r.red2_op == VBE_OP_ARGMAX_REDUCE));
  }
  // type of the values an ARGMIN/ARGMAX compares
  std::string vt() const { return ctype(r.value_dtype[r.red_value]); }

  std::vector<char> soft;  // per step: float64 add/subtract/multiply/compare emulated

  Gen(const Run& r_, const Canon& c_) : r(r_), c(c_), L(layout_of(r_, c_)), soft(balance_f64(r_)) {
  }

  bool const_params = false;  // constants arrive as arguments of the element function
  std::string opnd(const Operand& a) {
    if (a.kind == 0) return "l" + std::to_string(a.idx);
    if (a.kind == 2) return "v" + std::to_string(a.idx);
    if (const_params) return "kc" + std::to_string(a.idx);
    return const_expr(a);
  }

  // constants are parameter words (so kernels that differ only in their
  // constants share one compiled module)
  std::string const_expr(const Operand& a) {
    std::string w = "p.w[" + std::to_string(L.consts + a.idx) + "]";
    switch (a.dtype) {
      case VBE_FLOAT64: return "__longlong_as_double(" + w + ")";
      case VBE_FLOAT32: return "__int_as_float((int)" + w + ")";
      case VBE_BOOL: return "(" + w + " != 0)";
      default: return w;
    }
  }

  std::string expr(const Step& s) {
    std::string a = s.nin > 0 ? opnd(s.a[0]) : "", b = s.nin > 1 ? opnd(s.a[1]) : "",
                d = s.nin > 2 ? opnd(s.a[2]) : "";
    bool i64t = s.dt_in == VBE_INT64;
    bool f32 = s.dt_in == VBE_FLOAT32;
    const bool sf = r.soft_f64 && s.dt_in == VBE_FLOAT64;  // float64 on the integer pipes available
    if (sf && soft[&s - &r.steps[0]]) {
      switch (s.op) {
        case VBE_OP_ADD: return "vbe_dadd(" + a + ", " + b + ")";
        case VBE_OP_SUBTRACT: return "vbe_dsub(" + a + ", " + b + ")";
        case VBE_OP_MULTIPLY: return "vbe_dmul(" + a + ", " + b + ")";
        case VBE_OP_LESS: return "vbe_dlt(" + a + ", " + b + ")";
        case VBE_OP_LESS_EQUAL: return "vbe_dle(" + a + ", " + b + ")";
        case VBE_OP_GREATER: return "vbe_dlt(" + b + ", " + a + ")";
        case VBE_OP_GREATER_EQUAL: return "vbe_dle(" + b + ", " + a + ")";
        case VBE_OP_EQUAL: return "vbe_deq(" + a + ", " + b + ")";
        case VBE_OP_NOT_EQUAL: return "(!vbe_deq(" + a + ", " + b + "))";
      }
    }
    if (const UserOp* u = user_op(s.op)) {
      std::string call = "vbe_user_" + u->name + "(" + a;
      if (s.nin > 1) call += ", " + b;
      if (s.nin > 2) call += ", " + d;
      return call + ")";
    }
    if (sf && s.op == VBE_OP_NEGATIVE) return "vbe_dneg(" + a + ")";
    // float64 products by a constant power of two: on the integer pipes
    // (measured faster on the stencils and, since its divides stopped
    // issuing an FP64 compare, on Black-Scholes: 1.797 against 1.843 ms)
    if (sf && s.op == VBE_OP_MULTIPLY) {
      if (pow2_const(s.a[1])) return "vbe_dmul_k(" + a + ", " + b + ")";
      if (pow2_const(s.a[0])) return "vbe_dmul_k(" + b + ", " + a + ")";
    }
    if (sf && s.op == VBE_OP_ABSOLUTE) return "vbe_dabs(" + a + ")";
    switch (s.op) {
      case VBE_OP_ADD: return i64t ? "vbe_iadd(" + a + "," + b + ")" : "(" + a + " + " + b + ")";
      case VBE_OP_SUBTRACT: return i64t ? "vbe_isub(" + a + "," + b + ")" : "(" + a + " - " + b + ")";
      case VBE_OP_MULTIPLY: return i64t ? "vbe_imul(" + a + "," + b + ")" : "(" + a + " * " + b + ")";
      case VBE_OP_DIVIDE:
        if (r.soft_f64 && s.dt_in == VBE_FLOAT64) return "vbe_ddiv(" + a + ", " + b + ")";
        return guard_div ? "vbe_zdiv(" + a + ", " + b + ")" : "(" + a + " / " + b + ")";
      case VBE_OP_MAXIMUM: return "vbe_max(" + a + "," + b + ")";
      case VBE_OP_MINIMUM: return "vbe_min(" + a + "," + b + ")";
      case VBE_OP_SQRT:
        if (r.soft_f64 && !f32) return "vbe_dsqrt(" + a + ")";
        return std::string(f32 ? "sqrtf(" : "sqrt(") + a + ")";
      case VBE_OP_EXP:
        if (r.soft_f64 && !f32) return "vbe_dexp(" + a + ")";
        return std::string(f32 ? "expf(" : "exp(") + a + ")";
      case VBE_OP_LOG:
        if (r.soft_f64 && !f32) return "vbe_dlog(" + a + ")";
        return std::string(f32 ? "logf(" : "log(") + a + ")";
      case VBE_OP_ABSOLUTE:
        return i64t ? "vbe_iabs(" + a + ")" : std::string(f32 ? "fabsf(" : "fabs(") + a + ")";
      case VBE_OP_NEGATIVE: return i64t ? "vbe_ineg(" + a + ")" : "(-" + a + ")";
      case VBE_OP_LESS: return "(" + a + " < " + b + ")";
      case VBE_OP_LESS_EQUAL: return "(" + a + " <= " + b + ")";
      case VBE_OP_GREATER: return "(" + a + " > " + b + ")";
      case VBE_OP_GREATER_EQUAL: return "(" + a + " >= " + b + ")";
      case VBE_OP_EQUAL: return "(" + a + " == " + b + ")";
      case VBE_OP_NOT_EQUAL: return "(" + a + " != " + b + ")";
      case VBE_OP_SELECT: return "(" + a + " ? " + b + " : " + d + ")";
      case VBE_OP_CAST:
        if (s.dt_out == VBE_BOOL) return "(" + a + " != 0)";
        return "((" + std::string(ctype(s.dt_out)) + ")" + a + ")";
      case VBE_OP_COPY: return a;
      case VBE_OP_RANDOM: {
        int w = L.rnd[s.random_idx];
        return std::string(r.soft_f64 ? "vbe_u01s" : "vbe_u01") + "((u64)p.w[" + std::to_string(w) +
               "], (u64)p.w[" + std::to_string(w + 1) + "], (u64)p.w[" + std::to_string(w + 2) + "], (u64)m)";
      }
    }
    fail(VBE_ERR_INVALID, "codegen: unsupported opcode");
  }

  std::string red_id() {
    int dt = arg() ? r.value_dtype[r.red_value] : r.red_dtype;
    switch (arg() ? (argmax() ? VBE_OP_MAX_REDUCE : VBE_OP_MIN_REDUCE) : r.red_op) {
      case VBE_OP_ADD_REDUCE: return dt == VBE_INT64 ? "((i64)0)" : (dt == VBE_FLOAT32 ? "0.0f" : "0.0");
      case VBE_OP_MIN_REDUCE:
        return dt == VBE_INT64 ? "((i64)0x7fffffffffffffffll)"
                               : (dt == VBE_FLOAT32 ? "__int_as_float(0x7f800000)"
                                                    : "__longlong_as_double(0x7ff0000000000000ll)");
      case VBE_OP_MAX_REDUCE:
        return dt == VBE_INT64 ? "((i64)0x8000000000000000ull)"
                               : (dt == VBE_FLOAT32 ? "__int_as_float(0xff800000)"
                                                    : "__longlong_as_double(0xfff0000000000000ll)");
    }
    return "0";
  }

  std::string comb(const std::string& a, const std::string& b) {
    switch (r.red_op) {
      case VBE_OP_ADD_REDUCE:
        return r.red_dtype == VBE_INT64 ? "vbe_iadd(" + a + "," + b + ")" : "(" + a + " + " + b + ")";
      case VBE_OP_MIN_REDUCE: return "vbe_min(" + a + "," + b + ")";
      case VBE_OP_MAX_REDUCE: return "vbe_max(" + a + "," + b + ")";
    }
    return a;
  }

  // the per-element function: loaded values in, values to store out
  std::string elem_name = "vbe_elem";
  std::string block_reduce_name = "vbe_block_reduce";
  bool emit_struct = true;
  bool guard_div = false;  // zero-numerator guard on native divisions
  void emit_elem() {
    if (emit_struct) o << "struct P { i64 w[" << L.nwords << "]; };\n";
    o << "__device__ __forceinline__ void " << elem_name << "(const P& p, i64 m";
    for (size_t s = 0; s < r.loads.size(); ++s) o << ", const " << ctype(r.loads[s].dtype) << " l" << s;
    for (size_t s = 0; s < r.stores.size(); ++s) o << ", " << ctype(r.stores[s].dtype) << "& o" << s;
    if (arg()) {
      o << ", " << vt() << "& acc, i64& acci, const i64 ai";
      if (r.has_red2) o << ", " << rt() << "& accm";
    } else if (r.has_red) {
      o << ", " << rt() << "& acc";
      if (kahan()) o << ", float& kc";
    }
    if (const_params)
      for (size_t k = 0; k < r.consts.size(); ++k) o << ", const " << ctype(r.consts[k].dtype) << " kc" << k;
    o << ") {\n  (void)m; (void)p;\n";
    for (auto& s : r.steps) o << "  const " << ctype(s.dt_out) << " v" << s.value << " = " << expr(s) << ";\n";
    for (size_t s = 0; s < r.stores.size(); ++s) o << "  o" << s << " = v" << r.store_value[s] << ";\n";
    if (r.has_red) {
      std::string x = "v" + std::to_string(r.red_value);
      if (arg()) {
        o << "  vbe_arg_upd(acc, acci, " << x << ", ai, " << (argmax() ? "true" : "false") << ");\n";
        // the paired MIN/MAX keeps its own value, combined as a lone one is
        if (r.has_red2) o << "  accm = " << comb("accm", x) << ";\n";
      } else if (kahan()) {
        o << "  { const float y = " << x << " - kc; const float t = acc + y; kc = (t - acc) - y; acc = t; }\n";
      } else {
        o << "  acc = " << comb("acc", x) << ";\n";
      }
    }
    o << "}\n";
  }

  void emit_block_reduce() {
    if (!r.has_red) return;
    if (arg()) {
      // (value, index) pairs: warp shuffles of both, then one warp over the
      // warps' pairs; returns the index of the block's best pair
      const std::string V = vt(), mx = argmax() ? "true" : "false";
      o << "__device__ __forceinline__ i64 " << block_reduce_name << "(" << V << " v, i64 i, " << V << "& vout) {\n"
        << "  __shared__ " << V << " shv[32];\n  __shared__ i64 shi[32];\n"
        << "  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;\n"
        << "  for (int off = 16; off > 0; off >>= 1) { const " << V
        << " tv = __shfl_down_sync(0xffffffffu, v, off); const i64 ti = __shfl_down_sync(0xffffffffu, i, off);"
        << " vbe_arg_upd(v, i, tv, ti, " << mx << "); }\n"
        << "  if (lane == 0) { shv[wid] = v; shi[wid] = i; }\n  __syncthreads();\n"
        << "  if (wid == 0) {\n    v = lane < nw ? shv[lane] : " << red_id() << ";\n"
        << "    i = lane < nw ? shi[lane] : (i64)0x7fffffffffffffffll;\n"
        << "    for (int off = 16; off > 0; off >>= 1) { const " << V
        << " tv = __shfl_down_sync(0xffffffffu, v, off); const i64 ti = __shfl_down_sync(0xffffffffu, i, off);"
        << " vbe_arg_upd(v, i, tv, ti, " << mx << "); }\n  }\n"
        << "  if (threadIdx.x == 0) vout = v;\n"
        << "  __syncthreads();\n  return i;\n}\n";
      if (!r.has_red2) return;
    }
    o << "__device__ __forceinline__ " << rt() << " " << block_reduce_name << (arg() ? "_v" : "") << "(" << rt()
      << " v) {\n"
      << "  __shared__ " << rt() << " sh[32];\n"
      << "  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;\n"
      << "  for (int off = 16; off > 0; off >>= 1) { " << rt() << " t = __shfl_down_sync(0xffffffffu, v, off); v = "
      << comb("v", "t") << "; }\n"
      << "  if (lane == 0) sh[wid] = v;\n  __syncthreads();\n"
      << "  if (wid == 0) {\n    v = lane < nw ? sh[lane] : " << red_id() << ";\n"
      << "    for (int off = 16; off > 0; off >>= 1) { " << rt()
      << " t = __shfl_down_sync(0xffffffffu, v, off); v = " << comb("v", "t") << "; }\n  }\n"
      << "  __syncthreads();\n  return v;\n}\n";
  }

  std::string T(int dt) { return ctype(dt); }
  std::string W(int k) { return "p.w[" + std::to_string(k) + "]"; }

  // argument list for vbe_elem given per-slot value expressions
  std::string call(const std::string& m, const std::vector<std::string>& lv, const std::vector<std::string>& sv,
                   const std::string& ai = "ri") {
    std::string s = (plain_sum ? "vbe_elem_p(p, " : "vbe_elem(p, ") + m;
    for (auto& x : lv) s += ", " + x;
    for (auto& x : sv) s += ", " + x;
    if (arg()) s += ", acc, acci, " + ai + (r.has_red2 ? ", accm" : "");
    else if (r.has_red) s += kahan() ? ", acc, kc" : ", acc";
    return s + ");";
  }

  void emit_pointers(const std::string& pfx) {
    for (size_t s = 0; s < r.loads.size(); ++s)
      o << pfx << "const auto lp" << s << " = vbe_ptr<const " << T(r.loads[s].dtype) << ">(" << W(L.lptr[s])
        << ");\n";
    for (size_t s = 0; s < r.stores.size(); ++s)
      o << pfx << "const auto sp" << s << " = vbe_ptr<" << T(r.stores[s].dtype) << ">(" << W(L.sptr[s]) << ");\n";
  }

  void emit_acc_init(const std::string& pfx) {
    if (!r.has_red) return;
    if (arg()) {
      o << pfx << vt() << " acc = " << red_id() << ";\n" << pfx << "i64 acci = (i64)0x7fffffffffffffffll;\n";
      if (r.has_red2) o << pfx << rt() << " accm = " << red_id() << ";\n";
      return;
    }
    o << pfx << rt() << " acc = " << red_id() << ";\n";
    if (kahan()) o << pfx << "float kc = 0.0f;\n";
  }

  std::string acc_final() { return kahan() ? "(acc - kc)" : "acc"; }

  // full-reduction epilogue: block partial, last block sums partials
  void emit_full_epilogue(const std::string& pfx, const std::string& part, const std::string& slot,
                          const std::string& count, const std::string& nparts, const std::string& out) {
    o << pfx << "{\n"
      << pfx << "  " << rt() << " bsum = " << block_reduce_name << "(" << acc_final() << ");\n"
      << pfx << "  __shared__ int s_last;\n"
      << pfx << "  if (threadIdx.x == 0) {\n"
      << pfx << "    vbe_ptr<" << rt() << ">(" << part << ")[" << slot << "] = bsum;\n"
      << pfx << "    __threadfence();\n"
      << pfx << "    unsigned prev = atomicAdd(vbe_ptr<unsigned>(" << count << "), 1u);\n"
      << pfx << "    s_last = (prev == (unsigned)(" << nparts << ") - 1u);\n"
      << pfx << "  }\n"
      << pfx << "  __syncthreads();\n"
      << pfx << "  if (s_last) {\n"
      << pfx << "    __threadfence();\n"
      << pfx << "    " << rt() << " v = " << red_id() << ";\n"
      << pfx << "    const auto pp = vbe_ptr<const volatile " << rt() << ">(" << part << ");\n"
      << pfx << "    for (i64 i = threadIdx.x; i < (i64)(" << nparts << "); i += blockDim.x) { " << rt()
      << " x = pp[i]; v = " << comb("v", "x") << "; }\n"
      << pfx << "    v = " << block_reduce_name << "(v);\n"
      << pfx << "    if (threadIdx.x == 0) { vbe_ptr<" << rt() << ">(" << out << ")[0] = v; vbe_ptr<unsigned>(" << count
      << ")[0] = 0u; }\n"
      << pfx << "  }\n"
      << pfx << "}\n";
  }

  // --------------------------------------------------------- tile kernels
  void emit_tile_kernel(int U, int maxreg = 0) {
    const int nd = c.spec.nd;
    o << "extern \"C\" __global__ void "
      << (maxreg ? "__maxnreg__(" + std::to_string(maxreg) + ")" : std::string("__launch_bounds__(1024)")) << " vbe_@TAG@_u"
      << U << (maxreg ? "r" + std::to_string(maxreg) : std::string()) << "(const P p) {\n"
      << "  vbe_grid_wait();\n";
    emit_pointers("  ");
    emit_acc_init("  ");
    // inner strides
    for (size_t s = 0; s < r.loads.size(); ++s)
      if (c.spec.load_cls[s] == 2) o << "  const i64 li" << s << " = " << W(L.lst[s] + nd - 1) << ";\n";
    for (size_t s = 0; s < r.stores.size(); ++s)
      if (c.spec.store_cls[s] == 2) o << "  const i64 si" << s << " = " << W(L.sst[s] + nd - 1) << ";\n";
    if (c.spec.vec) {
      emit_vec_body(U);
    } else {
      o << "  const i64 inner = " << W(L.inner) << ";\n"
        << "  const i64 bsu = (i64)blockDim.x * " << U << ";\n"
        << "  const i64 tpr = (inner + bsu - 1) / bsu;\n"
        << "  const i64 ntiles = " << W(L.nouter) << " * tpr;\n"
        << "  i64 t = blockIdx.x;\n"
        << "  i64 row = tpr ? t / tpr : 0, ct = t - row * tpr;\n"
        << "  const i64 rstep = tpr ? (i64)gridDim.x / tpr : 0, cstep = (i64)gridDim.x - rstep * tpr;\n"
        << "  for (; t < ntiles; t += gridDim.x) {\n";
      // row offsets
      auto rowoff = [&](const std::string& name, int stw) {
        if (nd == 1) {
          o << "    const i64 " << name << " = 0;\n";
        } else if (nd == 2) {
          o << "    const i64 " << name << " = row * " << W(stw) << ";\n";
        } else {
          o << "    i64 " << name << " = 0;\n    { i64 rr = row;\n";
          for (int k = nd - 2; k >= 0; --k)
            o << "      { const i64 ik = rr % " << W(L.dims0 + k) << "; rr /= " << W(L.dims0 + k) << "; " << name
              << " += ik * " << W(stw + k) << "; }\n";
          o << "    }\n";
        }
      };
      for (size_t s = 0; s < r.loads.size(); ++s) rowoff("lr" + std::to_string(s), L.lst[s]);
      for (size_t s = 0; s < r.stores.size(); ++s) rowoff("sr" + std::to_string(s), L.sst[s]);
      o << "    const i64 c0 = ct * bsu + threadIdx.x;\n";
      auto laddr = [&](size_t s, const std::string& col) {
        int cl = c.spec.load_cls[s];
        std::string b = "lr" + std::to_string(s);
        if (cl == 0) return "lp" + std::to_string(s) + "[" + b + "]";
        if (cl == 1) return "lp" + std::to_string(s) + "[" + b + " + " + col + "]";
        return "lp" + std::to_string(s) + "[" + b + " + " + col + " * li" + std::to_string(s) + "]";
      };
      auto saddr = [&](size_t s, const std::string& col) {
        int cl = c.spec.store_cls[s];
        std::string b = "sr" + std::to_string(s);
        if (cl == 0) return "sp" + std::to_string(s) + "[" + b + "]";
        if (cl == 1) return "sp" + std::to_string(s) + "[" + b + " + " + col + "]";
        return "sp" + std::to_string(s) + "[" + b + " + " + col + " * si" + std::to_string(s) + "]";
      };
      // full tile: all loads first
      o << "    if (ct * bsu + bsu <= inner) {\n";
      for (size_t s = 0; s < r.loads.size(); ++s) o << "      " << T(r.loads[s].dtype) << " a" << s << "[" << U << "];\n";
      for (size_t s = 0; s < r.stores.size(); ++s) o << "      " << T(r.stores[s].dtype) << " b" << s << "[" << U << "];\n";
      o << "#pragma unroll\n      for (int u = 0; u < " << U << "; ++u) {\n        const i64 col = c0 + (i64)u * blockDim.x;\n";
      for (size_t s = 0; s < r.loads.size(); ++s) o << "        a" << s << "[u] = " << laddr(s, "col") << ";\n";
      o << "      }\n#pragma unroll\n      for (int u = 0; u < " << U << "; ++u) {\n        const i64 col = c0 + (i64)u * blockDim.x;\n        (void)col;\n";
      {
        std::vector<std::string> lv, sv;
        for (size_t s = 0; s < r.loads.size(); ++s) lv.push_back("a" + std::to_string(s) + "[u]");
        for (size_t s = 0; s < r.stores.size(); ++s) sv.push_back("b" + std::to_string(s) + "[u]");
        o << "        " << call("row * inner + col", lv, sv) << "\n";
      }
      o << "      }\n#pragma unroll\n      for (int u = 0; u < " << U << "; ++u) {\n        const i64 col = c0 + (i64)u * blockDim.x;\n        (void)col;\n";
      for (size_t s = 0; s < r.stores.size(); ++s) o << "        " << saddr(s, "col") << " = b" << s << "[u];\n";
      o << "      }\n    } else {\n";
      o << "#pragma unroll\n      for (int u = 0; u < " << U << "; ++u) {\n        const i64 col = c0 + (i64)u * blockDim.x;\n        if (col < inner) {\n";
      {
        std::vector<std::string> lv, sv;
        for (size_t s = 0; s < r.loads.size(); ++s) lv.push_back(laddr(s, "col"));
        for (size_t s = 0; s < r.stores.size(); ++s) {
          o << "          " << T(r.stores[s].dtype) << " b" << s << ";\n";
          sv.push_back("b" + std::to_string(s));
        }
        o << "          " << call("row * inner + col", lv, sv) << "\n";
        for (size_t s = 0; s < r.stores.size(); ++s) o << "          " << saddr(s, "col") << " = b" << s << ";\n";
      }
      o << "        }\n      }\n    }\n";
      o << "    ct += cstep; row += rstep; if (ct >= tpr) { ct -= tpr; ++row; }\n  }\n";
    }
    if (c.spec.mode == Mode::FULL)
      emit_full_epilogue("  ", W(L.partials), "blockIdx.x", W(L.counter), "gridDim.x", W(L.red_ptr));
    o << "}\n";
  }

  int bulk_slots() const {
    int k = 0;
    for (size_t s = 0; s < r.loads.size(); ++s)
      if (c.spec.load_cls[s] == 1) ++k;
    return k;
  }

  // One-dimensional vector run with its unit-stride inputs staged through
  // shared memory by bulk asynchronous copies: chunks of CH elements, two
  // stages per CTA, thread 0 issues the copies of the next chunk while the
  // block computes on the current one; the tail (n mod CH) and broadcast
  // inputs use plain loads.
  void emit_bulk_kernel() {
    const int E = c.spec.E;
    o << "extern \"C\" __global__ void __launch_bounds__(1024) vbe_@TAG@_bulk(const P p) {\n"
      << "  VBE_DYN_SMEM;\n  vbe_grid_wait();\n";
    emit_pointers("  ");
    emit_acc_init("  ");
    o << "  const i64 n = " << W(L.inner) << ", CH = " << W(L.bulk_ch) << ";\n"
      << "  const i64 nfull = n / CH;\n"
      << "  const i64 bd = blockDim.x;\n";
    // stage layout: per stage the unit-stride slots' chunks, back to back
    std::string stage_bytes = "(";
    std::vector<std::string> off;
    std::string acc = "0";
    for (size_t s = 0; s < r.loads.size(); ++s) {
      if (c.spec.load_cls[s] != 1) {
        off.push_back("");
        continue;
      }
      off.push_back(acc);
      acc += " + CH * " + std::to_string(itemsize(r.loads[s].dtype));
    }
    stage_bytes += acc + ")";
    o << "  const i64 SB = " << stage_bytes << ";\n"
      << "  unsigned long long* bars = (unsigned long long*)(vbe_smem + 2 * SB);\n"
      << "  __shared__ int s_ok;\n";
    for (size_t s = 0; s < r.loads.size(); ++s)
      if (c.spec.load_cls[s] == 0) o << "  const " << T(r.loads[s].dtype) << " z" << s << " = lp" << s << "[0];\n";
    o << "  if (threadIdx.x == 0) { vbe_mbar_init(&bars[0], 1); vbe_mbar_init(&bars[1], 1); vbe_fence_mbar_init(); }\n"
      << "  __syncthreads();\n";
    auto issue = [&](const std::string& pfx, const std::string& chunk, const std::string& stage) {
      o << pfx << "{ const i64 ic = " << chunk << "; const int is = " << stage << ";\n"
        << pfx << "  vbe_mbar_expect_tx(&bars[is], (unsigned)SB);\n";
      for (size_t s = 0; s < r.loads.size(); ++s)
        if (c.spec.load_cls[s] == 1)
          o << pfx << "  vbe_bulk_g2s(vbe_smem + is * SB + " << off[s] << ", &lp" << s << "[ic * CH], (unsigned)(CH * "
            << itemsize(r.loads[s].dtype) << "), &bars[is]);\n";
      o << pfx << "}\n";
    };
    o << "  unsigned inflight = 0;\n"
      << "  if (threadIdx.x == 0) {\n";
    o << "    if ((i64)blockIdx.x < nfull) {";
    issue("      ", "(i64)blockIdx.x", "0");
    o << "      inflight |= 1; }\n";
    o << "    if ((i64)blockIdx.x + gridDim.x < nfull) {";
    issue("      ", "(i64)blockIdx.x + gridDim.x", "1");
    o << "      inflight |= 2; }\n  }\n";
    o << "  bool failed = false;\n"
      << "  int k = 0;\n"
      << "  for (i64 cc = blockIdx.x; cc < nfull; cc += gridDim.x, ++k) {\n"
      << "    const int st = k & 1;\n"
      << "    if (threadIdx.x == 0) { s_ok = vbe_mbar_wait_n(&bars[st], (unsigned)((k >> 1) & 1), VBE_CWAIT); if (s_ok) inflight &= ~(1u << st); }\n"
      << "    __syncthreads();\n"
      << "    if (!s_ok) { failed = true; break; }\n"
      << "    for (i64 vi = threadIdx.x; vi < CH / " << E << "; vi += bd) {\n";
    for (size_t s = 0; s < r.loads.size(); ++s)
      if (c.spec.load_cls[s] == 1)
        o << "      " << T(r.loads[s].dtype) << " a" << s << "[" << E << "];\n"
          << "      vbe_vload((const " << T(r.loads[s].dtype) << "*)(vbe_smem + st * SB + " << off[s] << ") + vi * " << E
          << ", a" << s << ");\n";
    for (size_t s = 0; s < r.stores.size(); ++s) o << "      " << T(r.stores[s].dtype) << " b" << s << "[" << E << "];\n";
    o << "#pragma unroll\n      for (int e = 0; e < " << E << "; ++e) {\n";
    {
      std::vector<std::string> lv, sv;
      for (size_t s = 0; s < r.loads.size(); ++s)
        lv.push_back(c.spec.load_cls[s] == 1 ? "a" + std::to_string(s) + "[e]" : "z" + std::to_string(s));
      for (size_t s = 0; s < r.stores.size(); ++s) sv.push_back("b" + std::to_string(s) + "[e]");
      o << "        " << call("cc * CH + vi * " + std::to_string(E) + " + e", lv, sv) << "\n";
    }
    o << "      }\n";
    for (size_t s = 0; s < r.stores.size(); ++s)
      o << "      vbe_vstore(sp" << s << " + cc * CH + vi * " << E << ", b" << s << ");\n";
    o << "    }\n"
      << "    __syncthreads();\n"
      << "    if (threadIdx.x == 0 && cc + 2 * (i64)gridDim.x < nfull) {\n"
      << "      vbe_fence_proxy_async();\n";
    issue("      ", "cc + 2 * (i64)gridDim.x", "st");
    o << "      inflight |= 1u << st;\n    }\n  }\n";
    // on a failed wait: report (the error word is mapped host memory),
    // drain the copies still in flight (bounded) and skip the rest; a full
    // reduction still takes part in the grid's final combine so that its
    // completion counter stays consistent
    o << "  if (failed) {\n"
      << "    if (threadIdx.x == 0) {\n"
      << "      vbe_ptr<volatile unsigned>(" << W(L.err) << ")[0] = 1u;\n"
      << "      for (int st = 0; st < 2; ++st)\n"
      << "        if (inflight & (1u << st)) vbe_mbar_wait(&bars[st], (unsigned)(((k + ((st - k) & 1)) >> 1) & 1));\n"
      << "    }\n"
      << "  } else\n";
    // tail with plain loads
    o << "  for (i64 e = nfull * CH + (i64)blockIdx.x * bd + threadIdx.x; e < n; e += (i64)gridDim.x * bd) {\n";
    {
      std::vector<std::string> lv, sv;
      for (size_t s = 0; s < r.loads.size(); ++s)
        lv.push_back(c.spec.load_cls[s] == 1 ? "lp" + std::to_string(s) + "[e]" : "z" + std::to_string(s));
      for (size_t s = 0; s < r.stores.size(); ++s) {
        o << "    " << T(r.stores[s].dtype) << " b" << s << ";\n";
        sv.push_back("b" + std::to_string(s));
      }
      o << "    " << call("e", lv, sv) << "\n";
      for (size_t s = 0; s < r.stores.size(); ++s) o << "    sp" << s << "[e] = b" << s << ";\n";
    }
    o << "  }\n";
    if (c.spec.mode == Mode::FULL)
      emit_full_epilogue("  ", W(L.partials), "blockIdx.x", W(L.counter), "gridDim.x", W(L.red_ptr));
    o << "}\n";
  }

  void emit_vec_body(int U) {
    const int E = c.spec.E;
    o << "  const i64 n = " << W(L.inner) << ";\n"
      << "  const i64 nvec = n / " << E << ";\n"
      << "  const i64 bd = blockDim.x;\n";
    // broadcast (stride-0) loads are read once
    for (size_t s = 0; s < r.loads.size(); ++s)
      if (c.spec.load_cls[s] == 0) o << "  const " << T(r.loads[s].dtype) << " z" << s << " = lp" << s << "[0];\n";
    o << "  for (i64 v0 = (i64)blockIdx.x * bd * " << U << "; v0 < nvec; v0 += (i64)gridDim.x * bd * " << U << ") {\n";
    auto body = [&](const std::string& pfx, bool guard) {
      for (size_t s = 0; s < r.loads.size(); ++s)
        if (c.spec.load_cls[s] == 1)
          o << pfx << T(r.loads[s].dtype) << " a" << s << "[" << (guard ? 1 : U) << "][" << E << "];\n";
      for (size_t s = 0; s < r.stores.size(); ++s)
        o << pfx << T(r.stores[s].dtype) << " b" << s << "[" << (guard ? 1 : U) << "][" << E << "];\n";
      int UU = guard ? 1 : U;
      std::string uidx = guard ? "0" : "u";
      if (!guard) o << "#pragma unroll\n";
      o << pfx << "for (int u = 0; u < " << UU << "; ++u) {\n";
      o << pfx << "  const i64 vi = " << (guard ? "vg" : "v0 + (i64)u * bd + threadIdx.x") << ";\n";
      for (size_t s = 0; s < r.loads.size(); ++s)
        if (c.spec.load_cls[s] == 1) o << pfx << "  vbe_vload(lp" << s << " + vi * " << E << ", a" << s << "[u]);\n";
      o << pfx << "}\n";
      if (!guard) o << "#pragma unroll\n";
      o << pfx << "for (int u = 0; u < " << UU << "; ++u) {\n";
      o << pfx << "  const i64 vi = " << (guard ? "vg" : "v0 + (i64)u * bd + threadIdx.x") << ";\n  (void)vi;\n";
      o << "#pragma unroll\n" << pfx << "  for (int e = 0; e < " << E << "; ++e) {\n";
      std::vector<std::string> lv, sv;
      for (size_t s = 0; s < r.loads.size(); ++s)
        lv.push_back(c.spec.load_cls[s] == 1 ? "a" + std::to_string(s) + "[u][e]" : "z" + std::to_string(s));
      for (size_t s = 0; s < r.stores.size(); ++s) sv.push_back("b" + std::to_string(s) + "[u][e]");
      o << pfx << "    " << call("vi * " + std::to_string(E) + " + e", lv, sv) << "\n";
      o << pfx << "  }\n";
      for (size_t s = 0; s < r.stores.size(); ++s) o << pfx << "  vbe_vstore(sp" << s << " + vi * " << E << ", b" << s << "[u]);\n";
      o << pfx << "}\n";
      (void)uidx;
    };
    o << "    if (v0 + bd * " << U << " <= nvec) {\n";
    body("      ", false);
    o << "    } else {\n"
      << "      for (int uu = 0; uu < " << U << "; ++uu) {\n"
      << "        const i64 vg = v0 + (i64)uu * bd + threadIdx.x;\n"
      << "        if (vg < nvec) {\n";
    body("          ", true);
    o << "        }\n      }\n    }\n  }\n";
    // scalar tail
    o << "  for (i64 e = nvec * " << E << " + (i64)blockIdx.x * bd + threadIdx.x; e < n; e += (i64)gridDim.x * bd) {\n";
    std::vector<std::string> lv, sv;
    for (size_t s = 0; s < r.loads.size(); ++s)
      lv.push_back(c.spec.load_cls[s] == 1 ? "lp" + std::to_string(s) + "[e]" : "z" + std::to_string(s));
    for (size_t s = 0; s < r.stores.size(); ++s) {
      o << "    " << T(r.stores[s].dtype) << " b" << s << ";\n";
      sv.push_back("b" + std::to_string(s));
    }
    o << "    " << call("e", lv, sv) << "\n";
    for (size_t s = 0; s < r.stores.size(); ++s) o << "    sp" << s << "[e] = b" << s << ";\n";
    o << "  }\n";
  }

  // ---------------------------------------------------- packed 1-D kernel
  void emit_packed_kernel(int U) {
    o << "extern \"C\" __global__ void __launch_bounds__(1024) vbe_@TAG@_pack_u" << U
      << "(const P* __restrict__ descs, const i64* __restrict__ prefix, int ninst, i64 total, i64 chunk, unsigned* work) {\n"
      << "  vbe_grid_wait();\n"
      << "  __shared__ i64 s_c;\n"
      << "  for (;;) {\n"
      << "    if (threadIdx.x == 0) s_c = (i64)atomicAdd(work, 1u);\n"
      << "    __syncthreads();\n"
      << "    const i64 cidx = s_c;\n"
      << "    __syncthreads();\n"
      << "    if (cidx >= total) break;\n"
      << "    int lo = 0, hi = ninst;\n"
      << "    while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (prefix[mid] <= cidx) lo = mid; else hi = mid; }\n"
      << "    const P& p = descs[lo];\n"
      << "    const i64 lc = cidx - prefix[lo];\n"
      << "    const i64 n = " << W(L.inner) << ";\n"
      << "    const i64 e0 = lc * chunk, e1 = min(n, e0 + chunk);\n";
    emit_pointers("    ");
    emit_acc_init("    ");
    for (size_t s = 0; s < r.loads.size(); ++s)
      if (c.spec.load_cls[s] == 2) o << "    const i64 li" << s << " = " << W(L.lst[s]) << ";\n";
    for (size_t s = 0; s < r.stores.size(); ++s)
      if (c.spec.store_cls[s] == 2) o << "    const i64 si" << s << " = " << W(L.sst[s]) << ";\n";
    o << "    for (i64 eb = e0 + threadIdx.x; eb < e1; eb += (i64)blockDim.x * " << U << ") {\n"
      << "#pragma unroll\n      for (int u = 0; u < " << U << "; ++u) {\n"
      << "        const i64 e = eb + (i64)u * blockDim.x;\n"
      << "        if (e < e1) {\n";
    std::vector<std::string> lv, sv;
    for (size_t s = 0; s < r.loads.size(); ++s) {
      int cl = c.spec.load_cls[s];
      lv.push_back("lp" + std::to_string(s) + (cl == 0 ? "[0]" : (cl == 1 ? "[e]" : "[e * li" + std::to_string(s) + "]")));
    }
    for (size_t s = 0; s < r.stores.size(); ++s) {
      o << "          " << T(r.stores[s].dtype) << " b" << s << ";\n";
      sv.push_back("b" + std::to_string(s));
    }
    o << "          " << call("e", lv, sv) << "\n";
    for (size_t s = 0; s < r.stores.size(); ++s) {
      int cl = c.spec.store_cls[s];
      o << "          sp" << s << (cl == 0 ? "[0]" : (cl == 1 ? "[e]" : "[e * si" + std::to_string(s) + "]")) << " = b"
        << s << ";\n";
    }
    o << "        }\n      }\n    }\n";
    if (r.has_red) {
      o << "    const i64 nch = n > 0 ? (n + chunk - 1) / chunk : 1;\n";
      emit_full_epilogue("    ", W(L.partials), "lc", W(L.counter), "nch", W(L.red_ptr));
    }
    o << "  }\n}\n";
  }

  // ------------------------------------------------------- axis kernels
  void emit_axis_kernel() {
    const int ndk = c.spec.ndk, ndr = c.spec.ndr;
    bool block = c.spec.mode == Mode::AXIS_BLOCK;
    o << "extern \"C\" __global__ void __launch_bounds__(1024) vbe_@TAG@_axis(const P p) {\n"
      << "  vbe_grid_wait();\n";
    emit_pointers("  ");
    if (r.has_red2) o << "  const auto rp2 = vbe_ptr<i64>(" << W(L.red2_ptr) << ");\n";
    o << "  const auto rp = vbe_ptr<" << rt() << ">(" << W(L.red_ptr) << ");\n"
      << "  const i64 nout = " << W(L.nout) << ", nred = " << W(L.nred) << ";\n";
    if (block)
      o << "  for (i64 oi = blockIdx.x; oi < nout; oi += gridDim.x) {\n";
    else
      o << "  for (i64 oi = (i64)blockIdx.x * blockDim.x + threadIdx.x; oi < nout; oi += (i64)gridDim.x * blockDim.x) {\n";
    // kept offsets
    std::vector<std::pair<std::string, int>> ks;  // name, first stride word
    for (size_t s = 0; s < r.loads.size(); ++s) ks.push_back({"lk" + std::to_string(s), L.lst[s]});
    for (size_t s = 0; s < r.stores.size(); ++s) ks.push_back({"sk" + std::to_string(s), L.sst[s]});
    ks.push_back({"rk", L.red_st});
    if (r.has_red2) ks.push_back({"rk2", L.red2_st});
    if (L.idx_st >= 0) ks.push_back({"ik", L.idx_st});
    for (auto& k : ks) o << "    i64 " << k.first << " = 0;\n";
    o << "    { i64 rr = oi;\n";
    for (int k = ndk - 1; k >= 0; --k) {
      o << "      { const i64 ix = rr % " << W(L.dims0 + k) << "; rr /= " << W(L.dims0 + k) << ";";
      for (auto& kk : ks) o << " " << kk.first << " += ix * " << W(kk.second + k) << ";";
      o << " }\n";
    }
    o << "    }\n";
    emit_acc_init("    ");
    auto emit_loops = [&]() {
    // reduced offsets of element ri + u * rs (names suffixed by u)
    std::vector<std::pair<std::string, int>> rs;
    for (size_t s = 0; s < r.loads.size(); ++s) rs.push_back({"lr" + std::to_string(s), L.lst[s] + ndk});
    for (size_t s = 0; s < r.stores.size(); ++s) rs.push_back({"sr" + std::to_string(s), L.sst[s] + ndk});
    if (L.idx_st >= 0) rs.push_back({"ir", L.idx_st + ndk});
    auto offsets = [&](const std::string& ind, const std::string& u, const std::string& rix) {
      for (auto& k : rs) o << ind << "i64 " << k.first << u << " = 0;\n";
      if (ndr == 1) {
        for (auto& k : rs) o << ind << k.first << u << " = (" << rix << ") * " << W(k.second) << ";\n";
      } else {
        o << ind << "{ i64 rr = " << rix << ";\n";
        for (int k = ndr - 1; k >= 0; --k) {
          o << ind << "  { const i64 ix = rr % " << W(L.dims0 + ndk + k) << "; rr /= " << W(L.dims0 + ndk + k) << ";";
          for (auto& kk : rs) o << " " << kk.first << u << " += ix * " << W(kk.second + k) << ";";
          o << " }\n";
        }
        o << ind << "}\n";
      }
    };
    // element u of this step: its loads (preloaded values), then the call and its stores
    auto element = [&](const std::string& ind, const std::string& u, const std::string& rix, bool preloaded) {
      std::vector<std::string> lv, sv;
      for (size_t s = 0; s < r.loads.size(); ++s)
        lv.push_back(preloaded ? "la" + std::to_string(s) + u
                               : "lp" + std::to_string(s) + "[lk" + std::to_string(s) + " + lr" + std::to_string(s) + u + "]");
      for (size_t s = 0; s < r.stores.size(); ++s) {
        o << ind << T(r.stores[s].dtype) << " b" << s << u << ";\n";
        sv.push_back("b" + std::to_string(s) + u);
      }
      o << ind << call(L.idx_st >= 0 ? "ik + ir" + u : "0", lv, sv, rix) << "\n";
      for (size_t s = 0; s < r.stores.size(); ++s)
        o << ind << "sp" << s << "[sk" << s << " + sr" << s << u << "] = b" << s << u << ";\n";
    };
    // A thread takes the reduced elements ri, ri + rs, ri + 2 rs, ... in
    // order. Four at a time, their loads issued before the first of them is
    // combined (a store of one element never touches another element's
    // inputs: the run's views are disjoint or identical), so four loads are
    // in flight instead of one; the combining order is unchanged.
    // Outputs whose reduced dimension is a contiguous, 16-byte aligned row
    // of every input and output: 16-byte vector loads (and stores) of E
    // consecutive elements. A thread takes chunks c, c + rs, ... (rs = 1 for
    // a thread per output, blockDim for a block per output), two chunks in
    // flight, then the elements past the last whole chunk one by one; a
    // thread per output thus still combines its elements in order. Decided
    // per output at run time (strides, alignment); otherwise the scalar
    // loop below.
    int visz = r.loads.empty() ? 0 : itemsize(r.loads[0].dtype);
    for (auto& l : r.loads)
      if (itemsize(l.dtype) != visz) visz = 0;
    for (auto& st : r.stores)
      if (itemsize(st.dtype) != visz) visz = 0;
    const bool vec_gen = ndr == 1 && (visz == 4 || visz == 8);
    if (vec_gen) {
      const int E = 16 / visz;
      const std::string E_ = std::to_string(E);
      o << "    bool vec = true;\n";
      for (size_t s = 0; s < r.loads.size(); ++s)
        o << "    vec = vec && " << W(L.lst[s] + ndk) << " == 1 && vbe_aligned16(lp" << s << " + lk" << s << ");\n";
      for (size_t s = 0; s < r.stores.size(); ++s)
        o << "    vec = vec && " << W(L.sst[s] + ndk) << " == 1 && vbe_aligned16(sp" << s << " + sk" << s << ");\n";
      o << "    if (vec) {\n"
        << "      const i64 cs = " << (block ? "(i64)blockDim.x" : "(i64)1") << ", nv = nred / " << E << ";\n"
        << "      i64 ci = " << (block ? "(i64)threadIdx.x" : "(i64)0") << ";\n";
      auto chunks = [&](int nu, const std::string& ind) {
        for (int u = 0; u < nu; ++u) {
          const std::string us = std::to_string(u), base = "(ci + " + us + " * cs) * " + E_;
          for (size_t s = 0; s < r.loads.size(); ++s)
            o << ind << T(r.loads[s].dtype) << " lq" << s << "_" << us << "[" << E << "];\n"
              << ind << "vbe_vload(lp" << s << " + (lk" << s << " + " << base << "), lq" << s << "_" << us << ");\n";
        }
        for (int u = 0; u < nu; ++u) {
          const std::string us = std::to_string(u), base = "(ci + " + us + " * cs) * " + E_;
          for (size_t s = 0; s < r.stores.size(); ++s)
            o << ind << T(r.stores[s].dtype) << " bq" << s << "_" << us << "[" << E << "];\n";
          for (int e = 0; e < E; ++e) {
            std::vector<std::string> lv, sv;
            const std::string es = std::to_string(e);
            for (size_t s = 0; s < r.loads.size(); ++s) lv.push_back("lq" + std::to_string(s) + "_" + us + "[" + es + "]");
            for (size_t s = 0; s < r.stores.size(); ++s) sv.push_back("bq" + std::to_string(s) + "_" + us + "[" + es + "]");
            const std::string rix = base + " + " + es;
            const std::string m = L.idx_st >= 0 ? "ik + (" + rix + ") * " + W(L.idx_st + ndk) : "0";
            o << ind << call(m, lv, sv, rix) << "\n";
          }
          for (size_t s = 0; s < r.stores.size(); ++s)
            o << ind << "vbe_vstore(sp" << s << " + (sk" << s << " + " << base << "), bq" << s << "_" << us << ");\n";
        }
      };
      o << "      for (; ci + cs < nv; ci += 2 * cs) {\n";
      chunks(2, "        ");
      o << "      }\n"
        << "      for (; ci < nv; ci += cs) {\n";
      chunks(1, "        ");
      o << "      }\n"
        << "      for (i64 ri = nv * " << E << " + " << (block ? "(i64)threadIdx.x" : "(i64)0") << "; ri < nred; ri += cs) {\n";
      offsets("        ", "", "ri");
      element("        ", "", "ri", false);
      o << "      }\n"
        << "    } else {\n";
    }
    constexpr int UR = 4;
    o << "    const i64 rs = " << (block ? "(i64)blockDim.x" : "(i64)1") << ";\n"
      << "    i64 ri = " << (block ? "(i64)threadIdx.x" : "(i64)0") << ";\n"
      << "    for (; ri + " << UR - 1 << " * rs < nred; ri += " << UR << " * rs) {\n";
    for (int u = 0; u < UR; ++u) {
      const std::string us = "_" + std::to_string(u), rix = "ri + " + std::to_string(u) + " * rs";
      offsets("      ", us, rix);
      for (size_t s = 0; s < r.loads.size(); ++s)
        o << "      const " << T(r.loads[s].dtype) << " la" << s << us << " = lp" << s << "[lk" << s << " + lr" << s << us
          << "];\n";
    }
    for (int u = 0; u < UR; ++u)
      element("      ", "_" + std::to_string(u), "ri + " + std::to_string(u) + " * rs", true);
    o << "    }\n"
      << "    for (; ri < nred; ri += rs) {\n";
    offsets("      ", "", "ri");
    element("      ", "", "ri", false);
    o << "    }\n";
    if (vec_gen) o << "    }\n";
    };
    if (kahan()) {
      // A float32 sum of n terms in order is within (n - 1) x 2^-24 of the
      // sum of magnitudes, inside the reduction tolerance (1e-5 of it) for
      // n <= 128: short reduced extents skip the compensation
      o << "    if (nred <= 128) {\n";
      plain_sum = true;
      emit_loops();
      plain_sum = false;
      o << "    } else {\n";
      emit_loops();
      o << "    }\n";
    } else {
      emit_loops();
    }
    if (arg() && r.has_red2 && block) {
      o << "    { " << vt() << " bv; const i64 bi = " << block_reduce_name << "(acc, acci, bv); const " << rt()
        << " mv = " << block_reduce_name << "_v(accm); if (threadIdx.x == 0) { rp[rk] = mv; rp2[rk2] = bi; } }\n";
    } else if (arg() && r.has_red2) {
      o << "    rp[rk] = accm;\n    rp2[rk2] = acci;\n";
    } else if (arg() && block) {
      o << "    { " << vt() << " bv; const i64 v = " << block_reduce_name
        << "(acc, acci, bv); if (threadIdx.x == 0) rp[rk] = v; }\n";
    } else if (arg()) {
      o << "    rp[rk] = acci;\n";
    } else if (block) {
      o << "    { " << rt() << " v = vbe_block_reduce(" << acc_final() << "); if (threadIdx.x == 0) rp[rk] = v; }\n";
    } else {
      o << "    rp[rk] = " << acc_final() << ";\n";
    }
    o << "  }\n}\n";
  }
};

}  // namespace

// Everything the generated text depends on (not sizes, strides, addresses
// or constant values, which are parameter words), as a compact key.
static std::string signature(const Run& r, const Canon& c) {
  std::string k;
  auto put = [&](int64_t v) { k.append((const char*)&v, sizeof v); };
  put((int64_t)r.steps.size());
  for (auto& s : r.steps) {
    put(s.op); put(s.dt_out); put(s.dt_in); put(s.nin); put(s.value); put(s.random_idx);
    for (int a = 0; a < s.nin; ++a) { put(s.a[a].kind); put(s.a[a].idx); put(s.a[a].dtype); put(pow2_const(s.a[a])); }
  }
  put((int64_t)r.value_dtype.size());
  for (int d : r.value_dtype) put(d);
  put((int64_t)r.loads.size());
  for (auto& l : r.loads) put(l.dtype);
  put((int64_t)r.stores.size());
  for (size_t q = 0; q < r.stores.size(); ++q) { put(r.stores[q].dtype); put(r.store_value[q]); }
  put(r.has_red); put(r.red_op); put(r.red_dtype); put(r.red_value); put(r.nrandom); put(r.soft_f64);
  put(r.has_red2); put(r.red2_op);
  put((int64_t)r.consts.size());
  for (auto& o : r.consts) put(o.dtype);
  const Spec& p = c.spec;
  put((int)p.mode); put(p.nd); put(p.ndk); put(p.ndr); put(p.vec); put(p.E); put(p.red_cls); put(p.packed);
  for (int v : p.load_cls) put(v);
  put(-1);
  for (int v : p.store_cls) put(v);
  return k;
}

static std::string generate_source_uncached(const Run& r, const Canon& c, std::string* entry_prefix);

// Generated sources are memoised by signature: a serving loop or a long
// batch plans many runs of a few signatures.
std::shared_ptr<const RunSource> run_source(const Run& r, const Canon& c) {
  static std::mutex mu;
  static std::unordered_map<std::string, std::shared_ptr<const RunSource>> memo;
  const std::string key = signature(r, c);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
  }
  auto e = std::make_shared<RunSource>();
  e->src = generate_source_uncached(r, c, &e->prefix);
  e->key = src_key(e->src);
  std::lock_guard<std::mutex> lk(mu);
  if (memo.size() > 4096) memo.clear();
  memo[key] = e;
  return e;
}

std::string generate_source(const Run& r, const Canon& c, std::string* entry_prefix, std::string* key_out) {
  auto e = run_source(r, c);
  if (entry_prefix) *entry_prefix = e->prefix;
  if (key_out) *key_out = e->key;
  return e->src;
}

static std::string generate_source_uncached(const Run& r, const Canon& c, std::string* entry_prefix) {
  Gen g(r, c);
  g.o << "// generated by libvbe: " << r.steps.size() << " operations, " << r.loads.size() << " loads, "
      << r.stores.size() << " stores\n";
  g.o << kPrelude;
  if (uses_soft_f64(r))
    g.o << sf64_include()
        << "__device__ __forceinline__ double vbe_u01s(u64 seed, u64 key, u64 step, u64 m) {\n"
        << "  u64 z = seed + (key + step * m + 1ull) * 0x9E3779B97F4A7C15ull;\n"
        << "  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;\n"
        << "  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;\n"
        << "  return vbe_u53_to_unit((z ^ (z >> 31)) >> 11);\n}\n";
  g.o << user_op_defs({&r});
  g.emit_elem();
  if (!tile_mode(c.spec.mode) && g.kahan()) {  // the axis kernel's plain-sum variant
    g.plain_sum = true;
    g.emit_struct = false;
    g.elem_name = "vbe_elem_p";
    g.emit_elem();
    g.elem_name = "vbe_elem";
    g.emit_struct = true;
    g.plain_sum = false;
  }
  g.emit_block_reduce();
  if (tile_mode(c.spec.mode)) {
    for (int U : {1, 2, 4}) g.emit_tile_kernel(U);
    if (reg_cap_variants(r))
      for (int U : {1, 2})
        for (int cap : kRegCaps) g.emit_tile_kernel(U, cap);
    if (c.spec.vec && g.bulk_slots() > 0) g.emit_bulk_kernel();
    if (c.spec.nd == 1)
      for (int U : {1, 4}) g.emit_packed_kernel(U);
  } else {
    g.emit_axis_kernel();
  }
  // kernel names carry the run's form, its operation count and a hash of
  // the source, so profiles tell the kernels apart
  std::string src = g.o.str();
  static const char* mode_tag[] = {"e", "r", "at", "ab"};
  std::string tag = std::string(mode_tag[(int)c.spec.mode]) + std::to_string(r.steps.size()) + "_" +
                    hex64(fnv1a(src.data(), src.size())).substr(8);
  for (size_t pos; (pos = src.find("@TAG@")) != std::string::npos;) src.replace(pos, 5, tag);
  if (entry_prefix) *entry_prefix = "vbe_" + tag;
  return src;
}

// ------------------------------------------------------ tile-fused groups

namespace {

struct GroupLayout {
  int nwords = 0;
  std::vector<int> dims;                 // per run: rows, cols
  std::vector<std::vector<int>> lw, sw;  // per run, per slot: pointer, row stride, column stride (-1: shared)
  std::vector<int> consts, rnd;          // per run: first constant word, first RANDOM word
  std::vector<int> ren;                  // per renamed base: source, destination, offset, pitch, rows, cols, count
  std::vector<int> red;                  // per run: reduction output, partials, counter (-1: no reduction)
  std::vector<int> stg;                  // per staged base: offset of the reference view, element count
  int err = -1;                          // error word of the tensor-copy form
};

// Inputs staged through shared memory: a base the group reads from memory
// through several views that differ by small shifts (a stencil's
// neighbours) is copied once per block, tile plus halo, into shared memory
// with coalesced row loads; every read of it is then a shared-memory load at
// a compile-time offset.
struct StagedSlot {
  int k, s, dr, dc;  // run, load slot, shift from the reference view
};
struct StagedBase {
  int64_t base = 0;
  int dtype = 0;
  int ref_k = 0, ref_s = 0;                // reference view (its pointer and row-stride words)
  int rlo = 0, rhi = 0, clo = 0, chi = 0;  // union box around the tile, reference coordinates
  std::vector<StagedSlot> slots;
};

std::vector<StagedBase> staging_plan(const Group& g) {
  std::set<int64_t> written;
  for (auto& r : g.runs)
    for (auto& st : r.stores) written.insert(st.base);
  std::vector<StagedBase> out;
  for (size_t k = 0; k < g.runs.size(); ++k)
    for (size_t s = 0; s < g.runs[k].loads.size(); ++s) {
      const Slot& sl = g.runs[k].loads[s];
      if (g.lds[k][s].prod >= 0 || sl.st.size() != 2 || sl.st[1] != 1 || sl.st[0] <= 16) continue;
      const bool renamed = std::find(g.renamed.begin(), g.renamed.end(), sl.base) != g.renamed.end();
      if (written.count(sl.base) && !renamed) continue;  // read in place: no staging
      if (!g.base_nelem.count(sl.base)) continue;
      int sb = -1;
      for (size_t x = 0; x < out.size(); ++x) {
        const Slot& ref = g.runs[out[x].ref_k].loads[out[x].ref_s];
        if (out[x].base == sl.base && ref.st == sl.st && ref.dtype == sl.dtype) sb = (int)x;
      }
      if (sb < 0) {
        StagedBase x;
        x.base = sl.base;
        x.dtype = sl.dtype;
        x.ref_k = (int)k;
        x.ref_s = (int)s;
        out.push_back(x);
        sb = (int)out.size() - 1;
      }
      const Slot& ref = g.runs[out[sb].ref_k].loads[out[sb].ref_s];
      const int64_t P = ref.st[0], delta = sl.offset - ref.offset;
      const int64_t dr = delta >= 0 ? (delta + P / 2) / P : -((-delta + P / 2) / P);
      const int64_t dc = delta - dr * P;
      if (std::llabs(dr) > 8 || std::llabs(dc) > 8) continue;
      out[sb].slots.push_back({(int)k, (int)s, (int)dr, (int)dc});
    }
  std::vector<StagedBase> keep;
  for (auto& x : out) {
    if (x.slots.size() < 2) continue;
    x.rlo = x.clo = 1 << 20;
    x.rhi = x.chi = -(1 << 20);
    for (auto& q : x.slots) {
      x.rlo = std::min(x.rlo, g.box[q.k][0] + q.dr);
      x.rhi = std::max(x.rhi, g.box[q.k][1] + q.dr);
      x.clo = std::min(x.clo, g.box[q.k][2] + q.dc);
      x.chi = std::max(x.chi, g.box[q.k][3] + q.dc);
    }
    keep.push_back(x);
  }
  return keep;
}

// per run, per load slot: (staged base, slot index) or (-1, -1)
std::vector<std::vector<std::pair<int, int>>> staged_index(const Group& g, const std::vector<StagedBase>& sp) {
  std::vector<std::vector<std::pair<int, int>>> ix(g.runs.size());
  for (size_t k = 0; k < g.runs.size(); ++k) ix[k].assign(g.runs[k].loads.size(), {-1, -1});
  for (size_t b = 0; b < sp.size(); ++b)
    for (size_t q = 0; q < sp[b].slots.size(); ++q) ix[sp[b].slots[q].k][sp[b].slots[q].s] = {(int)b, (int)q};
  return ix;
}

GroupLayout group_layout(const Group& g) {
  GroupLayout L;
  const int m = (int)g.runs.size();
  int w = 4;  // anchor rows, anchor cols, tiles per row, tiles
  for (int k = 0; k < m; ++k) {
    L.dims.push_back(w);
    w += 2;
  }
  L.lw.resize(m);
  L.sw.resize(m);
  for (int k = 0; k < m; ++k) {
    for (size_t s = 0; s < g.runs[k].loads.size(); ++s) {
      if (g.lds[k][s].prod >= 0) {
        L.lw[k].push_back(-1);
        continue;
      }
      L.lw[k].push_back(w);
      w += 3;
    }
    for (size_t s = 0; s < g.runs[k].stores.size(); ++s) {
      if (k != m - 1) {
        L.sw[k].push_back(-1);
        continue;
      }
      L.sw[k].push_back(w);
      w += 3;
    }
  }
  for (int k = 0; k < m; ++k) {
    L.consts.push_back(w);
    w += (int)g.runs[k].consts.size();
    L.rnd.push_back(w);
    w += 3 * g.runs[k].nrandom;
  }
  for (size_t r = 0; r < g.renamed.size(); ++r) {
    L.ren.push_back(w);
    w += 7;
  }
  for (int k = 0; k < m; ++k) {
    L.red.push_back(g.runs[k].has_red ? w : -1);
    if (g.runs[k].has_red) w += 3;
  }
  for (size_t b = 0; b < staging_plan(g).size(); ++b) {
    L.stg.push_back(w);
    w += 5;  // reference view's offset, base size; tensor copies: x and y of the box origin, column shift
  }
  L.err = w++;
  L.nwords = w;
  return L;
}

// box of run k around a th x tw tile: rows, columns
int box_rows(const Group& g, int k, int th) { return th + g.box[k][1] - g.box[k][0]; }
int box_cols(const Group& g, int k, int tw) { return tw + g.box[k][3] - g.box[k][2]; }

// shared-memory offsets of the consumed stores for one tile shape
std::vector<std::vector<int64_t>> group_smem(const Group& g, int th, int tw, int64_t* total) {
  std::vector<std::vector<int64_t>> off(g.runs.size());
  int64_t acc = 0;
  for (size_t k = 0; k < g.runs.size(); ++k)
    for (size_t s = 0; s < g.runs[k].stores.size(); ++s) {
      if (!g.consumed[k][s]) {
        off[k].push_back(-1);
        continue;
      }
      off[k].push_back(acc);
      int64_t pts = (int64_t)box_rows(g, (int)k, th) * box_cols(g, (int)k, tw);
      acc += (pts * itemsize(g.runs[k].stores[s].dtype) + 15) / 16 * 16;
    }
  *total = acc;
  return off;
}

// row length of a staged input's shared-memory box: the tile's columns plus
// halo, and for tensor copies one 16-byte unit more, the copy starting at the
// 16-byte boundary at or below the box's first column
int staged_cols(const StagedBase& b, int tw, bool tma) {
  const int sc = tw + b.chi - b.clo;
  if (!tma) return sc;
  const int a = 16 / itemsize(b.dtype);
  return (sc + a - 1 + a - 1) / a * a;
}

// shared-memory offsets of the staged inputs, placed after *total (tensor
// copies: `stages` stages per input, 128-byte aligned, stage s at off + s x
// stage bytes; then a "full" and an "empty" mbarrier per stage)
std::vector<int64_t> staged_smem(const std::vector<StagedBase>& sp, int th, int tw, int64_t* total,
                                 int stages = 0) {
  const bool tma = stages > 0;
  std::vector<int64_t> off;
  int64_t acc = *total;
  const int64_t al = tma ? 128 : 16;
  acc = (acc + al - 1) / al * al;
  for (auto& b : sp) {
    off.push_back(acc);
    const int64_t pts = (int64_t)(th + b.rhi - b.rlo) * staged_cols(b, tw, tma);
    acc += (pts * itemsize(b.dtype) + al - 1) / al * al * (tma ? stages : 1);
  }
  if (tma) acc += 16 * stages;
  *total = acc;
  return off;
}

int64_t staged_stage_bytes(const StagedBase& b, int th, int tw) {
  const int64_t pts = (int64_t)(th + b.rhi - b.rlo) * staged_cols(b, tw, true);
  return (pts * itemsize(b.dtype) + 127) / 128 * 128;
}

constexpr int64_t kGroupSmemLimit = 200 * 1024;

bool group_stacked(const Group& g);
// stages of the tensor-copy form: three when the tile's values stay in
// registers (shared memory holds only the stages), else two
int tma_stages(const Group& g) { return group_stacked(g) ? 3 : 2; }

// A group whose runs share one shape and read each other's values only at
// the same point (no shifts, no halos) is evaluated point by point: every
// run in turn on the point, the values passed in registers (no shared
// memory, no block barriers). At most one run may reduce.
bool group_stacked(const Group& g) {
  int nred = 0;
  for (size_t k = 0; k < g.runs.size(); ++k) {
    if (g.box[k] != std::array<int, 4>{0, 0, 0, 0} || g.runs[k].shape != g.runs.back().shape) return false;
    for (auto& ld : g.lds[k])
      if (ld.prod >= 0 && (ld.dr != 0 || ld.dc != 0)) return false;
    nred += g.runs[k].has_red ? 1 : 0;
  }
  return nred <= 1;
}

// Tensor copies need whole rows (the base a whole number of rows of the
// row stride) and 16-byte row strides; a reduction only in a group whose
// values stay in registers (its persistent blocks accumulate over all their
// tiles and combine once, after the tile loop).
bool tma_ok(const Group& g) {
  for (auto& r : g.runs)
    if (r.has_red && !group_stacked(g)) return false;
  for (auto& b : staging_plan(g)) {
    const Slot& ref = g.runs[b.ref_k].loads[b.ref_s];
    const int64_t P = ref.st[0], ne = g.base_nelem.at(b.base);
    if ((P * itemsize(b.dtype)) % 16 != 0 || ne % P != 0 || ne / P >= (1ll << 31) || P >= (1ll << 31)) return false;
  }
  return true;
}

// ------------------------------------------------------- row-sweep form
//
// One warp owns a strip of WO anchor columns and R anchor rows and walks the
// rows top to bottom. Every node of the group (a staged input, or a run)
// handles one row per step, at a fixed lead: at step t it produces row
// i0 + t + rhi of its own box (rhi: the node's bottom margin), so that every
// row a later node reads at that step is already produced, this step or an
// earlier one. A node keeps the last `depth` rows it produced in registers,
// as many as its consumers still read, so every point of every run is
// evaluated once, with no halo recomputed above or below (the first steps of
// a strip, before its anchor row 0, produce the rows the first anchor rows
// need). Lane l of node n holds column j0 + s_n + l; a consumer reading a
// producer at column shift dc takes the value from lane l + s_l + dc - s_n
// by a warp shuffle (none where that is 0). The lane shifts s_n are chosen
// to need as few shuffles as possible. WO is 32 minus the widest column
// margin, so the lanes of every node cover its box; the lanes outside it
// compute values nobody reads, and never touch memory.
struct SweepNode {
  int rlo = 0, rhi = 0, clo = 0, chi = 0;  // margins around the anchor tile
  int s = 0;                               // lane shift
  std::vector<int> depth;                  // per value (staged: one; run: per store slot): rows kept
};
struct SweepLoad {
  int node = -1, value = 0;  // producer node and value (-1: read from memory)
  int d = 0, delta = 0;      // rows back in the producer's history, lane shift of the shuffle
};
struct SweepPlan {
  bool ok = false;
  int wo = 0, t0 = 0;                     // anchor columns per warp, first step (<= 0)
  int nsb = 0;                            // staged inputs first, then the runs
  std::vector<SweepNode> nodes;
  std::vector<std::vector<SweepLoad>> ld;  // per run, per load slot
};

constexpr int kSweepMaxHistoryBytes = 384;  // register history per thread

SweepPlan sweep_plan(const Group& g) {
  SweepPlan P;
  const int m = (int)g.runs.size();
  for (auto& r : g.runs)
    if (r.has_red || r.has_red2) return P;
  const std::vector<StagedBase> sp = staging_plan(g);
  if (group_stacked(g) && sp.empty()) return P;  // no shifts anywhere: the stacked form is this already
  const auto six = staged_index(g, sp);
  P.nsb = (int)sp.size();
  for (auto& b : sp) {
    SweepNode n;
    n.rlo = b.rlo;
    n.rhi = b.rhi;
    n.clo = b.clo;
    n.chi = b.chi;
    n.depth.assign(1, 1);
    P.nodes.push_back(n);
  }
  for (int k = 0; k < m; ++k) {
    SweepNode n;
    n.rlo = g.box[k][0];
    n.rhi = g.box[k][1];
    n.clo = g.box[k][2];
    n.chi = g.box[k][3];
    n.depth.assign(g.runs[k].stores.size(), 1);
    P.nodes.push_back(n);
  }
  int spread = 0;
  P.t0 = 0;
  for (auto& n : P.nodes) {
    spread = std::max(spread, n.chi - n.clo);
    P.t0 = std::min(P.t0, n.rlo - n.rhi);
  }
  P.wo = 32 - spread;
  if (P.wo < 16) return P;
  // loads served by nodes: history depth, and the edges the shifts align
  struct Edge { int l, n, dc, w; };
  std::vector<Edge> edges;
  P.ld.resize(m);
  for (int k = 0; k < m; ++k) {
    const int me = P.nsb + k;
    P.ld[k].resize(g.runs[k].loads.size());
    for (size_t s = 0; s < g.runs[k].loads.size(); ++s) {
      SweepLoad& L = P.ld[k][s];
      int dr = 0, dc = 0;
      if (six[k][s].first >= 0) {
        const StagedSlot& q = sp[six[k][s].first].slots[six[k][s].second];
        L.node = six[k][s].first;
        L.value = 0;
        dr = q.dr;
        dc = q.dc;
      } else if (g.lds[k][s].prod >= 0) {
        L.node = P.nsb + g.lds[k][s].prod;
        L.value = g.lds[k][s].prod_store;
        dr = g.lds[k][s].dr;
        dc = g.lds[k][s].dc;
      } else {
        continue;  // read from memory at the point itself
      }
      SweepNode& n = P.nodes[L.node];
      L.d = n.rhi - P.nodes[me].rhi - dr;
      if (L.d < 0) return P;  // cannot happen with margins taken from the consumers
      n.depth[L.value] = std::max(n.depth[L.value], L.d + 1);
      edges.push_back({me, L.node, dc, itemsize(g.runs[k].loads[s].dtype) > 4 ? 2 : 1});
    }
  }
  int64_t hist = 0;
  for (int b = 0; b < P.nsb; ++b) hist += (int64_t)(P.nodes[b].depth[0] + 2) * itemsize(sp[b].dtype);
  for (int k = 0; k < m; ++k)
    for (size_t s = 0; s < g.runs[k].stores.size(); ++s)
      if (g.consumed[k][s]) hist += (int64_t)P.nodes[P.nsb + k].depth[s] * itemsize(g.runs[k].stores[s].dtype);
  if (hist > kSweepMaxHistoryBytes) return P;
  // lane shifts: node n may take s in [wo - 32 + chi, clo] (its box on the
  // lanes); coordinate descent on the number of shuffled values
  const int N = (int)P.nodes.size();
  for (auto& n : P.nodes) n.s = n.clo;
  auto cost = [&](int x) {
    int c = 0;
    for (auto& e : edges)
      if ((e.l == x || e.n == x) && P.nodes[e.l].s + e.dc - P.nodes[e.n].s != 0) c += e.w;
    return c;
  };
  for (int pass = 0; pass < 16; ++pass) {
    bool changed = false;
    for (int x = 0; x < N; ++x) {
      SweepNode& n = P.nodes[x];
      const int cur = n.s;
      int best = cur, bc = cost(x);
      for (int v = P.wo - 32 + n.chi; v <= n.clo; ++v) {
        n.s = v;
        const int c = cost(x);
        if (c < bc) {
          bc = c;
          best = v;
        }
      }
      n.s = best;
      changed = changed || best != cur;
    }
    if (!changed) break;
  }
  for (int k = 0; k < m; ++k) {
    const int me = P.nsb + k;
    for (size_t s = 0; s < g.runs[k].loads.size(); ++s) {
      SweepLoad& L = P.ld[k][s];
      if (L.node < 0) continue;
      const int dc = six[k][s].first >= 0 ? sp[six[k][s].first].slots[six[k][s].second].dc : g.lds[k][s].dc;
      L.delta = P.nodes[me].s + dc - P.nodes[L.node].s;
    }
  }
  P.ok = true;
  return P;
}

// Tile shapes the tuner chooses from; two of them also in the staged form
// (inputs through shared memory) and two in the pipelined tensor-copy form,
// where the group has stencil inputs; and the row-sweep form at three strip
// lengths where the group allows it
std::vector<TileShape> group_shapes(const Group& g) {
  std::vector<TileShape> out;
  const bool can_stage = !staging_plan(g).empty();
  const bool can_tma = can_stage && tma_ok(g);
  for (auto t : std::vector<std::array<int, 4>>{{8, 16, 128, 0}, {16, 32, 256, 0}, {32, 32, 256, 0}, {16, 64, 256, 0},
                                                {32, 64, 256, 0}, {32, 32, 256, 1}, {16, 64, 256, 1},
                                                {32, 32, 256, 2}, {16, 64, 256, 2}}) {
    TileShape ts;
    ts.th = t[0];
    ts.tw = t[1];
    ts.block = t[2];
    ts.staged = t[3] == 1;
    ts.tma = t[3] == 2;
    if (ts.staged && !can_stage) continue;
    if (ts.tma && !can_tma) continue;
    group_smem(g, ts.th, ts.tw, &ts.smem);
    if (group_stacked(g)) ts.smem = 0;
    if (ts.staged || ts.tma) staged_smem(staging_plan(g), ts.th, ts.tw, &ts.smem, ts.tma ? tma_stages(g) : 0);
    if (ts.smem <= kGroupSmemLimit) out.push_back(ts);
  }
  const SweepPlan sw = sweep_plan(g);
  if (sw.ok)
    for (int R : {24, 32, 64}) {
      TileShape ts;
      ts.th = R;
      ts.tw = sw.wo;
      ts.block = 256;
      ts.sweep = true;
      out.push_back(ts);
    }
  return out;
}

}  // namespace

// The pipelined tensor-copy form, warp-specialised: the block is the
// compute threads plus one producer warp. Persistent blocks walk tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ...; tile k of a block uses stage
// k mod NS. Lane 0 of the producer warp waits until the compute warps have
// released a stage ("empty" mbarrier, one arrival per compute warp), then
// issues the tile's input boxes into it (one 2-D tensor copy per staged
// input, completing on the stage's "full" mbarrier). Compute threads wait on
// "full", compute, and their warp releases the stage; they meet at block
// barriers only where a phase hands values through shared memory. Every
// wait is bounded; a wait that runs out sets the error word and the thread
// stops working (compute threads keep releasing stages so that no wait
// depends on them), and the producer waits, bounded, for its copies in
// flight before it leaves.
static void emit_tma_prologue(std::ostringstream& o, const Group& g, const GroupLayout& GL, const TileShape& ts,
                              const std::vector<StagedBase>& sp, const std::vector<int64_t>& sgoff, int64_t total,
                              const std::string& pre) {
  auto W = [](int k) { return "p.w[" + std::to_string(k) + "]"; };
  const int nb = (int)sp.size();
  const int NS = tma_stages(g);
  const int NW = ts.block / 32;  // compute warps
  int64_t tx = 0;
  for (auto& b : sp) tx += (int64_t)(ts.th + b.rhi - b.rlo) * staged_cols(b, ts.tw, true) * itemsize(b.dtype);
  const std::string err = "vbe_ptr<volatile unsigned>(" + W(GL.err) + ")[0] = 1u";
  o << "struct __align__(64) PT" << ts.suffix() << " { vbe_tmap tm[" << nb << "]; i64 w[" << GL.nwords << "]; };\n"
    << "extern \"C\" __global__ void __launch_bounds__(" << ts.block + 32 << ") vbe_@TAG@" << ts.suffix()
    << "(const __grid_constant__ PT" << ts.suffix() << " pt) {\n"
    << "  const P& p = *reinterpret_cast<const P*>(pt.w);\n"
    << "  VBE_DYN_SMEM;\n"
    << "  vbe_grid_wait();\n"
    << "  unsigned long long* const full = (unsigned long long*)(vbe_smem + " << (total - 16 * NS) << ");\n"
    << "  unsigned long long* const empty = full + " << NS << ";\n"
    << "  __shared__ volatile int s_abort;  // set by compute threads whose wait ran out\n"
    << "  if (threadIdx.x == 0) {\n"
    << "    for (int s = 0; s < " << NS << "; ++s) { vbe_mbar_init(&full[s], 1); vbe_mbar_init(&empty[s], " << NW
    << "); }\n"
    << "    vbe_fence_mbar_init();\n"
    << "    s_abort = 0;\n"
    << "  }\n"
    << "  __syncthreads();\n"
    << pre
    << "  const i64 ntiles = p.w[3], tpr = p.w[2];\n"
    << "  if (threadIdx.x >= " << ts.block << ") {\n"
    << "    if (threadIdx.x == " << ts.block << ") {  // the producer\n"
    << "      unsigned nis[" << NS << "] = {};  // copies issued per stage\n"
    << "      int kt = 0;\n"
    << "      for (i64 t = blockIdx.x; t < ntiles; t += gridDim.x, ++kt) {\n"
    << "        const int st = kt % " << NS << ";\n"
    << "        if (kt >= " << NS << " && !vbe_mbar_wait(&empty[st], (unsigned)((kt / " << NS << " - 1) & 1))) { "
    << err << "; break; }\n"
    << "        // compute threads that gave up release stages without waiting for\n"
    << "        // their copies: issue nothing more, so a stage never has two in flight\n"
    << "        if (kt >= " << NS << " && s_abort) break;\n"
    << "        const i64 ti = t / tpr, tj = t - ti * tpr;\n"
    << "        vbe_fence_proxy_async();\n"
    << "        vbe_mbar_expect_tx(&full[st], " << tx << "u);\n";
  for (int b = 0; b < nb; ++b) {
    const int64_t stage = staged_stage_bytes(sp[b], ts.th, ts.tw);
    o << "        vbe_tma_2d(vbe_smem + " << sgoff[b] << " + st * " << stage << ", &pt.tm[" << b << "], (int)(tj * "
      << ts.tw << " + " << W(GL.stg[b] + 2) << "), (int)(ti * " << ts.th << " + " << W(GL.stg[b] + 3)
      << "), &full[st]);\n";
  }
  o << "        ++nis[st];\n"
    << "      }\n"
    << "      // the last copies issued into each stage have landed before the block leaves\n"
    << "      for (int s = 0; s < " << NS << "; ++s)\n"
    << "        if (nis[s] && !vbe_mbar_wait(&full[s], (nis[s] - 1u) & 1u)) " << err << ";\n"
    << "    }\n"
    << "  } else {\n"
    << "    bool failed = false;\n"
    << "    int kt = 0;\n"
    << "    for (i64 t = blockIdx.x; t < ntiles; t += gridDim.x, ++kt) {\n"
    << "      const int st = kt % " << NS << ";\n"
    << "      if (!failed && !vbe_mbar_wait_n(&full[st], (unsigned)((kt / " << NS << ") & 1), VBE_CWAIT)) { "
    << "failed = true; s_abort = 1; " << err << "; }\n";
  // phases meeting at block barriers must agree on whether to run
  if (!group_stacked(g)) o << "      failed = vbe_bar_or(1, " << ts.block << ", failed);\n";
  o << "      if (!failed) {\n"
    << "    const i64 ti = t / tpr, tj = t - ti * tpr;\n"
    << "    const i64 i0 = ti * " << ts.th << ", j0 = tj * " << ts.tw << ";\n";
  for (int b = 0; b < nb; ++b) {
    const std::string T = ctype(sp[b].dtype);
    const int64_t stage = staged_stage_bytes(sp[b], ts.th, ts.tw);
    o << "    const " << T << "* const sg" << b << " = (const " << T << "*)(vbe_smem + " << sgoff[b] << " + st * " << stage
      << ") + " << W(GL.stg[b] + 4) << ";\n";
  }
}

// closes the tile: the warp releases the stage; phases that hand values
// through shared memory also wait for every compute warp before the next
// tile overwrites them
static void emit_tma_epilogue(std::ostringstream& o, const Group& g, const TileShape& ts) {
  o << "      }\n"
    << "      __syncwarp();\n"
    << "      if ((threadIdx.x & 31) == 0) vbe_mbar_arrive(&empty[st]);\n";
  if (!group_stacked(g)) o << "      vbe_bar_sync(1, " << ts.block << ");\n";
  o << "    }\n"
    << "  }\n";
}

// elements of renamed bases the anchor does not write: copied to the new buffer
static void emit_copy_through(std::ostringstream& o, const Group& g, const GroupLayout& GL) {
  const int anchor = (int)g.runs.size() - 1;
  auto W = [](int k) { return "p.w[" + std::to_string(k) + "]"; };
  for (size_t rr = 0; rr < g.renamed.size(); ++rr) {
    const std::string T = ctype(g.runs[anchor].stores[g.renamed_slot[rr]].dtype);
    const int w = GL.ren[rr];
    o << "  {\n"
      << "    const auto src = vbe_ptr<const " << T << ">(" << W(w) << ");\n"
      << "    const auto dst = vbe_ptr<" << T << ">(" << W(w + 1) << ");\n"
      << "    const i64 off = " << W(w + 2) << ", P = " << W(w + 3) << ", S0 = " << W(w + 4) << ", S1 = " << W(w + 5)
      << ", nc = " << W(w + 6) << ";\n"
      << "    const i64 gap = P - S1, ng = (S0 - 1) * gap;\n"
      << "    for (i64 q = (i64)blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += (i64)gridDim.x * blockDim.x) {\n"
      << "      i64 e;\n"
      << "      if (q < off) e = q;\n"
      << "      else if (q - off < ng) { const i64 u = q - off, rw = u / gap; e = off + rw * P + S1 + (u - rw * gap); }\n"
      << "      else e = off + (S0 - 1) * P + S1 + (q - off - ng);\n"
      << "      dst[e] = src[e];\n"
      << "    }\n"
      << "  }\n";
  }
}

// The stacked form (group_stacked): one loop over the tile's points; per
// point every run in order, values handed on in registers.
static void emit_stacked(std::ostringstream& o, const Group& g, const GroupLayout& GL,
                  const std::vector<std::unique_ptr<Gen>>& gens, const std::vector<std::vector<std::string>>& cdecl,
                  const TileShape& ts, const std::vector<StagedBase>& sp,
                  const std::vector<std::vector<std::pair<int, int>>>& six) {
  const int m = (int)g.runs.size(), anchor = m - 1;
  auto W = [](int k) { return "p.w[" + std::to_string(k) + "]"; };
  const int TH = ts.th, TW = ts.tw;
  o << "    const i64 rows = " << W(GL.dims[anchor]) << ", cols = " << W(GL.dims[anchor] + 1) << ";\n"
    << "    const i64 r0 = i0, c0 = j0;\n"
    << "    const bool inside = r0 + " << TH << " <= rows && c0 + " << TW << " <= cols;\n";
  std::vector<std::vector<int64_t>> pats;
  std::vector<std::pair<int, int>> pat_word;
  auto mem_slot = [&](const std::string& name, const std::string& T, int w, const Slot& sl) {
    int q = -1;
    for (size_t i = 0; i < pats.size(); ++i)
      if (pats[i] == sl.st) q = (int)i;
    if (q < 0) {
      pats.push_back(sl.st);
      q = (int)pats.size() - 1;
      pat_word.push_back({q, w});
    }
    o << "    const auto " << name << " = vbe_ptr<" << T << ">(" << W(w) << ") + (r0 * " << W(w + 1) << " + c0 * "
      << W(w + 2) << ");\n";
    return name + "[ix" + std::to_string(q) + "]";
  };
  std::vector<std::vector<std::string>> lv(m), sm(m);
  for (int k = 0; k < m; ++k) {
    const Run& r = g.runs[k];
    for (size_t s = 0; s < r.loads.size(); ++s) {
      const GroupLoad& ld = g.lds[k][s];
      if (six[k][s].first >= 0) {
        const StagedBase& B = sp[six[k][s].first];
        const StagedSlot& q = B.slots[six[k][s].second];
        const int SC = staged_cols(B, TW, ts.tma);
        lv[k].push_back("sg" + std::to_string(six[k][s].first) + "[li * " + std::to_string(SC) + " + lj + " +
                        std::to_string((q.dr - B.rlo) * SC + (q.dc - B.clo)) + "]");
      } else if (ld.prod >= 0) {
        lv[k].push_back("b" + std::to_string(ld.prod) + "_" + std::to_string(ld.prod_store));
      } else {
        lv[k].push_back(mem_slot("l" + std::to_string(k) + "p" + std::to_string(s), "const " + std::string(ctype(r.loads[s].dtype)),
                                 GL.lw[k][s], r.loads[s]));
      }
    }
    for (size_t s = 0; s < r.stores.size(); ++s)
      sm[k].push_back(k == anchor ? mem_slot("s" + std::to_string(s) + "p", ctype(r.stores[s].dtype), GL.sw[k][s],
                                             r.stores[s])
                                  : "");
    for (size_t q = 0; q < cdecl[k].size(); ++q) {
      const std::string& d = cdecl[k][q];
      const size_t eq = d.find(" = ");
      o << "    const " << d.substr(0, eq) << " c" << k << "_" << q << d.substr(eq) << ";\n";
    }
  }
  for (auto& pw : pat_word) {
    const std::string q = std::to_string(pw.first);
    o << "    const int pa" << q << " = (int)" << W(pw.second + 1);
    if (pats[pw.first][1] != 1) o << ", pb" << q << " = (int)" << W(pw.second + 2);
    o << ";\n";
  }
  int red = -1;
  for (int k = 0; k < m; ++k)
    if (g.runs[k].has_red) red = k;
  if (red >= 0 && !ts.tma) {  // the tensor-copy form accumulates across its tiles
    gens[red]->o.str("");
    gens[red]->emit_acc_init("    ");
    o << gens[red]->o.str();
  }
  const int NK = (TH * TW + ts.block - 1) / ts.block;
  const bool partial = NK * ts.block > TH * TW;
  auto body = [&](const std::string& ind) {
    for (auto& pw : pat_word) {
      const std::string q = std::to_string(pw.first);
      o << ind << "const int ix" << q << " = li * pa" << q << " + "
        << (pats[pw.first][1] == 1 ? std::string("lj") : "lj * pb" + q) << ";\n";
    }
    for (int k = 0; k < m; ++k) {
      const Run& r = g.runs[k];
      for (size_t s = 0; s < r.stores.size(); ++s)
        o << ind << ctype(r.stores[s].dtype) << " b" << k << "_" << s << ";\n";
      o << ind << "vbe_elem" << k << "(p, (r0 + li) * cols + (c0 + lj)";
      for (auto& x : lv[k]) o << ", " << x;
      for (size_t s = 0; s < r.stores.size(); ++s) o << ", b" << k << "_" << s;
      if (r.has_red) o << (gens[k]->kahan() ? ", acc, kc" : ", acc");
      for (size_t q = 0; q < r.consts.size(); ++q) o << ", c" << k << "_" << q;
      o << ");\n";
    }
    for (size_t s = 0; s < g.runs[anchor].stores.size(); ++s)
      o << ind << sm[anchor][s] << " = b" << anchor << "_" << s << ";\n";
  };
  auto loop = [&](bool checked) {
    o << "#pragma unroll\n"
      << "      for (int kq = 0; kq < " << NK << "; ++kq) {\n"
      << "        const int q = threadIdx.x + kq * " << ts.block << ";\n"
      << "        const int li = q / " << TW << ", lj = q - li * " << TW << ";\n";
    std::string cond;
    if (partial) cond = "q < " + std::to_string(TH * TW);
    if (checked) {
      if (!cond.empty()) cond += " && ";
      cond += "r0 + li < rows && c0 + lj < cols";
    }
    if (cond.empty()) {
      body("        ");
    } else {
      o << "        if (" << cond << ") {\n";
      body("          ");
      o << "        }\n";
    }
    o << "      }\n";
  };
  o << "    if (inside) {\n";
  loop(false);
  o << "    } else {\n";
  loop(true);
  o << "    }\n";
  if (red >= 0 && !ts.tma) {
    const int w = GL.red[red];
    gens[red]->o.str("");
    gens[red]->emit_full_epilogue("    ", W(w + 1), "blockIdx.x", W(w + 2), "gridDim.x", W(w));
    o << gens[red]->o.str();
  }
}

// lane shifts of the row-sweep form (bool through int: shuffles move 32 or 64 bits)
const char* kSweepPrelude = R"CUDA(
template <class T> __device__ __forceinline__ T vbe_lane_dn(T v, unsigned d) { return __shfl_down_sync(0xffffffffu, v, d); }
template <class T> __device__ __forceinline__ T vbe_lane_up(T v, unsigned d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ bool vbe_lane_dn(bool v, unsigned d) { return __shfl_down_sync(0xffffffffu, (int)v, d) != 0; }
__device__ __forceinline__ bool vbe_lane_up(bool v, unsigned d) { return __shfl_up_sync(0xffffffffu, (int)v, d) != 0; }
)CUDA";

// A constant of a group's source as an exact literal (group sources are
// already keyed by their constants' values): hexadecimal floating literals
// for finite values, the bit pattern otherwise.
static std::string const_literal(const Operand& a) {
  char buf[64];
  switch (a.dtype) {
    case VBE_FLOAT64:
      if (std::isfinite(a.f)) {
        snprintf(buf, sizeof buf, "(%a)", a.f);
        return buf;
      }
      return "__longlong_as_double(" + std::to_string(const_bits(a)) + "ll)";
    case VBE_FLOAT32: {
      const float f = (float)a.f;
      if (std::isfinite(f)) {
        snprintf(buf, sizeof buf, "(%af)", (double)f);
        return buf;
      }
      return "__int_as_float(" + std::to_string((int)(uint32_t)const_bits(a)) + ")";
    }
    case VBE_BOOL:
      return a.i ? "true" : "false";
    default:
      snprintf(buf, sizeof buf, "((long long)0x%llxull)", (unsigned long long)a.i);
      return buf;
  }
}

// The row-sweep form (sweep_plan): warp gw takes strip (ti, tj) of the
// anchor, rows i0 .. i0 + R - 1 and columns j0 .. j0 + WO - 1. Staged inputs
// are loaded PF rows ahead of their use, so that a row's loads are in flight
// while the rows before it are computed. Steps t0 .. -1 fill the histories;
// steps 0 .. R - 1 produce one anchor row each. Every lane runs every step
// (warp shuffles need the whole warp); loads and stores are guarded by the
// lane's column lying in its node's box, and rows always lie in the runs'
// shapes (the margins come from what the consumers read).
//
// Each history (and each staged input's prefetch ring) is a ring of
// registers whose size is a power of two; the step loop is unrolled by the
// largest ring size U, so that at step t the value of t - d sits in a fixed
// register and nothing is moved between registers. Strides and constants are
// literals (the group's source is keyed by them), so the row offsets of an
// unrolled block fold into the loads' and stores' immediate offsets, and one
// pointer per stream advances once per block.
static void emit_sweep(std::ostringstream& o, const Group& g, const GroupLayout& GL, const TileShape& ts) {
  const SweepPlan P = sweep_plan(g);
  const std::vector<StagedBase> sp = staging_plan(g);
  const int m = (int)g.runs.size(), anchor = m - 1, NW = ts.block / 32, R = ts.th, WO = ts.tw;
  const int PF = 2;
  // 32-bit groups: four blocks per SM (64 registers a thread); left to the
  // compiler, they got 48 and re-derived values inside the loop instead
  // (measured: 204 against 189 instructions per cell on shallow water)
  bool wide = false;
  for (auto& r : g.runs) {
    for (auto& sl : r.loads) wide = wide || itemsize(sl.dtype) > 4;
    for (auto& sl : r.stores) wide = wide || itemsize(sl.dtype) > 4;
  }
  const int minb = wide ? 0 : 4;
  const int nn = (int)P.nodes.size();
  auto W = [](int k) { return "p.w[" + std::to_string(k) + "]"; };
  auto I = [](int64_t v) { return std::to_string(v); };
  auto pow2 = [](int v) {
    int r = 1;
    while (r < v) r <<= 1;
    return r;
  };
  std::vector<std::vector<int>> ring(nn);
  int U = 1;
  for (int n = 0; n < nn; ++n) {
    for (int d : P.nodes[n].depth) ring[n].push_back(pow2(n < P.nsb ? PF + d : d));
    for (int r : ring[n]) U = std::max(U, r);
  }
  // the register holding value v of node n produced at step q (any integer)
  auto reg = [&](int n, int v, int q) {
    const int S = ring[n][v];
    return "r" + I(n) + "_" + I(v) + "_" + I(((q % S) + S) % S);
  };
  auto strides = [](const Slot& sl) { return std::make_pair(sl.st[0], sl.st[1]); };
  o << "extern \"C\" __global__ void __launch_bounds__(" << ts.block << (minb ? ", " + std::to_string(minb) : std::string()) << ") vbe_@TAG@" << ts.suffix()
    << "(const P p) {\n"
    << "  vbe_grid_wait();\n"
    << "  const i64 gw = (i64)blockIdx.x * " << NW << " + (threadIdx.x >> 5);\n"
    << "  if (gw < p.w[3]) {  // the whole warp or none of it\n"
    << "    const int lane = threadIdx.x & 31;\n"
    << "    const i64 ti = gw / p.w[2], tj = gw - ti * p.w[2];\n"
    << "    const i64 i0 = ti * " << R << ", j0 = tj * " << WO << ";\n"
    << "    const int reff = (int)min((i64)" << R << ", p.w[0] - i0), weff = (int)min((i64)" << WO
    << ", p.w[1] - j0);\n";
  for (int n = 0; n < nn; ++n) {
    const SweepNode& N = P.nodes[n];
    o << "    const int x" << n << " = lane + (" << N.s << ");\n"
      << "    const bool ok" << n << " = x" << n << " >= " << N.clo << " && x" << n << " < weff + " << N.chi << ";\n";
  }
  // staged inputs: pointer at the row of step 0, ring registers, the first PF rows
  for (int b = 0; b < P.nsb; ++b) {
    const StagedBase& B = sp[b];
    const SweepNode& N = P.nodes[b];
    const std::string T = ctype(B.dtype);
    const int64_t Pr = g.runs[B.ref_k].loads[B.ref_s].st[0];
    o << "    auto sq" << b << " = vbe_ptr<const " << T << ">(" << W(GL.lw[B.ref_k][B.ref_s]) << ") + ((i0 + "
      << N.rhi << ") * " << Pr << "ll + j0 + x" << b << ");\n"
      << "    " << T;
    for (int r = 0; r < ring[b][0]; ++r) o << (r ? ", " : " ") << "r" << b << "_0_" << r << " = 0";
    o << ";\n";
    for (int q = P.t0; q < P.t0 + PF; ++q)
      if (q + N.rhi >= N.rlo)
        o << "    if (ok" << b << (q > 0 ? " && " + I(q) + " < reff" : "") << ") " << reg(b, 0, q) << " = sq" << b
          << "[" << I(q * Pr) << "ll];\n";
  }
  // runs: memory pointers at the row of step 0, rings of the values they hand on
  for (int k = 0; k < m; ++k) {
    const Run& r = g.runs[k];
    const int n = P.nsb + k;
    for (size_t s = 0; s < r.loads.size(); ++s) {
      if (P.ld[k][s].node >= 0) continue;
      auto st = strides(r.loads[s]);
      o << "    auto lq" << k << "_" << s << " = vbe_ptr<const " << ctype(r.loads[s].dtype) << ">("
        << W(GL.lw[k][s]) << ") + ((i0 + " << P.nodes[n].rhi << ") * " << st.first << "ll + (j0 + x" << n << ") * "
        << st.second << "ll);\n";
    }
    for (size_t s = 0; s < r.stores.size(); ++s) {
      const std::string T = ctype(r.stores[s].dtype);
      if (k == anchor) {
        auto st = strides(r.stores[s]);
        o << "    auto oq" << s << " = vbe_ptr<" << T << ">(" << W(GL.sw[k][s]) << ") + (i0 * " << st.first
          << "ll + (j0 + x" << n << ") * " << st.second << "ll);\n";
      } else {
        o << "    " << T;
        for (int q = 0; q < ring[n][s]; ++q) o << (q ? ", " : " ") << "r" << n << "_" << s << "_" << q << " = 0";
        o << ";\n";
      }
    }
  }
  // one step: q the step index modulo the rings (its registers), rel the
  // row offset from the pointers, t its index at run time; check: whether
  // a load PF steps ahead may run past the strip
  auto advance = [&](int64_t rows, const std::string& ind) {
    for (int b = 0; b < P.nsb; ++b)
      o << ind << "sq" << b << " = sq" << b << " + " << I(rows * g.runs[sp[b].ref_k].loads[sp[b].ref_s].st[0])
        << "ll;\n";
    for (int k = 0; k < m; ++k)
      for (size_t s = 0; s < g.runs[k].loads.size(); ++s)
        if (P.ld[k][s].node < 0)
          o << ind << "lq" << k << "_" << s << " = lq" << k << "_" << s << " + "
            << I(rows * g.runs[k].loads[s].st[0]) << "ll;\n";
    for (size_t s = 0; s < g.runs[anchor].stores.size(); ++s)
      o << ind << "oq" << s << " = oq" << s << " + " << I(rows * g.runs[anchor].stores[s].st[0]) << "ll;\n";
  };
  auto step = [&](int q, int rel, const std::string& t, bool fill, bool check, const std::string& ind) {
    for (int b = 0; b < P.nsb; ++b) {
      const SweepNode& N = P.nodes[b];
      if (fill && q + PF + N.rhi < N.rlo) continue;  // a row above the input's box
      const int64_t Pr = g.runs[sp[b].ref_k].loads[sp[b].ref_s].st[0];
      const bool guard = fill ? q + PF > 0 : check;
      o << ind << "if (ok" << b << (guard ? " && " + t + " + " + I(PF) + " < reff" : "") << ") "
        << reg(b, 0, q + PF) << " = sq" << b << "[" << I((int64_t)(rel + PF) * Pr) << "ll];\n";
    }
    for (int k = 0; k < m; ++k) {
      const Run& r = g.runs[k];
      const int n = P.nsb + k;
      const SweepNode& N = P.nodes[n];
      if (fill && q < N.rlo - N.rhi) continue;  // rows above this run's box
      o << ind << "{  // run " << k << "\n"
        << ind << "  const i64 rr = i0 + (" << t << " + " << N.rhi << "), cc = j0 + x" << n << ";\n";
      for (size_t s = 0; s < r.loads.size(); ++s) {
        const std::string T = ctype(r.loads[s].dtype), a = "a" + I((int)s);
        const SweepLoad& L = P.ld[k][s];
        if (L.node < 0) {
          o << ind << "  const " << T << " " << a << " = ok" << n << " ? lq" << k << "_" << s << "["
            << I((int64_t)rel * r.loads[s].st[0]) << "ll] : (" << T << ")0;\n";
          continue;
        }
        std::string x = reg(L.node, L.value, q - L.d);
        if (L.delta > 0) x = "vbe_lane_dn(" + x + ", " + I(L.delta) + "u)";
        if (L.delta < 0) x = "vbe_lane_up(" + x + ", " + I(-L.delta) + "u)";
        o << ind << "  const " << T << " " << a << " = " << x << ";\n";
      }
      for (size_t s = 0; s < r.stores.size(); ++s) o << ind << "  " << ctype(r.stores[s].dtype) << " b" << s << ";\n";
      o << ind << "  vbe_elem" << k << "(p, rr * " << r.shape[1] << "ll + cc";
      for (size_t s = 0; s < r.loads.size(); ++s) o << ", a" << s;
      for (size_t s = 0; s < r.stores.size(); ++s) o << ", b" << s;
      for (auto& cst : r.consts) o << ", " << const_literal(cst);
      o << ");\n";
      if (k == anchor) {
        o << ind << "  if (ok" << n << ") {\n";
        for (size_t s = 0; s < r.stores.size(); ++s)
          o << ind << "    oq" << s << "[" << I((int64_t)rel * r.stores[s].st[0]) << "ll] = b" << s << ";\n";
        o << ind << "  }\n";
      } else {
        for (size_t s = 0; s < r.stores.size(); ++s) o << ind << "  " << reg(n, (int)s, q) << " = b" << s << ";\n";
      }
      o << ind << "}\n";
    }
  };
  for (int t = P.t0; t < 0; ++t) {
    o << "    {  // fill step " << t << "\n";
    step(t, t, I(t), true, false, "      ");
    o << "    }\n";
  }
  o << "    int tb = 0;\n"
    << "    for (; tb + " << U << " <= reff; tb += " << U << ") {\n";
  for (int j = 0; j < U; ++j) step(j, j, "tb + " + I(j), false, j + PF >= U, "      ");
  advance(U, "      ");  // every stream moves on by U rows
  o << "    }\n";
  for (int j = 0; j + 1 < U; ++j) {  // the last steps of a ragged strip
    o << "    if (tb + " << j << " < reff) {\n";
    step(j, j, "tb + " + I(j), false, true, "      ");
    o << "    }\n";
  }
  o << "  }\n";
  emit_copy_through(o, g, GL);
  o << "}\n";
}

std::vector<TmaBox> group_tma_boxes(const Group& g, const TileShape& ts) {
  std::vector<TmaBox> out;
  for (auto& b : staging_plan(g)) {
    const Slot& ref = g.runs[b.ref_k].loads[b.ref_s];
    TmaBox x;
    x.base = b.base;
    x.isz = itemsize(b.dtype);
    x.pitch = ref.st[0];
    x.rows = g.base_nelem.at(b.base) / ref.st[0];
    x.box_cols = staged_cols(b, ts.tw, true);
    x.box_rows = ts.th + b.rhi - b.rlo;
    x.ref_k = b.ref_k;
    x.ref_s = b.ref_s;
    out.push_back(x);
  }
  return out;
}

// Everything a group's source depends on, as a key: the runs (views with
// their bases numbered by first appearance, operations, constants,
// reductions), the shifts, margins, renamed bases and base sizes. Planning
// the same group again (every iteration of a solver, every request of a
// shape) then reuses its source instead of generating it anew.
static std::string group_key(const Group& g) {
  std::string k;
  std::vector<int64_t> ids;
  auto put = [&](int64_t v) { k.append((const char*)&v, sizeof v); };
  auto bid = [&](int64_t b) {
    for (size_t i = 0; i < ids.size(); ++i)
      if (ids[i] == b) return (int64_t)i;
    ids.push_back(b);
    return (int64_t)ids.size() - 1;
  };
  auto slot = [&](const Slot& sl) {
    put(bid(sl.base));
    put(sl.offset);
    put(sl.dtype);
    put((int64_t)sl.st.size());
    for (auto v : sl.st) put(v);
  };
  auto operand = [&](const Operand& a) {
    int64_t fb;
    memcpy(&fb, &a.f, 8);
    put(a.kind);
    put(a.idx);
    put(a.dtype);
    put(a.i);
    put(fb);
  };
  put((int64_t)g.runs.size());
  for (auto& r : g.runs) {
    put((int64_t)r.shape.size());
    for (auto v : r.shape) put(v);
    put((int64_t)r.loads.size());
    for (auto& sl : r.loads) slot(sl);
    put((int64_t)r.stores.size());
    for (auto& sl : r.stores) slot(sl);
    for (int v : r.store_value) put(v);
    put((int64_t)r.steps.size());
    for (auto& st : r.steps) {
      put(st.op); put(st.dt_out); put(st.dt_in); put(st.nin); put(st.value); put(st.random_idx);
      for (int a = 0; a < st.nin; ++a) operand(st.a[a]);
    }
    put((int64_t)r.value_dtype.size());
    for (int d : r.value_dtype) put(d);
    put(r.has_red); put(r.red_op); put(r.red_dtype); put(r.red_value);
    put((int64_t)r.red_axes.size());
    for (int a : r.red_axes) put(a);
    if (r.has_red) slot(r.red_out);
    put(r.has_red2); put(r.red2_op);
    if (r.has_red2) slot(r.red2_out);
    put(r.nrandom);
    put((int64_t)r.consts.size());
    for (auto& o : r.consts) operand(o);
    put(r.soft_f64);
  }
  for (auto& b : g.box)
    for (int v : b) put(v);
  for (auto& l : g.lds) {
    put((int64_t)l.size());
    for (auto& x : l) { put(x.prod); put(x.prod_store); put(x.dr); put(x.dc); }
  }
  for (auto& c : g.consumed) {
    put((int64_t)c.size());
    for (char x : c) put(x);
  }
  put((int64_t)g.renamed.size());
  for (size_t i = 0; i < g.renamed.size(); ++i) {
    put(bid(g.renamed[i]));
    put(g.renamed_slot[i]);
    put(g.renamed_nelem[i]);
  }
  put((int64_t)g.base_nelem.size());
  for (int64_t b : ids) {
    auto it = g.base_nelem.find(b);
    put(it == g.base_nelem.end() ? -1 : it->second);
  }
  return k;
}

static std::string generate_group_source_uncached(const Group& g, std::string* entry_prefix,
                                                  std::vector<TileShape>* shapes_out);

std::shared_ptr<const GroupSource> group_source(const Group& g) {
  if (g.source) return g.source;
  static std::mutex mu;
  static std::unordered_map<std::string, std::shared_ptr<const GroupSource>> memo;
  const std::string key = group_key(g);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = memo.find(key);
    if (it != memo.end()) return g.source = it->second;
  }
  auto e = std::make_shared<GroupSource>();
  e->src = generate_group_source_uncached(g, &e->prefix, &e->shapes);
  e->key = src_key(e->src);
  std::lock_guard<std::mutex> lk(mu);
  if (memo.size() > 1024) memo.clear();
  memo[key] = e;
  return g.source = e;
}

std::string generate_group_source(const Group& g, std::string* entry_prefix, std::vector<TileShape>* shapes_out,
                                  std::string* key_out) {
  auto e = group_source(g);
  if (entry_prefix) *entry_prefix = e->prefix;
  if (shapes_out) *shapes_out = e->shapes;
  if (key_out) *key_out = e->key;
  return e->src;
}

static std::string generate_group_source_uncached(const Group& g, std::string* entry_prefix,
                                                  std::vector<TileShape>* shapes_out) {
  const int m = (int)g.runs.size();
  const int anchor = m - 1;
  GroupLayout GL = group_layout(g);
  std::ostringstream o;
  int nsteps = 0;
  bool soft = false;
  for (auto& r : g.runs) {
    nsteps += (int)r.steps.size();
    soft = soft || uses_soft_f64(r);
  }
  o << "// generated by libvbe: tile-fused group of " << m << " runs, " << nsteps << " operations\n";
  o << kPrelude;
  const std::vector<TileShape> shapes = group_shapes(g);
  for (auto& ts : shapes)
    if (ts.tma) {
      o << kTmaPrelude;
      break;
    }
  for (auto& ts : shapes)
    if (ts.sweep) {
      o << kSweepPrelude;
      break;
    }
  if (soft)
    o << sf64_include()
      << "__device__ __forceinline__ double vbe_u01s(u64 seed, u64 key, u64 step, u64 m) {\n"
      << "  u64 z = seed + (key + step * m + 1ull) * 0x9E3779B97F4A7C15ull;\n"
      << "  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;\n"
      << "  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;\n"
      << "  return vbe_u53_to_unit((z ^ (z >> 31)) >> 11);\n}\n";
  o << "struct P { i64 w[" << GL.nwords << "]; };\n";
  {
    std::vector<const Run*> rs;
    for (auto& r : g.runs) rs.push_back(&r);
    o << user_op_defs(rs);
  }
  // one element function per run, reading its constants at the group's words
  std::vector<Canon> canons(m);
  std::vector<std::vector<std::string>> cdecl(m);  // per run: the constants, decoded once per block
  std::vector<std::unique_ptr<Gen>> gens(m);
  for (int k = 0; k < m; ++k) {
    const Run& r = g.runs[k];
    Canon& cn = canons[k];
    cn.spec.mode = r.has_red ? Mode::FULL : Mode::ELEM;
    cn.spec.nd = 2;
    cn.spec.load_cls.assign(r.loads.size(), 2);
    cn.spec.store_cls.assign(r.stores.size(), 2);
    gens[k].reset(new Gen(r, cn));
    Gen& gen = *gens[k];
    gen.L.consts = GL.consts[k];
    for (int q = 0; q < r.nrandom; ++q) gen.L.rnd[q] = GL.rnd[k] + 3 * q;
    gen.elem_name = "vbe_elem" + std::to_string(k);
    gen.guard_div = true;
    gen.const_params = true;
    for (auto& cst : r.consts) cdecl[k].push_back(std::string(ctype(cst.dtype)) + " = " + gen.const_expr(cst));
    gen.emit_struct = false;
    gen.block_reduce_name = "vbe_block_reduce" + std::to_string(k);
    gen.emit_elem();
    gen.emit_block_reduce();
    o << gen.o.str();
    gen.o.str("");
  }
  auto W = [](int k) { return "p.w[" + std::to_string(k) + "]"; };
  for (const TileShape& ts : shapes) {
    if (ts.sweep) {
      emit_sweep(o, g, GL, ts);
      continue;
    }
    int64_t total = 0;
    auto soff = group_smem(g, ts.th, ts.tw, &total);
    if (group_stacked(g)) total = 0;
    const std::vector<StagedBase> sp = (ts.staged || ts.tma) ? staging_plan(g) : std::vector<StagedBase>();
    const auto six = staged_index(g, sp);
    const std::vector<int64_t> sgoff = staged_smem(sp, ts.th, ts.tw, &total, ts.tma ? tma_stages(g) : 0);
    if (ts.tma) {
      // a reduction accumulates over all of a block's tiles (every thread,
      // the producer warp's at the identity) and is combined after the loop
      std::string pre;
      for (int k = 0; k < m; ++k)
        if (g.runs[k].has_red) {
          gens[k]->o.str("");
          gens[k]->emit_acc_init("  ");
          pre = gens[k]->o.str();
        }
      emit_tma_prologue(o, g, GL, ts, sp, sgoff, total, pre);
    } else {
      o << "extern \"C\" __global__ void __launch_bounds__(" << ts.block << ") vbe_@TAG@" << ts.suffix()
        << "(const P p) {\n"
        << "  VBE_DYN_SMEM;\n"
        << "  vbe_grid_wait();\n"
        << "  if ((i64)blockIdx.x < p.w[3]) {\n"
        << "    const i64 ti = (i64)blockIdx.x / p.w[2], tj = (i64)blockIdx.x - ti * p.w[2];\n"
        << "    const i64 i0 = ti * " << ts.th << ", j0 = tj * " << ts.tw << ";\n";
    }
    // staged inputs: tile plus halo, coalesced along rows, elements outside
    // the base skipped (their cells are never read)
    for (size_t b = 0; b < sp.size() && !ts.tma; ++b) {
      const StagedBase& B = sp[b];
      const std::string T = ctype(B.dtype);
      const int SR = ts.th + B.rhi - B.rlo, SC = ts.tw + B.chi - B.clo, w = GL.lw[B.ref_k][B.ref_s];
      o << "    const " << T << "* const sg" << b << " = (const " << T << "*)(vbe_smem + " << sgoff[b] << ");\n"
        << "    {\n"
        << "      const auto stp = vbe_ptr<const " << T << ">(" << W(w) << ");\n"
        << "      const i64 P = " << W(w + 1) << ", soff = " << W(GL.stg[b]) << ", sne = " << W(GL.stg[b] + 1) << ";\n"
        << "      " << T << "* const sb = (" << T << "*)(vbe_smem + " << sgoff[b] << ");\n"
        << "      for (int q = threadIdx.x; q < " << SR * SC << "; q += " << ts.block << ") {\n"
        << "        const int u = q / " << SC << ", v = q - u * " << SC << ";\n"
        << "        const i64 e = (i0 + (" << B.rlo << ") + u) * P + (j0 + (" << B.clo << ") + v);\n"
        << "        if (soff + e >= 0 && soff + e < sne) sb[q] = stp[e];\n"
        << "      }\n"
        << "    }\n";
    }
    if (!sp.empty() && !ts.tma) o << "    __syncthreads();\n";
    if (group_stacked(g)) {
      emit_stacked(o, g, GL, gens, cdecl, ts, sp, six);
    } else {
    for (int k = 0; k < m; ++k) {
      const Run& r = g.runs[k];
      const int BH = box_rows(g, k, ts.th), BW = box_cols(g, k, ts.tw);
      o << "    {  // run " << k << ": " << r.steps.size() << " operations over a " << BH << " x " << BW << " box\n"
        << "      const i64 rows = " << W(GL.dims[k]) << ", cols = " << W(GL.dims[k] + 1) << ";\n"
        << "      const i64 r0 = i0 + (" << g.box[k][0] << "), c0 = j0 + (" << g.box[k][2] << ");\n"
        << "      const bool inside = r0 >= 0 && c0 >= 0 && r0 + " << BH << " <= rows && c0 + " << BW
        << " <= cols;\n";
      // memory slots: pointer to the box origin and 32-bit offsets inside the
      // box (strides are limited to 2^24 when the group is formed); slots
      // with equal strides share one offset per point
      std::vector<std::vector<int64_t>> pats;
      auto pattern = [&](const Slot& sl) {
        for (size_t q = 0; q < pats.size(); ++q)
          if (pats[q] == sl.st) return (int)q;
        pats.push_back(sl.st);
        return (int)pats.size() - 1;
      };
      std::vector<std::pair<int, int>> pat_word;  // (pattern, stride word of a slot using it)
      auto mem_slot = [&](const char* pfx, const std::string& n, const std::string& T, int w, const Slot& sl) {
        int q = pattern(sl);
        if ((int)pat_word.size() <= q) pat_word.push_back({q, w});
        o << "      const auto " << pfx << "p" << n << " = vbe_ptr<" << T << ">(" << W(w) << ") + (r0 * " << W(w + 1)
          << " + c0 * " << W(w + 2) << ");\n";
        return std::string(pfx) + "p" + n + "[ix" + std::to_string(q) + "]";
      };
      std::vector<std::string> lv, sv, sm;
      for (size_t s = 0; s < r.loads.size(); ++s) {
        const std::string T = ctype(r.loads[s].dtype), n = std::to_string(s);
        const GroupLoad& ld = g.lds[k][s];
        if (six[k][s].first >= 0) {
          const StagedBase& B = sp[six[k][s].first];
          const StagedSlot& q = B.slots[six[k][s].second];
          const int SC = staged_cols(B, ts.tw, ts.tma);
          lv.push_back("sg" + std::to_string(six[k][s].first) + "[li * " + std::to_string(SC) + " + lj + " +
                       std::to_string((g.box[k][0] + q.dr - B.rlo) * SC + (g.box[k][2] + q.dc - B.clo)) + "]");
        } else if (ld.prod < 0) {
          lv.push_back(mem_slot("l", n, "const " + T, GL.lw[k][s], r.loads[s]));
        } else {
          const int pk = ld.prod;
          const int roff = g.box[k][0] + ld.dr - g.box[pk][0], coff = g.box[k][2] + ld.dc - g.box[pk][2];
          const int PBW = box_cols(g, pk, ts.tw);
          o << "      const " << T << "* sl" << n << " = (const " << T << "*)(vbe_smem + " << soff[pk][ld.prod_store]
            << ") + " << (roff * PBW + coff) << ";\n";
          lv.push_back("sl" + n + "[li * " + std::to_string(PBW) + " + lj]");
        }
      }
      for (size_t s = 0; s < r.stores.size(); ++s) {
        const std::string T = ctype(r.stores[s].dtype), n = std::to_string(s);
        if (g.consumed[k][s])
          o << "      " << T << "* ss" << n << " = (" << T << "*)(vbe_smem + " << soff[k][s] << ");\n";
        sm.push_back(k == anchor ? mem_slot("s", n, T, GL.sw[k][s], r.stores[s]) : "");
        sv.push_back("b" + n);
      }
      for (auto& pw : pat_word) {
        const std::string q = std::to_string(pw.first);
        o << "      const int pa" << q << " = (int)" << W(pw.second + 1);
        if (pats[pw.first][1] != 1) o << ", pb" << q << " = (int)" << W(pw.second + 2);
        o << ";\n";
      }
      for (size_t q = 0; q < cdecl[k].size(); ++q) {
        const std::string& d = cdecl[k][q];
        const size_t eq = d.find(" = ");
        o << "      const " << d.substr(0, eq) << " kc" << q << d.substr(eq) << ";\n";
      }
      // points of the box in row-major order, blockDim at a time, unrolled
      // (a compile-time trip count lets loads of several points overlap).
      // Tiles whose box lies inside the run's shape skip the bounds tests.
      const int NK = (BH * BW + ts.block - 1) / ts.block;
      const bool partial = NK * ts.block > BH * BW;
      auto body = [&](const std::string& ind) {
        for (auto& pw : pat_word) {
          const std::string q = std::to_string(pw.first);
          o << ind << "const int ix" << q << " = li * pa" << q << " + "
            << (pats[pw.first][1] == 1 ? std::string("lj") : "lj * pb" + q) << ";\n";
        }
        for (size_t s = 0; s < r.stores.size(); ++s) o << ind << ctype(r.stores[s].dtype) << " b" << s << ";\n";
        o << ind << "vbe_elem" << k << "(p, (r0 + li) * cols + (c0 + lj)";
        for (auto& x : lv) o << ", " << x;
        for (auto& x : sv) o << ", " << x;
        if (r.has_red) o << (gens[k]->kahan() ? ", acc, kc" : ", acc");
        for (size_t q = 0; q < r.consts.size(); ++q) o << ", kc" << q;
        o << ");\n";
        for (size_t s = 0; s < r.stores.size(); ++s) {
          if (g.consumed[k][s]) o << ind << "ss" << s << "[q] = b" << s << ";\n";
          if (k == anchor) o << ind << sm[s] << " = b" << s << ";\n";
        }
      };
      auto loop = [&](bool checked) {
        o << "#pragma unroll\n"
          << "        for (int kq = 0; kq < " << NK << "; ++kq) {\n"
          << "          const int q = threadIdx.x + kq * " << ts.block << ";\n"
          << "          const int li = q / " << BW << ", lj = q - li * " << BW << ";\n";
        std::string cond;
        if (partial) cond = "q < " + std::to_string(BH * BW);
        if (checked) {
          if (!cond.empty()) cond += " && ";
          cond += "r0 + li >= 0 && r0 + li < rows && c0 + lj >= 0 && c0 + lj < cols";
        }
        if (cond.empty()) {
          body("          ");
        } else {
          o << "          if (" << cond << ") {\n";
          body("            ");
          o << "          }\n";
        }
        o << "        }\n";
      };
      if (r.has_red) {
        gens[k]->o.str("");
        gens[k]->emit_acc_init("      ");
        o << gens[k]->o.str();
      }
      o << "      if (inside) {\n";
      loop(false);
      o << "      } else {\n";
      loop(true);
      o << "      }\n";
      if (r.has_red) {
        // each point of this run belongs to exactly one tile (no halo), so
        // block partials summed in block order give the whole reduction
        const int w = GL.red[k];
        gens[k]->o.str("");
        gens[k]->emit_full_epilogue("      ", W(w + 1), "blockIdx.x", W(w + 2), "gridDim.x", W(w));
        o << gens[k]->o.str();
      }
      if (k != anchor) o << (ts.tma ? "      vbe_bar_sync(1, " + std::to_string(ts.block) + ");\n" : "      __syncthreads();\n");
      o << "    }\n";
    }
    }
    if (ts.tma) {
      emit_tma_epilogue(o, g, ts);
      for (int k = 0; k < m; ++k)
        if (g.runs[k].has_red) {
          const int w = GL.red[k];
          gens[k]->o.str("");
          gens[k]->emit_full_epilogue("  ", W(w + 1), "blockIdx.x", W(w + 2), "gridDim.x", W(w));
          o << gens[k]->o.str();
        }
    }
    else o << "  }\n";
    emit_copy_through(o, g, GL);
    o << "}\n";
  }
  std::string src = o.str();
  std::string tag = "g" + std::to_string(m) + "_" + hex64(fnv1a(src.data(), src.size())).substr(8);
  for (size_t pos; (pos = src.find("@TAG@")) != std::string::npos;) src.replace(pos, 5, tag);
  if (entry_prefix) *entry_prefix = "vbe_" + tag;
  if (shapes_out) *shapes_out = shapes;
  return src;
}

void fill_group_words(const Group& g, const TileShape& ts, const std::vector<std::vector<uintptr_t>>& load_ptrs,
                      const std::vector<std::vector<uintptr_t>>& store_ptrs,
                      const std::vector<std::pair<uintptr_t, uintptr_t>>& renamed_ptrs,
                      const std::vector<uintptr_t>& red_ptrs, uintptr_t partials, uintptr_t counters, LaunchArgs* out,
                      uintptr_t err_word) {
  const int m = (int)g.runs.size();
  const int anchor = m - 1;
  GroupLayout GL = group_layout(g);
  std::vector<int64_t>& w = out->w;
  w.assign(GL.nwords, 0);
  const int64_t R = g.rows(anchor), C = g.cols(anchor);
  const int64_t tpr = (C + ts.tw - 1) / ts.tw;
  w[0] = R;
  w[1] = C;
  w[2] = tpr;
  w[3] = ((R + ts.th - 1) / ts.th) * tpr;
  for (int k = 0; k < m; ++k) {
    const Run& r = g.runs[k];
    w[GL.dims[k]] = r.shape[0];
    w[GL.dims[k] + 1] = r.shape[1];
    for (size_t s = 0; s < r.loads.size(); ++s) {
      int q = GL.lw[k][s];
      if (q < 0) continue;
      w[q] = (int64_t)(load_ptrs[k][s] + (uintptr_t)(r.loads[s].offset * itemsize(r.loads[s].dtype)));
      w[q + 1] = r.loads[s].st[0];
      w[q + 2] = r.loads[s].st[1];
    }
    for (size_t s = 0; s < r.stores.size(); ++s) {
      int q = GL.sw[k][s];
      if (q < 0) continue;
      w[q] = (int64_t)(store_ptrs[k][s] + (uintptr_t)(r.stores[s].offset * itemsize(r.stores[s].dtype)));
      w[q + 1] = r.stores[s].st[0];
      w[q + 2] = r.stores[s].st[1];
    }
    for (size_t q = 0; q < r.consts.size(); ++q) w[GL.consts[k] + q] = const_bits(r.consts[q]);
    int ri = 0;
    for (auto& st : r.steps) {
      if (st.op != VBE_OP_RANDOM) continue;
      w[GL.rnd[k] + 3 * ri] = (int64_t)st.seed;
      w[GL.rnd[k] + 3 * ri + 1] = (int64_t)st.key;
      w[GL.rnd[k] + 3 * ri + 2] = st.rstep;
      ++ri;
    }
  }
  for (size_t rr = 0; rr < g.renamed.size(); ++rr) {
    const Slot& st = g.runs[anchor].stores[g.renamed_slot[rr]];
    const int q = GL.ren[rr];
    w[q] = (int64_t)renamed_ptrs[rr].first;
    w[q + 1] = (int64_t)renamed_ptrs[rr].second;
    w[q + 2] = st.offset;
    w[q + 3] = st.st[0];
    w[q + 4] = R;
    w[q + 5] = C;
    w[q + 6] = g.renamed_nelem[rr] - R * C;
  }
  // staged inputs: the reference view's offset in its base and the base's
  // size; for tensor copies the box origin relative to the tile origin, its
  // column rounded down to a 16-byte boundary, and that rounding
  const std::vector<StagedBase> sp = staging_plan(g);
  for (size_t b = 0; b < sp.size(); ++b) {
    const Slot& ref = g.runs[sp[b].ref_k].loads[sp[b].ref_s];
    w[GL.stg[b]] = ref.offset;
    w[GL.stg[b] + 1] = g.base_nelem.at(sp[b].base);
    const int64_t P = ref.st[0], a = 16 / itemsize(sp[b].dtype);
    int64_t r_ref = ref.offset / P, c_ref = ref.offset % P;
    if (c_ref < 0) {
      c_ref += P;
      --r_ref;
    }
    const int64_t cx = sp[b].clo + c_ref;
    const int64_t dx = ((cx % a) + a) % a;
    w[GL.stg[b] + 2] = cx - dx;
    w[GL.stg[b] + 3] = sp[b].rlo + r_ref;
    w[GL.stg[b] + 4] = dx;
  }
  w[GL.err] = (int64_t)err_word;
  // reductions: one partial per block, a region and a completion counter per reducing run
  int nq = 0;
  for (int k = 0; k < m; ++k) {
    if (GL.red[k] < 0) continue;
    const Run& r = g.runs[k];
    w[GL.red[k]] = (int64_t)(red_ptrs[k] + (uintptr_t)(r.red_out.offset * itemsize(r.red_dtype)));
    w[GL.red[k] + 1] = (int64_t)(partials + (uintptr_t)(nq * w[3] * 8));
    w[GL.red[k] + 2] = (int64_t)(counters + (uintptr_t)(nq * 4));
    ++nq;
  }
}

std::vector<std::pair<const char*, const char*>> nvrtc_headers() {
  return {{"sf64_tables.h", kSf64Tables}, {"sf64.cuh", kSf64Code}};
}

}  // namespace vbe
