// mcore: a multi-core, blocked CPU interpreter of vector bytecode -- the
// paper's multi-core Vector Engine (section "Vector Engine" of the
// implementation, and the "mcore" engine of section "Performance Study"),
// restated as a CPU baseline for the GPU executor.
//
// It forms kernels exactly as that section describes: instructions are
// scanned in order and added to the current kernel while they are
// "blockable" with it (the new instruction's inputs share no data with the
// kernel's outputs, or represent precisely the same data; its output shares
// no data with the kernel's inputs and outputs, or the same data), and
// while they cover the same index space. A kernel is then executed block by
// block: its index space is cut into a user-chosen number of blocks, worker
// threads take blocks from a shared counter, and each block runs every
// instruction of the kernel in order before the next block starts, so a
// block's data stays in the core's cache. Axis reductions run as kernels of
// their own, blocked over their outputs.
//
// Semantics (the same as the reference interpreter's): NumPy ufunc rules;
// integers wrap modulo 2^64; float32 exp/log are evaluated in float64 and
// rounded once; float32 sums accumulate in float64; MAXIMUM / MINIMUM return
// the first operand when it wins the comparison or is NaN; ARGMIN / ARGMAX
// return the first extreme, a NaN counting as the extreme; an instruction
// whose output partially overlaps one of its inputs reads a copy of that
// input. RANDOM is the counter form of splitmix64 (Steele, Lea and Flood,
// "Fast splittable pseudorandom number generators", OOPSLA 2014).
//
// This is a baseline, not part of the GPU library: it shares no code with
// it or with the reference interpreter.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <mutex>
#include <cstdint>
#include <cstring>
#include <thread>
#include <type_traits>
#include <vector>

extern "C" {

enum { MC_BOOL = 0, MC_INT64 = 1, MC_FLOAT32 = 2, MC_FLOAT64 = 3 };

typedef struct mc_base {
  int32_t dtype;
  int32_t pad;
  int64_t nelem;
  void* data;  // caller-owned host memory of nelem elements
} mc_base;

typedef struct mc_view {
  int32_t base;  // index into the bases
  int32_t ndim;
  int64_t offset;
  int64_t shape[8];
  int64_t strides[8];
} mc_view;

typedef struct mc_instr {
  int32_t op;          // the library's opcode numbers (vbe.h)
  int32_t const_slot;  // -1 or the input slot holding the constant
  int32_t out;         // view index, -1 for none
  int32_t in[3];       // view indices, -1 unused
  int32_t axis;
  int32_t pad;
  double kf;           // the constant, for float dtypes
  int64_t ki;          // the constant, for int64 / bool
  uint64_t seed, key;
  int64_t step;
} mc_instr;

}  // extern "C"

namespace {

enum {
  ADD = 1, SUBTRACT, MULTIPLY, DIVIDE, MAXIMUM, MINIMUM, SQRT, EXP, LOG, ABSOLUTE, NEGATIVE, LESS, LESS_EQUAL,
  GREATER, GREATER_EQUAL, EQUAL, NOT_EQUAL, SELECT, CAST, COPY, RANDOM, ADD_REDUCE, MIN_REDUCE, MAX_REDUCE, SYNC,
  DISCARD, FREE, ARGMIN_REDUCE, ARGMAX_REDUCE
};

struct Fail {
  int code;
};

int isz(int dt) { return dt == MC_BOOL ? 1 : (dt == MC_FLOAT32 ? 4 : 8); }
bool is_reduce(int op) {
  return op == ADD_REDUCE || op == MIN_REDUCE || op == MAX_REDUCE || op == ARGMIN_REDUCE || op == ARGMAX_REDUCE;
}
bool is_control(int op) { return op == SYNC || op == DISCARD || op == FREE; }

// a view resolved to its base's memory
struct V {
  int base = -1, dtype = 0, ndim = 0;
  char* data = nullptr;
  int64_t offset = 0, shape[8] = {}, strides[8] = {}, size = 1, lo = 0, hi = -1;
};

V resolve(const mc_view& v, const mc_base* bases, int nbases) {
  if (v.base < 0 || v.base >= nbases || v.ndim < 0 || v.ndim > 8) throw Fail{-1};
  V r;
  r.base = v.base;
  r.dtype = bases[v.base].dtype;
  r.data = static_cast<char*>(bases[v.base].data);
  r.ndim = v.ndim;
  r.offset = v.offset;
  r.lo = r.hi = v.offset;
  for (int k = 0; k < v.ndim; ++k) {
    r.shape[k] = v.shape[k];
    r.strides[k] = v.strides[k];
    if (v.shape[k] < 0) throw Fail{-1};
    r.size *= v.shape[k];
    if (v.shape[k] > 0) {
      int64_t span = (v.shape[k] - 1) * v.strides[k];
      if (span < 0) r.lo += span;
      else r.hi += span;
    }
  }
  if (r.size > 0 && (r.lo < 0 || r.hi >= bases[v.base].nelem)) throw Fail{-2};
  if (r.size == 0) r.hi = r.lo - 1;
  return r;
}

bool same_mapping(const V& a, const V& b) {
  if (a.base != b.base || a.offset != b.offset || a.ndim != b.ndim) return false;
  for (int k = 0; k < a.ndim; ++k)
    if (a.shape[k] != b.shape[k] || (a.shape[k] > 1 && a.strides[k] != b.strides[k])) return false;
  return true;
}

// conservative: the reachable element ranges intersect
bool share_data(const V& a, const V& b) {
  if (a.base != b.base || a.size == 0 || b.size == 0) return false;
  return !(a.hi < b.lo || b.hi < a.lo);
}

bool self_overlapping(const V& v) {
  if (v.size <= 1) return false;
  std::vector<std::pair<int64_t, int64_t>> d;
  for (int k = 0; k < v.ndim; ++k)
    if (v.shape[k] > 1) d.push_back({std::llabs(v.strides[k]), v.shape[k]});
  std::sort(d.begin(), d.end());
  int64_t span = 0;
  for (auto& p : d) {
    if (p.first <= span) return true;
    span += p.first * (p.second - 1);
  }
  return false;
}

bool same_shape(const V& a, const V& b) {
  if (a.ndim != b.ndim) return false;
  for (int k = 0; k < a.ndim; ++k)
    if (a.shape[k] != b.shape[k]) return false;
  return true;
}

// ------------------------------------------------------------ operands
struct Operand {
  bool is_const = false;
  V v;
  double kf = 0;
  int64_t ki = 0;
  std::vector<char> copy;  // a private copy (partial overlap with the output)
};

template <class T>
inline T load(const Operand& o, int64_t elem) {
  return reinterpret_cast<const T*>(o.v.data)[elem];
}

// splitmix64 finaliser (the published mixing function of SplitMix64)
inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ull;

// ------------------------------------------------------- elementwise op
// value of operand o at the element whose offset into its base is `e`
struct Val {
  double f;
  int64_t i;
};

inline Val get(const Operand& o, int dt, int64_t e) {
  Val r{0, 0};
  if (o.is_const) {
    if (dt == MC_FLOAT64) r.f = o.kf;
    else if (dt == MC_FLOAT32) r.f = (double)(float)o.kf;
    else if (dt == MC_BOOL) r.i = o.ki != 0;
    else r.i = o.ki;
    return r;
  }
  switch (o.v.dtype) {
    case MC_FLOAT64: r.f = load<double>(o, e); break;
    case MC_FLOAT32: r.f = load<float>(o, e); break;
    case MC_INT64: r.i = load<int64_t>(o, e); break;
    default: r.i = load<uint8_t>(o, e) != 0; break;
  }
  return r;
}

inline void put(const V& out, int64_t e, Val v, bool is_float) {
  switch (out.dtype) {
    case MC_FLOAT64: reinterpret_cast<double*>(out.data)[e] = is_float ? v.f : (double)v.i; break;
    case MC_FLOAT32: reinterpret_cast<float*>(out.data)[e] = is_float ? (float)v.f : (float)v.i; break;
    case MC_INT64: reinterpret_cast<int64_t*>(out.data)[e] = is_float ? (int64_t)v.f : v.i; break;
    default: reinterpret_cast<uint8_t*>(out.data)[e] = is_float ? (v.f != 0.0) : (v.i != 0); break;
  }
}

inline int64_t wrap_add(int64_t a, int64_t b) { return (int64_t)((uint64_t)a + (uint64_t)b); }
inline int64_t wrap_sub(int64_t a, int64_t b) { return (int64_t)((uint64_t)a - (uint64_t)b); }
inline int64_t wrap_mul(int64_t a, int64_t b) { return (int64_t)((uint64_t)a * (uint64_t)b); }

struct Ins {
  mc_instr raw;
  int op;
  V out;
  int nin = 0;
  Operand in[3];
  int in_dt = 0;  // dtype of the arithmetic inputs
  void (*seg)(const Ins&, int64_t, int64_t, const int64_t*) = nullptr;  // typed loop, if any
};

// apply one elementwise instruction to row-major flat indices [lo, hi)
void apply_elem(const Ins& I, int64_t lo, int64_t hi) {
  const V& o = I.out;
  int64_t idx[8];
  int64_t rem = lo;
  for (int k = o.ndim - 1; k >= 0; --k) {
    idx[k] = o.shape[k] ? rem % o.shape[k] : 0;
    rem = o.shape[k] ? rem / o.shape[k] : 0;
  }
  // element offsets of the output and every view input, kept incrementally
  int64_t eo = o.offset, ei[3] = {0, 0, 0};
  const V* iv[3] = {nullptr, nullptr, nullptr};
  for (int j = 0; j < I.nin; ++j)
    if (!I.in[j].is_const) {
      iv[j] = &I.in[j].v;
      ei[j] = iv[j]->offset;
    }
  for (int k = 0; k < o.ndim; ++k) {
    eo += idx[k] * o.strides[k];
    for (int j = 0; j < I.nin; ++j)
      if (iv[j]) ei[j] += idx[k] * iv[j]->strides[k];
  }
  const bool fin = I.in_dt == MC_FLOAT32 || I.in_dt == MC_FLOAT64;
  const bool f32 = I.raw.op != CAST && I.out.dtype == MC_FLOAT32;
  for (int64_t t = lo; t < hi; ++t) {
    Val a = I.nin > 0 ? get(I.in[0], I.op == SELECT ? MC_BOOL : I.in_dt, ei[0]) : Val{0, 0};
    Val b = I.nin > 1 ? get(I.in[1], I.op == SELECT ? o.dtype : I.in_dt, ei[1]) : Val{0, 0};
    Val r{0, 0};
    bool rf = fin;
    switch (I.op) {
      case ADD: if (fin) r.f = a.f + b.f; else r.i = wrap_add(a.i, b.i); break;
      case SUBTRACT: if (fin) r.f = a.f - b.f; else r.i = wrap_sub(a.i, b.i); break;
      case MULTIPLY: if (fin) r.f = a.f * b.f; else r.i = wrap_mul(a.i, b.i); break;
      case DIVIDE: r.f = a.f / b.f; break;
      case MAXIMUM: if (fin) r.f = (a.f > b.f || std::isnan(a.f)) ? a.f : b.f; else r.i = a.i > b.i ? a.i : b.i; break;
      case MINIMUM: if (fin) r.f = (a.f < b.f || std::isnan(a.f)) ? a.f : b.f; else r.i = a.i < b.i ? a.i : b.i; break;
      case SQRT: r.f = std::sqrt(a.f); break;
      case EXP: r.f = std::exp(a.f); break;
      case LOG: r.f = std::log(a.f); break;
      case ABSOLUTE: if (fin) r.f = std::fabs(a.f); else r.i = a.i < 0 ? wrap_sub(0, a.i) : a.i; break;
      case NEGATIVE: if (fin) r.f = -a.f; else r.i = wrap_sub(0, a.i); break;
      case LESS: rf = false; r.i = fin ? a.f < b.f : a.i < b.i; break;
      case LESS_EQUAL: rf = false; r.i = fin ? a.f <= b.f : a.i <= b.i; break;
      case GREATER: rf = false; r.i = fin ? a.f > b.f : a.i > b.i; break;
      case GREATER_EQUAL: rf = false; r.i = fin ? a.f >= b.f : a.i >= b.i; break;
      case EQUAL: rf = false; r.i = fin ? a.f == b.f : a.i == b.i; break;
      case NOT_EQUAL: rf = false; r.i = fin ? a.f != b.f : a.i != b.i; break;
      case SELECT: {
        Val c = get(I.in[2], o.dtype, ei[2]);
        rf = o.dtype == MC_FLOAT32 || o.dtype == MC_FLOAT64;
        r = a.i ? b : c;
        break;
      }
      case CAST:
      case COPY: r = a; break;
      case RANDOM: {
        uint64_t m = (uint64_t)t;
        uint64_t z = mix64(I.raw.seed + (I.raw.key + (uint64_t)I.raw.step * m + 1) * kGamma);
        r.f = (double)(z >> 11) * 0x1p-53;
        rf = true;
        break;
      }
      default: throw Fail{-1};
    }
    if (f32 && rf && (I.op == EXP || I.op == LOG)) r.f = (double)(float)r.f;  // once, from float64
    if (I.op == CAST && o.dtype == MC_BOOL) {
      r.i = fin ? (a.f != 0.0) : (a.i != 0);
      rf = false;
    }
    put(o, eo, r, rf);
    // advance the row-major index
    for (int k = o.ndim - 1; k >= 0; --k) {
      eo += o.strides[k];
      for (int j = 0; j < I.nin; ++j)
        if (iv[j]) ei[j] += iv[j]->strides[k];
      if (++idx[k] < o.shape[k]) break;
      eo -= o.strides[k] * o.shape[k];
      for (int j = 0; j < I.nin; ++j)
        if (iv[j]) ei[j] -= iv[j]->strides[k] * o.shape[k];
      idx[k] = 0;
    }
  }
}

// ----------------------------------------------------- typed segments
// The common operations run over a row segment (consecutive indices along
// the innermost dimension) in a loop typed on the element type, with the
// operation fixed at compile time; a constant operand is a stride-0 input.

typedef void (*SegFn)(const Ins& I, int64_t n, int64_t eo, const int64_t* ei);

template <class T>
inline T const_as(const Operand& o) {
  if (std::is_floating_point<T>::value) return (T)o.kf;
  return (T)o.ki;
}

template <class T>
struct Src {
  const T* p;
  int64_t s;
  T k;
};

template <class T>
inline Src<T> src(const Ins& I, int j, int64_t e, int nd) {
  Src<T> r{nullptr, 0, T()};
  if (I.in[j].is_const) {
    r.k = const_as<T>(I.in[j]);
  } else {
    r.p = reinterpret_cast<const T*>(I.in[j].v.data) + e;
    r.s = nd ? I.in[j].v.strides[nd - 1] : 0;
  }
  return r;
}

template <class T>
inline T at(const Src<T>& a, int64_t i) {
  return a.p ? a.p[i * a.s] : a.k;
}

template <class T, int OP>
void seg_binary(const Ins& I, int64_t n, int64_t eo, const int64_t* ei) {
  const int nd = I.out.ndim;
  T* o = reinterpret_cast<T*>(I.out.data) + eo;
  const int64_t so = nd ? I.out.strides[nd - 1] : 0;
  Src<T> a = src<T>(I, 0, ei[0], nd), b = src<T>(I, 1, ei[1], nd);
  for (int64_t i = 0; i < n; ++i) {
    T x = at(a, i), y = at(b, i), r;
    if (OP == ADD) r = x + y;
    else if (OP == SUBTRACT) r = x - y;
    else if (OP == MULTIPLY) r = x * y;
    else if (OP == DIVIDE) r = x / y;
    else if (OP == MAXIMUM) r = (x > y || x != x) ? x : y;
    else r = (x < y || x != x) ? x : y;  // MINIMUM
    o[i * so] = r;
  }
}

template <class T, int OP>
void seg_unary(const Ins& I, int64_t n, int64_t eo, const int64_t* ei) {
  const int nd = I.out.ndim;
  T* o = reinterpret_cast<T*>(I.out.data) + eo;
  const int64_t so = nd ? I.out.strides[nd - 1] : 0;
  Src<T> a = src<T>(I, 0, ei[0], nd);
  for (int64_t i = 0; i < n; ++i) {
    T x = at(a, i), r;
    if (OP == SQRT) r = std::sqrt(x);
    else if (OP == EXP) r = (T)std::exp((double)x);  // float32: in float64, rounded once
    else if (OP == LOG) r = (T)std::log((double)x);
    else if (OP == ABSOLUTE) r = std::fabs(x);
    else if (OP == NEGATIVE) r = -x;
    else r = x;  // COPY
    o[i * so] = r;
  }
}

template <class T, int OP>
void seg_compare(const Ins& I, int64_t n, int64_t eo, const int64_t* ei) {
  const int nd = I.out.ndim;
  uint8_t* o = reinterpret_cast<uint8_t*>(I.out.data) + eo;
  const int64_t so = nd ? I.out.strides[nd - 1] : 0;
  Src<T> a = src<T>(I, 0, ei[0], nd), b = src<T>(I, 1, ei[1], nd);
  for (int64_t i = 0; i < n; ++i) {
    T x = at(a, i), y = at(b, i);
    bool r;
    if (OP == LESS) r = x < y;
    else if (OP == LESS_EQUAL) r = x <= y;
    else if (OP == GREATER) r = x > y;
    else if (OP == GREATER_EQUAL) r = x >= y;
    else if (OP == EQUAL) r = x == y;
    else r = x != y;
    o[i * so] = r;
  }
}

template <class T>
void seg_select(const Ins& I, int64_t n, int64_t eo, const int64_t* ei) {
  const int nd = I.out.ndim;
  T* o = reinterpret_cast<T*>(I.out.data) + eo;
  const int64_t so = nd ? I.out.strides[nd - 1] : 0;
  Src<uint8_t> c = src<uint8_t>(I, 0, ei[0], nd);
  if (I.in[0].is_const) c.k = I.in[0].ki != 0;
  Src<T> a = src<T>(I, 1, ei[1], nd), b = src<T>(I, 2, ei[2], nd);
  for (int64_t i = 0; i < n; ++i) o[i * so] = at(c, i) ? at(a, i) : at(b, i);
}

template <class T>
SegFn pick_typed(int op) {
  switch (op) {
    case ADD: return seg_binary<T, ADD>;
    case SUBTRACT: return seg_binary<T, SUBTRACT>;
    case MULTIPLY: return seg_binary<T, MULTIPLY>;
    case DIVIDE: return std::is_floating_point<T>::value ? seg_binary<T, DIVIDE> : nullptr;
    case MAXIMUM: return seg_binary<T, MAXIMUM>;
    case MINIMUM: return seg_binary<T, MINIMUM>;
    case SQRT: return std::is_floating_point<T>::value ? seg_unary<T, SQRT> : nullptr;
    case EXP: return std::is_floating_point<T>::value ? seg_unary<T, EXP> : nullptr;
    case LOG: return std::is_floating_point<T>::value ? seg_unary<T, LOG> : nullptr;
    case ABSOLUTE: return std::is_floating_point<T>::value ? seg_unary<T, ABSOLUTE> : nullptr;
    case NEGATIVE: return std::is_floating_point<T>::value ? seg_unary<T, NEGATIVE> : nullptr;
    case COPY: return seg_unary<T, COPY>;
    case LESS: return seg_compare<T, LESS>;
    case LESS_EQUAL: return seg_compare<T, LESS_EQUAL>;
    case GREATER: return seg_compare<T, GREATER>;
    case GREATER_EQUAL: return seg_compare<T, GREATER_EQUAL>;
    case EQUAL: return seg_compare<T, EQUAL>;
    case NOT_EQUAL: return seg_compare<T, NOT_EQUAL>;
    case SELECT: return seg_select<T>;
    default: return nullptr;
  }
}

// the typed loop of an instruction, or nullptr for the generic path
// (integer arithmetic, which must wrap, casts, RANDOM, booleans)
SegFn pick_seg(const Ins& I) {
  const int dt = I.op == SELECT || I.op == COPY ? I.out.dtype : I.in_dt;
  if (I.op == SELECT && I.nin == 3 && !I.in[0].is_const && I.in[0].v.dtype != MC_BOOL) return nullptr;
  for (int j = 0; j < I.nin; ++j) {
    if (I.in[j].is_const) continue;
    if (I.op == SELECT && j == 0) continue;
    if (I.in[j].v.dtype != dt) return nullptr;
  }
  const bool cmp = I.op >= LESS && I.op <= NOT_EQUAL;
  if (!cmp && I.out.dtype != dt) return nullptr;
  if (dt == MC_FLOAT64) return pick_typed<double>(I.op);
  if (dt == MC_FLOAT32) return pick_typed<float>(I.op);
  if (dt == MC_INT64 && (cmp || I.op == COPY || I.op == SELECT || I.op == MAXIMUM || I.op == MINIMUM))
    return pick_typed<int64_t>(I.op);
  return nullptr;
}

// run an instruction over flat indices [lo, hi) one row segment at a time
void apply_segments(const Ins& I, SegFn fn, int64_t lo, int64_t hi) {
  const V& o = I.out;
  const int nd = o.ndim;
  int64_t idx[8];
  int64_t rem = lo;
  for (int k = nd - 1; k >= 0; --k) {
    idx[k] = o.shape[k] ? rem % o.shape[k] : 0;
    rem = o.shape[k] ? rem / o.shape[k] : 0;
  }
  int64_t eo = o.offset, ei[3] = {0, 0, 0};
  for (int j = 0; j < I.nin; ++j)
    if (!I.in[j].is_const) ei[j] = I.in[j].v.offset;
  for (int k = 0; k < nd; ++k) {
    eo += idx[k] * o.strides[k];
    for (int j = 0; j < I.nin; ++j)
      if (!I.in[j].is_const) ei[j] += idx[k] * I.in[j].v.strides[k];
  }
  int64_t t = lo;
  while (t < hi) {
    const int64_t n = nd ? std::min(hi - t, o.shape[nd - 1] - idx[nd - 1]) : 1;
    fn(I, n, eo, ei);
    t += n;
    if (nd == 0) break;
    // advance the row-major index by n: the innermost dimension first
    int k = nd - 1;
    idx[k] += n;
    eo += n * o.strides[k];
    for (int j = 0; j < I.nin; ++j)
      if (!I.in[j].is_const) ei[j] += n * I.in[j].v.strides[k];
    while (k > 0 && idx[k] == o.shape[k]) {
      eo -= o.strides[k] * o.shape[k];
      for (int j = 0; j < I.nin; ++j)
        if (!I.in[j].is_const) ei[j] -= I.in[j].v.strides[k] * o.shape[k];
      idx[k] = 0;
      --k;
      ++idx[k];
      eo += o.strides[k];
      for (int j = 0; j < I.nin; ++j)
        if (!I.in[j].is_const) ei[j] += I.in[j].v.strides[k];
    }
  }
}

// ------------------------------------------------------------ reduction
// out[kept index] = reduce over axis of in; blocked over the outputs
void apply_reduce(const Ins& I, int64_t lo, int64_t hi) {
  const V& x = I.in[0].v;
  const V& o = I.out;
  const int ax = I.raw.axis;
  const int64_t n = x.shape[ax], st = x.strides[ax];
  int kept[8], nk = 0;
  for (int k = 0; k < x.ndim; ++k)
    if (k != ax) kept[nk++] = k;
  const bool fin = x.dtype == MC_FLOAT32 || x.dtype == MC_FLOAT64;
  for (int64_t t = lo; t < hi; ++t) {
    int64_t rem = t, ex = x.offset, eo = o.offset;
    for (int j = nk - 1; j >= 0; --j) {
      int64_t s = o.shape[j], q = s ? rem % s : 0;
      rem = s ? rem / s : 0;
      ex += q * x.strides[kept[j]];
      eo += q * o.strides[j];
    }
    Val r{0, 0};
    bool rf = fin;
    if (I.op == ADD_REDUCE) {
      if (x.dtype == MC_FLOAT64) {
        const double* px = reinterpret_cast<const double*>(x.data) + ex;
        double acc = 0.0;
        for (int64_t m = 0; m < n; ++m) acc += px[m * st];
        r.f = acc;
      } else if (x.dtype == MC_FLOAT32) {
        const float* px = reinterpret_cast<const float*>(x.data) + ex;
        double acc = 0.0;  // float32 sums accumulate in float64
        for (int64_t m = 0; m < n; ++m) acc += (double)px[m * st];
        r.f = acc;
      } else if (fin) {
        double acc = 0.0;
        for (int64_t m = 0; m < n; ++m) acc += get(I.in[0], x.dtype, ex + m * st).f;
        r.f = acc;
      } else {
        int64_t acc = 0;
        for (int64_t m = 0; m < n; ++m) acc = wrap_add(acc, get(I.in[0], x.dtype, ex + m * st).i);
        r.i = acc;
      }
    } else if (I.op == MIN_REDUCE || I.op == MAX_REDUCE) {
      const bool mx = I.op == MAX_REDUCE;
      Val acc = get(I.in[0], x.dtype, ex);
      for (int64_t m = 1; m < n; ++m) {
        Val v = get(I.in[0], x.dtype, ex + m * st);
        if (fin) {
          bool keep = mx ? (acc.f > v.f || std::isnan(acc.f)) : (acc.f < v.f || std::isnan(acc.f));
          if (!keep) acc = v;
        } else if (mx ? v.i > acc.i : v.i < acc.i) {
          acc = v;
        }
      }
      r = acc;
    } else {  // ARGMIN / ARGMAX: the first extreme; a NaN is the extreme
      const bool mx = I.op == ARGMAX_REDUCE;
      int64_t best = 0;
      Val bv = get(I.in[0], x.dtype, ex);
      for (int64_t m = 1; m < n; ++m) {
        if (fin && std::isnan(bv.f)) break;
        Val v = get(I.in[0], x.dtype, ex + m * st);
        bool better = fin ? (std::isnan(v.f) || (mx ? v.f > bv.f : v.f < bv.f)) : (mx ? v.i > bv.i : v.i < bv.i);
        if (better) {
          best = m;
          bv = v;
        }
      }
      r.i = best;
      rf = false;
    }
    put(o, eo, r, rf);
  }
}

// ------------------------------------------------------------- kernels
struct Kernel {
  std::vector<int> ins;  // indices into the instruction list
  int64_t space = 0;     // index-space size (elements, or reduction outputs)
  bool reduce = false;
};

// the paper's two blockable properties, plus a common index space
bool blockable(const Kernel& k, const std::vector<Ins>& I, const Ins& n) {
  if (k.reduce || is_reduce(n.op)) return false;
  const Ins& first = I[k.ins[0]];
  if (!same_shape(first.out, n.out)) return false;
  for (int a : k.ins) {
    const V& ao = I[a].out;
    for (int j = 0; j < n.nin; ++j) {  // 1. inputs of N vs outputs of A
      if (n.in[j].is_const) continue;
      const V& ni = n.in[j].v;
      if (share_data(ni, ao) && !same_mapping(ni, ao)) return false;
    }
    // 2. output of N vs inputs and outputs of A
    if (share_data(n.out, ao) && !same_mapping(n.out, ao)) return false;
    for (int j = 0; j < I[a].nin; ++j) {
      if (I[a].in[j].is_const) continue;
      const V& ai = I[a].in[j].v;
      if (share_data(n.out, ai) && !same_mapping(n.out, ai)) return false;
    }
  }
  return true;
}

// Worker threads for one mcore_run call: each kernel is handed to all of
// them, and they take its blocks from a shared counter until none is left.
class Pool {
 public:
  // kernels of fewer than `inline_below` element-operations run on the
  // calling thread alone (too little work to wake the others for)
  Pool(int n, int64_t inline_below) : inline_below_(inline_below) {
    for (int t = 1; t < n; ++t) th_.emplace_back([this] { loop(); });
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  void run(const Kernel& k, const std::vector<Ins>& I, int64_t nblocks) {
    if (k.space <= 0) return;
    nb_ = std::max<int64_t>(1, std::min<int64_t>(nblocks, k.space));
    bs_ = (k.space + nb_ - 1) / nb_;
    k_ = &k;
    I_ = &I;
    next_.store(0);
    failed_.store(0);
    if (th_.empty() || k.space * (int64_t)k.ins.size() < inline_below_) {
      work();
      if (failed_.load()) throw Fail{failed_.load()};
      return;
    }
    {
      std::lock_guard<std::mutex> lk(mu_);
      ++gen_;
      busy_ = (int)th_.size();
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [this] { return busy_ == 0; });
    if (failed_.load()) throw Fail{failed_.load()};
  }

 private:
  void work() {
    try {
      for (;;) {
        int64_t b = next_.fetch_add(1);
        if (b >= nb_ || failed_.load()) return;
        const int64_t lo = b * bs_, hi = std::min(k_->space, lo + bs_);
        for (int i : k_->ins) {
          const Ins& x = (*I_)[i];
          if (k_->reduce) apply_reduce(x, lo, hi);
          else if (x.seg) apply_segments(x, x.seg, lo, hi);
          else apply_elem(x, lo, hi);
        }
      }
    } catch (const Fail& f) {
      failed_.store(f.code);
    }
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
      }
      work();
      std::lock_guard<std::mutex> lk(mu_);
      if (--busy_ == 0) done_.notify_one();
    }
  }
  int64_t inline_below_ = 0;
  std::vector<std::thread> th_;
  std::mutex mu_;
  std::condition_variable cv_, done_;
  bool stop_ = false;
  uint64_t gen_ = 0;
  int busy_ = 0;
  const Kernel* k_ = nullptr;
  const std::vector<Ins>* I_ = nullptr;
  int64_t nb_ = 1, bs_ = 1;
  std::atomic<int64_t> next_{0};
  std::atomic<int> failed_{0};
};

}  // namespace

extern "C" {

// Execute ninstrs instructions in order on the bases' host memory with
// nthreads worker threads and (up to) nblocks data blocks per kernel; a
// kernel of fewer than inline_below element-operations runs on the calling
// thread alone.
// Returns 0, -1 (an invalid instruction or operand), -2 (a view outside its
// base), -3 (unsupported operation). *nkernels receives the kernels formed.
int mcore_run(const mc_base* bases, int32_t nbases, const mc_view* views, int32_t nviews, const mc_instr* instrs,
              int32_t ninstrs, int32_t nthreads, int64_t nblocks, int64_t inline_below, int64_t* nkernels) {
  try {
    if (nthreads < 1 || nblocks < 1) return -1;
    std::vector<Ins> I;
    I.reserve(ninstrs);  // no reallocation: operands keep their copies in place
    int64_t kernels = 0;
    std::vector<Kernel> cur;
    Pool pool(nthreads, inline_below);
    auto flush = [&]() {
      for (auto& k : cur) pool.run(k, I, nblocks);
      kernels += (int64_t)cur.size();
      cur.clear();
    };
    for (int32_t i = 0; i < ninstrs; ++i) {
      const mc_instr& m = instrs[i];
      Ins x;
      x.raw = m;
      x.op = m.op;
      if (m.op < ADD || m.op > ARGMAX_REDUCE) return -3;
      if (is_control(m.op)) {
        // SYNC, DISCARD and FREE end the current kernel; the caller owns the
        // memory, so they need no other action here
        flush();
        I.push_back(x);
        continue;
      }
      if (m.out < 0 || m.out >= nviews) return -1;
      x.out = resolve(views[m.out], bases, nbases);
      if (self_overlapping(x.out)) return -1;
      for (int j = 0; j < 3; ++j) {
        if (j == m.const_slot) {
          x.in[j].is_const = true;
          x.in[j].kf = m.kf;
          x.in[j].ki = m.ki;
          x.nin = j + 1;
        } else if (m.in[j] >= 0) {
          if (m.in[j] >= nviews) return -1;
          x.in[j].v = resolve(views[m.in[j]], bases, nbases);
          x.nin = j + 1;
        }
      }
      x.in_dt = x.out.dtype;
      for (int j = 0; j < x.nin; ++j)
        if (!x.in[j].is_const && !(m.op == SELECT && j == 0)) {
          x.in_dt = x.in[j].v.dtype;
          break;
        }
      I.push_back(x);
      Ins& y = I.back();
      if (!is_reduce(y.op)) y.seg = pick_seg(y);
      // an output that partially overlaps an input: that input is read from
      // a private copy, taken right before the instruction runs
      bool own = false;
      for (int j = 0; j < y.nin; ++j)
        if (!y.in[j].is_const && share_data(y.in[j].v, y.out) && !same_mapping(y.in[j].v, y.out)) own = true;
      int64_t space = y.out.size;
      if (is_reduce(y.op)) {
        if (y.nin != 1 || y.in[0].is_const || y.raw.axis < 0 || y.raw.axis >= y.in[0].v.ndim) return -1;
        if ((y.op == MIN_REDUCE || y.op == MAX_REDUCE || y.op == ARGMIN_REDUCE || y.op == ARGMAX_REDUCE) &&
            y.in[0].v.shape[y.raw.axis] == 0)
          return -1;
      }
      const int idx = (int)I.size() - 1;
      if (!own && !cur.empty() && blockable(cur.back(), I, y)) {
        cur.back().ins.push_back(idx);
        continue;
      }
      flush();
      Kernel k;
      k.ins.push_back(idx);
      k.space = space;
      k.reduce = is_reduce(y.op);
      cur.push_back(k);
      if (own) {
        // every earlier kernel has run (flushed above): copy and run now
        for (int j = 0; j < y.nin; ++j) {
          Operand& o = y.in[j];
          if (o.is_const || !share_data(o.v, y.out) || same_mapping(o.v, y.out)) continue;
          const int s = isz(o.v.dtype);
          o.copy.resize((size_t)(o.v.hi - o.v.lo + 1) * s);
          std::memcpy(o.copy.data(), o.v.data + o.v.lo * s, o.copy.size());
          // the copy stands for elements lo..hi of the base: rebase the view
          o.v.data = o.copy.data();
          o.v.offset -= o.v.lo;
          o.v.hi -= o.v.lo;
          o.v.lo = 0;
        }
        flush();
      }
    }
    flush();
    if (nkernels) *nkernels = kernels;
    return 0;
  } catch (const Fail& f) {
    return f.code;
  }
}

}  // extern "C"
