// Bytecode IR: dtype and opcode tables, view geometry, overlap test and
// batch validation.
//
// The opcode set and its operand counts follow the paper's section
// "Bytecode" (one opcode per mnemonic, the opcode fixes the number of
// operands, operands are multidimensional arrays). Views follow section
// "Numerical Python" (array-base / array-view).
#include <algorithm>
#include <cctype>
#include <deque>
#include <mutex>
#include <cstring>
#include <numeric>
#include <set>
#include <sstream>

#include "vbe_core.h"

namespace vbe {

void fail(int code, const std::string& msg) { throw Error{code, msg}; }

void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    fail(e == cudaErrorMemoryAllocation ? VBE_ERR_OOM : VBE_ERR_CUDA,
         std::string(what) + ": " + cudaGetErrorString(e));
  }
}

int itemsize(int dt) {
  switch (dt) {
    case VBE_BOOL: return 1;
    case VBE_INT64: return 8;
    case VBE_FLOAT32: return 4;
    case VBE_FLOAT64: return 8;
  }
  fail(VBE_ERR_INVALID, "unknown dtype " + std::to_string(dt));
}

const char* ctype(int dt) {
  switch (dt) {
    case VBE_BOOL: return "bool";
    case VBE_INT64: return "long long";
    case VBE_FLOAT32: return "float";
    case VBE_FLOAT64: return "double";
  }
  return "?";
}

const char* dtype_name(int dt) {
  switch (dt) {
    case VBE_BOOL: return "bool";
    case VBE_INT64: return "int64";
    case VBE_FLOAT32: return "float32";
    case VBE_FLOAT64: return "float64";
  }
  return "?";
}

bool is_float(int dt) { return dt == VBE_FLOAT32 || dt == VBE_FLOAT64; }

OpKind op_kind(int op) {
  switch (op) {
    case VBE_OP_ADD: case VBE_OP_SUBTRACT: case VBE_OP_MULTIPLY:
    case VBE_OP_MAXIMUM: case VBE_OP_MINIMUM: return K_ARITH;
    case VBE_OP_DIVIDE: return K_DIV;
    case VBE_OP_SQRT: case VBE_OP_EXP: case VBE_OP_LOG: return K_FUNARY;
    case VBE_OP_ABSOLUTE: case VBE_OP_NEGATIVE: return K_SUNARY;
    case VBE_OP_LESS: case VBE_OP_LESS_EQUAL: case VBE_OP_GREATER: case VBE_OP_GREATER_EQUAL:
    case VBE_OP_EQUAL: case VBE_OP_NOT_EQUAL: return K_CMP;
    case VBE_OP_SELECT: return K_SELECT;
    case VBE_OP_CAST: return K_CAST;
    case VBE_OP_COPY: return K_COPY;
    case VBE_OP_RANDOM: return K_RANDOM;
    case VBE_OP_ADD_REDUCE: case VBE_OP_MIN_REDUCE: case VBE_OP_MAX_REDUCE: return K_REDUCE;
    case VBE_OP_ARGMIN_REDUCE: case VBE_OP_ARGMAX_REDUCE: return K_REDUCE;
    case VBE_OP_SYNC: case VBE_OP_DISCARD: case VBE_OP_FREE: return K_CONTROL;
  }
  if (user_op(op)) return K_USER;
  fail(VBE_ERR_INVALID, "unknown opcode " + std::to_string(op));
}

// ------------------------------------------------ user-defined operations

namespace {
std::mutex g_user_mu;
std::deque<UserOp> g_user_ops;  // stable addresses
constexpr int kMaxUserOps = 1024;
}  // namespace

const UserOp* user_op(int op) {
  if (op < VBE_OP_USER_BASE) return nullptr;
  std::lock_guard<std::mutex> lk(g_user_mu);
  const size_t i = (size_t)(op - VBE_OP_USER_BASE);
  return i < g_user_ops.size() ? &g_user_ops[i] : nullptr;
}

int register_user_op(const std::string& name, const std::string& body, int nin, int dtype) {
  bool ok = !name.empty() && name.size() <= 48 && (isalpha((unsigned char)name[0]) || name[0] == '_');
  for (char ch : name) ok = ok && (isalnum((unsigned char)ch) || ch == '_');
  if (!ok) fail(VBE_ERR_INVALID, "operation name must be an identifier of at most 48 characters");
  if (nin < 1 || nin > 3) fail(VBE_ERR_INVALID, "a user operation takes 1 to 3 inputs");
  if (dtype != VBE_FLOAT32 && dtype != VBE_FLOAT64 && dtype != VBE_INT64)
    fail(VBE_ERR_INVALID, "a user operation works on float32, float64 or int64");
  std::lock_guard<std::mutex> lk(g_user_mu);
  for (size_t i = 0; i < g_user_ops.size(); ++i) {
    const UserOp& u = g_user_ops[i];
    if (u.name != name) continue;
    if (u.body == body && u.nin == nin && u.dtype == dtype) return VBE_OP_USER_BASE + (int)i;
    fail(VBE_ERR_INVALID, "operation " + name + " is registered with another definition");
  }
  if ((int)g_user_ops.size() >= kMaxUserOps) fail(VBE_ERR_INVALID, "user operation table is full");
  UserOp u;
  u.name = name;
  u.body = body;
  u.nin = nin;
  u.dtype = dtype;
  g_user_ops.push_back(u);
  return VBE_OP_USER_BASE + (int)g_user_ops.size() - 1;
}

int op_arity(int op) {
  switch (op_kind(op)) {
    case K_ARITH: case K_DIV: case K_CMP: return 2;
    case K_FUNARY: case K_SUNARY: case K_CAST: case K_COPY: case K_REDUCE: return 1;
    case K_SELECT: return 3;
    case K_RANDOM: case K_CONTROL: return 0;
    case K_USER: return user_op(op)->nin;
  }
  return 0;
}

const char* op_name(int op) {
  static const char* names[] = {"?", "ADD", "SUBTRACT", "MULTIPLY", "DIVIDE", "MAXIMUM", "MINIMUM",
                                "SQRT", "EXP", "LOG", "ABSOLUTE", "NEGATIVE", "LESS", "LESS_EQUAL",
                                "GREATER", "GREATER_EQUAL", "EQUAL", "NOT_EQUAL", "SELECT", "CAST",
                                "COPY", "RANDOM", "ADD_REDUCE", "MIN_REDUCE", "MAX_REDUCE", "SYNC",
                                "DISCARD", "FREE", "ARGMIN_REDUCE", "ARGMAX_REDUCE"};
  if (const UserOp* u = user_op(op)) return u->name.c_str();
  if (op < 1 || op > VBE_OP_ARGMAX_REDUCE) return "?";
  return names[op];
}

// ------------------------------------------------------------------ views

int64_t ViewDesc::size() const {
  int64_t n = 1;
  for (int k = 0; k < ndim; ++k) n *= shape[k];
  return n;
}

bool ViewDesc::same_shape(const ViewDesc& o) const {
  if (ndim != o.ndim) return false;
  for (int k = 0; k < ndim; ++k)
    if (shape[k] != o.shape[k]) return false;
  return true;
}

bool ViewDesc::identical(const ViewDesc& o) const {
  if (base != o.base || offset != o.offset || !same_shape(o)) return false;
  for (int k = 0; k < ndim; ++k)
    if (shape[k] > 1 && strides[k] != o.strides[k]) return false;
  return true;
}

void ViewDesc::finish() {
  if (size() == 0) {
    lo = 0;
    hi = -1;
    return;
  }
  lo = hi = offset;
  for (int k = 0; k < ndim; ++k) {
    int64_t e = (shape[k] - 1) * strides[k];
    if (e < 0) lo += e; else hi += e;
  }
}

bool ViewDesc::self_overlapping() const {
  if (size() <= 1) return false;
  std::vector<std::pair<int64_t, int64_t>> d;
  for (int k = 0; k < ndim; ++k)
    if (shape[k] > 1) d.push_back({std::llabs(strides[k]), shape[k]});
  std::sort(d.begin(), d.end());
  int64_t span = 0;
  for (auto& p : d) {
    if (p.first <= span) return true;
    span += p.first * (p.second - 1);
  }
  return false;
}

// Exact overlap test for views whose strides form a divisibility chain.
// Each view is normalised (size-1 and stride-0 dimensions dropped, negative
// strides flipped); the union of the two stride sets, sorted s_0 > s_1 >
// ... plus an implicit stride 1, defines mixed-radix digits. When every
// stride divides the next larger one and neither view carries across a
// digit, an element's address determines its digits uniquely, so the views
// overlap exactly when their boxes of digits intersect. Otherwise the
// answer is the conservative "may overlap".
namespace {
struct NormDim {
  int64_t s, n;
};
// dims: at most VBE_MAX_NDIM entries, sorted by decreasing stride
bool normalise(const ViewDesc& v, int64_t* off, NormDim* dims, int* nd) {
  *off = v.offset;
  int n = 0;
  for (int k = 0; k < v.ndim; ++k) {
    if (v.shape[k] <= 1 || v.strides[k] == 0) continue;
    int64_t st = v.strides[k];
    if (st < 0) {
      *off += (v.shape[k] - 1) * st;
      st = -st;
    }
    // insertion by decreasing stride (ndim is small)
    int j = n++;
    while (j > 0 && dims[j - 1].s < st) {
      dims[j] = dims[j - 1];
      --j;
    }
    dims[j] = {st, v.shape[k]};
  }
  *nd = n;
  for (int k = 1; k < n; ++k)
    if (dims[k].s == dims[k - 1].s) return false;
  return true;
}
}  // namespace

// The same-base, intersecting-range case of may_overlap (the cheap tests are
// inline in the header). No allocation: every array is bounded by the
// number of dimensions.
bool may_overlap_same_base(const ViewDesc& a, const ViewDesc& b) {
  int64_t oa, ob;
  NormDim da[VBE_MAX_NDIM], db[VBE_MAX_NDIM];
  int na, nb;
  if (!normalise(a, &oa, da, &na) || !normalise(b, &ob, db, &nb)) return true;
  // the union of both stride sets and 1, in decreasing order
  int64_t s[2 * VBE_MAX_NDIM + 1];
  int ns = 0;
  auto add = [&](int64_t v) {
    int j = 0;
    while (j < ns && s[j] > v) ++j;
    if (j < ns && s[j] == v) return;
    for (int q = ns; q > j; --q) s[q] = s[q - 1];
    s[j] = v;
    ++ns;
  };
  for (int k = 0; k < na; ++k) add(da[k].s);
  for (int k = 0; k < nb; ++k) add(db[k].s);
  add(1);
  for (int k = 1; k < ns; ++k)
    if (s[k - 1] % s[k] != 0) return true;
  // digit intervals of each view
  auto box = [&](int64_t off, const NormDim* d, int nd, int64_t* lo, int64_t* hi) {
    int64_t rem = off;
    for (int k = 0; k < ns; ++k) {
      const int64_t c = rem / s[k];
      rem -= c * s[k];
      int64_t ext = 1;
      for (int q = 0; q < nd; ++q)
        if (d[q].s == s[k]) ext = d[q].n;
      lo[k] = c;
      hi[k] = c + ext - 1;
      if (k > 0 && c + ext - 1 >= s[k - 1] / s[k]) return false;  // carries
    }
    return true;
  };
  int64_t alo[2 * VBE_MAX_NDIM + 1], ahi[2 * VBE_MAX_NDIM + 1], blo[2 * VBE_MAX_NDIM + 1], bhi[2 * VBE_MAX_NDIM + 1];
  if (!box(oa, da, na, alo, ahi) || !box(ob, db, nb, blo, bhi)) return true;
  for (int k = 0; k < ns; ++k)
    if (ahi[k] < blo[k] || bhi[k] < alo[k]) return false;
  return true;
}

// ------------------------------------------------------------- validation

static const ViewDesc& lookup_view(Ctx* c, int64_t h, const char* what, int idx) {
  auto it = c->views.find(h);
  if (it == c->views.end()) {
    std::ostringstream os;
    os << "instruction " << idx << ": unknown " << what << " view handle " << h;
    fail(VBE_ERR_INVALID, os.str());
  }
  return it->second;
}

std::vector<RInstr> resolve_batch(Ctx* c, const vbe_instr* prog, int64_t n) {
  if (n < 0 || (n > 0 && !prog)) fail(VBE_ERR_INVALID, "null program");
  std::vector<RInstr> out;
  out.reserve(n);
  std::set<int64_t> freed;
  for (int64_t i = 0; i < n; ++i) {
    const vbe_instr& s = prog[i];
    RInstr r;
    r.op = s.op;
    OpKind kind = op_kind(s.op);
    int ar = op_arity(s.op);
    auto err = [&](int code, const std::string& m) {
      std::ostringstream os;
      os << "instruction " << i << " (" << op_name(s.op) << "): " << m;
      fail(code, os.str());
    };
    r.nin = ar;
    r.const_slot = s.const_slot;
    if (r.const_slot < -1 || r.const_slot >= ar) err(VBE_ERR_INVALID, "bad const_slot");
    if ((kind == K_CAST || kind == K_REDUCE) && r.const_slot >= 0)
      err(VBE_ERR_INVALID, "a constant operand is not allowed here");
    if (s.out == 0) err(VBE_ERR_INVALID, "missing output view");
    r.out = lookup_view(c, s.out, "output", (int)i);
    r.h_out = s.out;
    r.has_out = true;
    auto bit = c->bases.find(r.out.base);
    if (bit == c->bases.end() || freed.count(r.out.base)) err(VBE_ERR_INVALID, "base is not live");
    r.dt_out = bit->second.dtype;
    if (kind == K_CONTROL) {
      if (s.op == VBE_OP_FREE) freed.insert(r.out.base);
      out.push_back(r);
      continue;
    }
    if (r.out.self_overlapping()) err(VBE_ERR_OVERLAP, "output view overlaps itself");
    for (int k = 0; k < ar; ++k) {
      if (k == r.const_slot) continue;
      if (s.in[k] == 0) err(VBE_ERR_INVALID, "missing input view " + std::to_string(k));
      r.in[k] = lookup_view(c, s.in[k], "input", (int)i);
      r.h_in[k] = s.in[k];
      auto ib = c->bases.find(r.in[k].base);
      if (ib == c->bases.end() || freed.count(r.in[k].base)) err(VBE_ERR_INVALID, "input base is not live");
      r.dt_in[k] = ib->second.dtype;
    }
    r.axis = s.axis;
    r.seed = s.seed;
    r.key = s.key;
    r.step = s.step;
    // dtype of a constant operand: that of the other inputs (SELECT: bool
    // for the condition, the output's for the values)
    if (r.const_slot >= 0) {
      int cd = r.dt_out;
      if (kind == K_SELECT) {
        cd = r.const_slot == 0 ? VBE_BOOL : r.dt_out;
      } else if (kind == K_COPY) {
        cd = r.dt_out;
      } else {
        for (int k = 0; k < ar; ++k)
          if (k != r.const_slot) { cd = r.dt_in[k]; break; }
      }
      r.dt_const = cd;
      r.dt_in[r.const_slot] = cd;
      if (is_float(cd)) r.kf = s.konst.f64; else r.ki = s.konst.i64;
      if (cd == VBE_FLOAT32) r.kf = (double)(float)r.kf;
      if (cd == VBE_BOOL) r.ki = r.ki != 0;
    }
    // dtype rules
    int d0 = r.dt_in[0];
    switch (kind) {
      case K_ARITH:
      case K_DIV:
        if (r.dt_in[0] != r.dt_in[1] || r.dt_in[0] != r.dt_out) err(VBE_ERR_DTYPE, "inputs and output must share one dtype");
        if (r.dt_out == VBE_BOOL) err(VBE_ERR_DTYPE, "bool arithmetic is not defined");
        if (kind == K_DIV && !is_float(r.dt_out)) err(VBE_ERR_DTYPE, "DIVIDE needs a float dtype");
        break;
      case K_FUNARY:
        if (d0 != r.dt_out || !is_float(d0)) err(VBE_ERR_DTYPE, "needs matching float dtypes");
        break;
      case K_SUNARY:
        if (d0 != r.dt_out || d0 == VBE_BOOL) err(VBE_ERR_DTYPE, "needs matching numeric dtypes");
        break;
      case K_CMP:
        if (r.dt_in[0] != r.dt_in[1]) err(VBE_ERR_DTYPE, "inputs must share one dtype");
        if (r.dt_out != VBE_BOOL) err(VBE_ERR_DTYPE, "comparisons write bool");
        break;
      case K_SELECT:
        if (r.dt_in[0] != VBE_BOOL) err(VBE_ERR_DTYPE, "SELECT condition must be bool");
        if (r.dt_in[1] != r.dt_out || r.dt_in[2] != r.dt_out) err(VBE_ERR_DTYPE, "SELECT values must have the output dtype");
        break;
      case K_CAST:
        break;
      case K_COPY:
        if (d0 != r.dt_out) err(VBE_ERR_DTYPE, "COPY keeps the dtype");
        break;
      case K_RANDOM:
        if (r.dt_out != VBE_FLOAT64) err(VBE_ERR_DTYPE, "RANDOM writes float64");
        break;
      case K_REDUCE:
        if (s.op == VBE_OP_ARGMIN_REDUCE || s.op == VBE_OP_ARGMAX_REDUCE) {
          if (d0 == VBE_BOOL) err(VBE_ERR_DTYPE, "argmin/argmax needs a numeric input");
          if (r.dt_out != VBE_INT64) err(VBE_ERR_DTYPE, "argmin/argmax writes int64");
        } else if (d0 != r.dt_out || d0 == VBE_BOOL) {
          err(VBE_ERR_DTYPE, "reduction keeps a numeric dtype");
        }
        break;
      case K_USER: {
        const UserOp* u = user_op(s.op);
        for (int k = 0; k < ar; ++k)
          if (r.dt_in[k] != u->dtype) err(VBE_ERR_DTYPE, std::string("inputs of ") + u->name + " must be " + dtype_name(u->dtype));
        if (r.dt_out != u->dtype) err(VBE_ERR_DTYPE, std::string("output of ") + u->name + " must be " + dtype_name(u->dtype));
        break;
      }
      default:
        break;
    }
    // shape rules
    if (kind == K_REDUCE) {
      const ViewDesc& x = r.in[0];
      if (r.axis < 0 || r.axis >= x.ndim) err(VBE_ERR_SHAPE, "reduction axis out of range");
      if (r.out.ndim != x.ndim - 1) err(VBE_ERR_SHAPE, "reduction output rank");
      for (int k = 0, j = 0; k < x.ndim; ++k) {
        if (k == r.axis) continue;
        if (x.shape[k] != r.out.shape[j++]) err(VBE_ERR_SHAPE, "reduction output shape");
      }
      if (s.op != VBE_OP_ADD_REDUCE && x.shape[r.axis] == 0)
        err(VBE_ERR_SHAPE, "min/max reduction over an empty axis");
    } else {
      for (int k = 0; k < ar; ++k) {
        if (k == r.const_slot) continue;
        if (!r.in[k].same_shape(r.out)) err(VBE_ERR_SHAPE, "input shape differs from output shape");
      }
    }
    out.push_back(r);
  }
  return out;
}

// 64-bit words at a time: each word is multiplied in, the state rotated
// and multiplied, then a splitmix64-style finaliser (keys for caches of
// generated sources and batches; not a cryptographic hash)
uint64_t hash64(const void* data, size_t n, uint64_t seed) {
  const unsigned char* p = (const unsigned char*)data;
  uint64_t h = seed ^ ((uint64_t)n * 0x9E3779B97F4A7C15ull);
  size_t i = 0;
  for (; i + 8 <= n; i += 8) {
    uint64_t w;
    memcpy(&w, p + i, 8);
    h ^= w * 0xBF58476D1CE4E5B9ull;
    h = ((h << 31) | (h >> 33)) * 0x94D049BB133111EBull;
  }
  uint64_t t = 0;
  for (size_t k = 0; i + k < n; ++k) t |= (uint64_t)p[i + k] << (8 * k);
  h ^= t * 0xBF58476D1CE4E5B9ull;
  h ^= h >> 30;
  h *= 0xBF58476D1CE4E5B9ull;
  h ^= h >> 27;
  h *= 0x94D049BB133111EBull;
  return h ^ (h >> 31);
}

uint64_t fnv1a(const void* data, size_t n, uint64_t h) {
  const unsigned char* p = (const unsigned char*)data;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

std::string hex64(uint64_t v) {
  char buf[20];
  snprintf(buf, sizeof buf, "%016llx", (unsigned long long)v);
  return buf;
}

}  // namespace vbe
