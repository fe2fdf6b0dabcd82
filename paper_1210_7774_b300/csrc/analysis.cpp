// Dependency and fusion analysis: turns a validated batch into runs
// (kernels) and host actions.
//
// Kernel formation follows the paper's section "Vector Engine"
// (implementation): instructions are scanned in order and added to the
// current kernel while they are blockable with it, i.e. (1) the new
// instruction's inputs and the kernel's outputs, and (2) the new
// instruction's output and the kernel's inputs and outputs, either share no
// data or are precisely the same data. "Precisely the same data" is read
// as an identical element mapping (same base, offset, shape and strides).
// On a GPU every element index of a run is handled by exactly one thread,
// so a value written to a view and read again through the identical view
// never leaves registers.
//
// Extensions for the GPU (each keeps the in-order result):
//  * all elementwise instructions of a run share one iteration shape;
//  * a reduction may join a run as its epilogue; a reduction of that
//    reduction's (dead) output merges into it (e.g. row sums then their
//    sum become one full reduction); nothing in the run may touch the
//    reduction's output;
//  * DISCARD / FREE end the life of a base's values (section "Vector
//    Engine Manager": discard invalidates the copies), so values of a base
//    that is discarded or freed before its next read are never stored;
//  * SYNC ends the run (the host may read the base);
//  * an instruction whose output partially overlaps one of its own inputs
//    first copies that input to an internal temporary, which gives the
//    "inputs are read before the output is written" reading.
#include <algorithm>
#include <cstring>
#include <map>
#include <set>
#include <sstream>

#include "vbe_core.h"

namespace vbe {

int64_t Run::elements() const {
  int64_t n = 1;
  for (auto s : shape) n *= s;
  return n;
}

namespace {

constexpr int kMaxSteps = 400;
constexpr int kMaxSlots = 40;

bool reads_base(const RInstr& r, int64_t base) {
  for (int k = 0; k < r.nin; ++k)
    if (k != r.const_slot && r.in[k].base == base) return true;
  return false;
}

}  // namespace

// true when base's contents written so far may still be read after
// instruction idx (by a later instruction, a SYNC, or after the batch)
bool live_after(const std::vector<RInstr>& prog, int64_t base, size_t idx) {
  for (size_t j = idx + 1; j < prog.size(); ++j) {
    const RInstr& r = prog[j];
    if (op_kind(r.op) == K_CONTROL) {
      if (r.out.base != base) continue;
      if (r.op == VBE_OP_SYNC) return true;
      return false;  // DISCARD or FREE
    }
    if (reads_base(r, base)) return true;
  }
  return true;
}

LiveIndex::LiveIndex(const std::vector<RInstr>& prog) {
  for (size_t j = 0; j < prog.size(); ++j) {
    const RInstr& r = prog[j];
    if (op_kind(r.op) == K_CONTROL) {
      ev[r.out.base].push_back({(int64_t)j, r.op == VBE_OP_SYNC ? 1 : 2});
      continue;
    }
    for (int k = 0; k < r.nin; ++k) {
      if (k == r.const_slot) continue;
      auto& e = ev[r.in[k].base];
      if (e.empty() || e.back().first != (int64_t)j) e.push_back({(int64_t)j, 0});
    }
  }
}

bool LiveIndex::live_after(int64_t base, size_t idx) const {
  auto it = ev.find(base);
  if (it == ev.end()) return true;  // nothing after it: still live after the batch
  const auto& e = it->second;
  auto nx = std::upper_bound(e.begin(), e.end(), std::make_pair((int64_t)idx, 3));
  if (nx == e.end()) return true;
  return nx->second != 2;  // a read or a SYNC: live; a DISCARD or FREE: dead
}

namespace {

struct Builder {
  Ctx* c;
  std::vector<RInstr>& prog;
  const LiveIndex& live;
  bool fuse;
  Plan plan;
  bool open = false;
  Run cur;
  std::vector<ViewDesc> load_views;       // per load slot
  std::vector<int> load_value;            // value id per load slot (unused: loads are operands)
  std::vector<std::pair<ViewDesc, int>> written;  // view -> latest value
  ViewDesc red_view;                      // reduction output view
  ViewDesc red2_view;                     // paired index reduction output view
  ViewDesc red_in;                        // the reduced view (when it is a plain view)
  bool red_in_known = false;
  int red_instr = -1;                     // batch index of the run's reduction
  std::vector<HostAction> pending;
  int last_instr = -1;

  Builder(Ctx* c_, std::vector<RInstr>& p, const LiveIndex& l, bool f) : c(c_), prog(p), live(l), fuse(f) {}

  int new_value(int dt) {
    cur.value_dtype.push_back(dt);
    return (int)cur.value_dtype.size() - 1;
  }

  Slot slot_of(const ViewDesc& v, int dt) {
    Slot s;
    s.base = v.base;
    s.offset = v.offset;
    s.dtype = dt;
    s.st.assign(v.strides, v.strides + v.ndim);
    return s;
  }

  Operand operand(const RInstr& r, int k) {
    Operand o;
    if (k == r.const_slot) {
      o.kind = 1;
      o.f = r.kf;
      o.i = r.ki;
      o.dtype = r.dt_const;
      o.idx = (int)cur.consts.size();
      cur.consts.push_back(o);
      return o;
    }
    const ViewDesc& v = r.in[k];
    for (auto it = written.rbegin(); it != written.rend(); ++it) {
      if (it->first.identical(v)) {
        o.kind = 2;
        o.idx = it->second;
        o.dtype = r.dt_in[k];
        return o;
      }
    }
    for (size_t s = 0; s < load_views.size(); ++s) {
      if (load_views[s].identical(v)) {
        o.kind = 0;
        o.idx = (int)s;
        o.dtype = r.dt_in[k];
        return o;
      }
    }
    load_views.push_back(v);
    cur.loads.push_back(slot_of(v, r.dt_in[k]));
    o.kind = 0;
    o.idx = (int)cur.loads.size() - 1;
    o.dtype = r.dt_in[k];
    return o;
  }

  int slot_count() const { return (int)(cur.loads.size() + written.size()); }

  bool conflicts(const RInstr& r) {
    // (1) inputs vs the run's outputs
    for (int k = 0; k < r.nin; ++k) {
      if (k == r.const_slot) continue;
      for (auto& w : written)
        if (may_overlap(r.in[k], w.first) && !r.in[k].identical(w.first)) return true;
      if (cur.has_red && may_overlap(r.in[k], red_view)) return true;
      if (cur.has_red2 && may_overlap(r.in[k], red2_view)) return true;
    }
    // (2) output vs the run's inputs and outputs
    for (auto& l : load_views)
      if (may_overlap(r.out, l) && !r.out.identical(l)) return true;
    for (auto& w : written)
      if (may_overlap(r.out, w.first) && !r.out.identical(w.first)) return true;
    if (cur.has_red && may_overlap(r.out, red_view)) return true;
    if (cur.has_red2 && may_overlap(r.out, red2_view)) return true;
    return false;
  }

  bool shape_is(const ViewDesc& v) const {
    if ((int)cur.shape.size() != v.ndim) return false;
    for (int k = 0; k < v.ndim; ++k)
      if (cur.shape[k] != v.shape[k]) return false;
    return true;
  }

  void start(const ViewDesc& shape_view) {
    cur = Run();
    cur.soft_f64 = (c->cfg.flags & VBE_NATIVE_F64) == 0;
    cur.shape.assign(shape_view.shape, shape_view.shape + shape_view.ndim);
    load_views.clear();
    written.clear();
    red_in_known = false;
    red_instr = -1;
    open = true;
  }

  void close() {
    if (!open) return;
    // stores: the latest value of every written view that is still live
    std::vector<std::pair<ViewDesc, int>> keep;
    for (size_t i = 0; i < written.size(); ++i) {
      bool superseded = false;
      for (size_t j = i + 1; j < written.size(); ++j)
        if (written[j].first.identical(written[i].first)) superseded = true;
      if (superseded) continue;
      if (!fuse || live.live_after(written[i].first.base, (size_t)last_instr)) keep.push_back(written[i]);
    }
    for (auto& w : keep) {
      cur.stores.push_back(slot_of(w.first, c->bases[w.first.base].dtype));
      cur.store_value.push_back(w.second);
    }
    PlanItem it;
    it.kind = 0;
    it.run = std::move(cur);
    plan.items.push_back(std::move(it));
    for (auto& a : pending) {
      PlanItem h;
      h.kind = 1;
      h.act = a;
      plan.items.push_back(h);
    }
    pending.clear();
    open = false;
    written.clear();
    load_views.clear();
  }

  void add_elementwise(const RInstr& r, int idx) {
    Step s;
    s.op = r.op;
    s.dt_out = r.dt_out;
    // operand dtype: the values' dtype for SELECT, else that of input 0
    s.dt_in = r.nin == 0 ? r.dt_out : (r.op == VBE_OP_SELECT ? r.dt_out : r.dt_in[0]);
    s.nin = r.nin;
    for (int k = 0; k < r.nin; ++k) s.a[k] = operand(r, k);
    s.value = new_value(r.dt_out);
    s.seed = r.seed;
    s.key = r.key;
    s.rstep = r.step;
    s.instr = idx;
    if (r.op == VBE_OP_RANDOM) s.random_idx = cur.nrandom++;
    cur.steps.push_back(s);
    cur.instrs.push_back(idx);
    // a new write to a view replaces the value any identical view held
    for (auto it = written.begin(); it != written.end();) {
      if (it->first.identical(r.out)) it = written.erase(it);
      else ++it;
    }
    written.push_back({r.out, s.value});
    last_instr = idx;
  }

  void add_reduction(const RInstr& r, int idx) {
    if (cur.has_red) {
      // merge with the run's reduction: its output is this one's input
      std::vector<int> kept;
      for (int d = 0; d < (int)cur.shape.size(); ++d)
        if (!std::binary_search(cur.red_axes.begin(), cur.red_axes.end(), d)) kept.push_back(d);
      cur.red_axes.push_back(kept[r.axis]);
      std::sort(cur.red_axes.begin(), cur.red_axes.end());
    } else {
      cur.has_red = true;
      cur.red_op = r.op;
      cur.red_dtype = r.dt_out;
      cur.red_axes = {r.axis};
      Operand x = operand(r, 0);
      // a reduction input that is a plain load or constant still needs a value id
      if (x.kind != 2) {
        Step s;
        s.op = VBE_OP_COPY;
        s.dt_out = s.dt_in = r.dt_in[0];
        s.nin = 1;
        s.a[0] = x;
        s.value = new_value(r.dt_in[0]);
        s.instr = idx;
        cur.steps.push_back(s);
        x.kind = 2;
        x.idx = s.value;
      }
      cur.red_value = x.idx;
      red_in = r.in[0];
      red_in_known = true;
    }
    red_view = r.out;
    red_instr = idx;
    cur.red_out = slot_of(r.out, r.dt_out);
    cur.instrs.push_back(idx);
    last_instr = idx;
  }

  bool can_merge_reduction(const RInstr& r, size_t idx) {
    if (!cur.has_red || r.op != cur.red_op || cur.has_red2) return false;
    if (r.op == VBE_OP_ARGMIN_REDUCE || r.op == VBE_OP_ARGMAX_REDUCE) return false;  // indices do not compose
    if (!r.in[0].identical(red_view)) return false;
    if (live.live_after(red_view.base, idx)) return false;
    // the merged output must not touch anything else in the run
    for (auto& l : load_views)
      if (may_overlap(r.out, l)) return false;
    for (auto& w : written)
      if (may_overlap(r.out, w.first)) return false;
    return true;
  }

  // ARGMIN_REDUCE (ARGMAX_REDUCE) right after the run's MIN_REDUCE
  // (MAX_REDUCE) of the identical view over the same single axis: the index
  // reduction is the same pass (the minimum's value and its first index)
  bool can_pair_arg(const RInstr& r) {
    if (!cur.has_red || cur.has_red2 || !red_in_known || cur.red_axes.size() != 1) return false;
    const bool mn = cur.red_op == VBE_OP_MIN_REDUCE && r.op == VBE_OP_ARGMIN_REDUCE;
    const bool mx = cur.red_op == VBE_OP_MAX_REDUCE && r.op == VBE_OP_ARGMAX_REDUCE;
    if (!(mn || mx) || !r.in[0].identical(red_in) || r.axis != cur.red_axes[0]) return false;
    // the view still holds the reduced values: nothing in the run wrote it
    // after the reduction (the reduction is the run's last instruction)
    if (last_instr != red_instr) return false;
    for (auto& l : load_views)
      if (may_overlap(r.out, l)) return false;
    for (auto& w : written)
      if (may_overlap(r.out, w.first)) return false;
    if (may_overlap(r.out, red_view)) return false;
    // a reduction that wrote into its own input has changed the values the
    // index must be taken from: in program order the ARGMIN reads them after
    // the MIN's store, so the pair would answer from stale values (staging
    // of a partially overlapping input already gives such a reduction a
    // private copy to read; this check does not rely on that)
    if (may_overlap(red_view, red_in)) return false;
    return true;
  }

  void add_arg_pair(const RInstr& r, int idx) {
    cur.has_red2 = true;
    cur.red2_op = r.op;
    cur.red2_out = slot_of(r.out, r.dt_out);
    red2_view = r.out;
    cur.instrs.push_back(idx);
    last_instr = idx;
  }

  void run_all() {
    for (size_t i = 0; i < prog.size(); ++i) {
      const RInstr& r = prog[i];
      OpKind kind = op_kind(r.op);
      if (kind == K_CONTROL) {
        HostAction a;
        a.base = r.out.base;
        a.kind = r.op == VBE_OP_FREE ? 0 : (r.op == VBE_OP_DISCARD ? 1 : 2);
        if (r.op == VBE_OP_SYNC) {
          close();
          PlanItem h;
          h.kind = 1;
          h.act = a;
          plan.items.push_back(h);
          continue;
        }
        if (open) {
          // values of this base written by the run are dead
          for (auto it = written.begin(); it != written.end();) {
            if (it->first.base == a.base) it = written.erase(it);
            else ++it;
          }
          if (cur.has_red && red_view.base == a.base) {
            // a discarded reduction output still has to be written: keep it
          }
          pending.push_back(a);
        } else {
          PlanItem h;
          h.kind = 1;
          h.act = a;
          plan.items.push_back(h);
        }
        continue;
      }
      if (kind == K_REDUCE) {
        const ViewDesc& x = r.in[0];
        bool joined = false;
        if (open && fuse && cur.has_red) {
          if (can_merge_reduction(r, i)) {
            add_reduction(r, (int)i);
            joined = true;
          } else if (can_pair_arg(r)) {
            add_arg_pair(r, (int)i);
            joined = true;
          }
        } else if (open && fuse && shape_is(x)) {
          if (!conflicts(r) && slot_count() < kMaxSlots && (int)cur.steps.size() < kMaxSteps) {
            add_reduction(r, (int)i);
            joined = true;
          }
        }
        if (!joined) {
          close();
          start(x);
          add_reduction(r, (int)i);
        }
        if (!fuse) close();
        continue;
      }
      bool joined = false;
      if (open && fuse && shape_is(r.out) && !conflicts(r) && slot_count() < kMaxSlots &&
          (int)cur.steps.size() < kMaxSteps) {
        add_elementwise(r, (int)i);
        joined = true;
      }
      if (!joined) {
        close();
        start(r.out);
        add_elementwise(r, (int)i);
      }
      if (!fuse) close();
    }
    close();
  }
};

}  // namespace

// Inputs that partially overlap their instruction's output are first
// copied to an internal contiguous temporary (freed right after).
static std::vector<RInstr> stage_partial_overlaps(Ctx* c, const std::vector<RInstr>& in, Plan* plan) {
  std::vector<RInstr> out;
  out.reserve(in.size());
  for (size_t i = 0; i < in.size(); ++i) {
    RInstr r = in[i];
    std::vector<RInstr> frees;
    if (op_kind(r.op) != K_CONTROL) {
      for (int k = 0; k < r.nin; ++k) {
        if (k == r.const_slot) continue;
        if (!may_overlap(r.out, r.in[k]) || r.out.identical(r.in[k])) continue;
        BaseRec b;
        b.dtype = r.dt_in[k];
        b.nelem = std::max<int64_t>(1, r.in[k].size());
        b.internal = true;
        int64_t h = c->next_handle++;
        c->bases[h] = b;
        ViewDesc v;
        v.base = h;
        v.offset = 0;
        v.ndim = r.in[k].ndim;
        int64_t acc = 1;
        for (int d = v.ndim - 1; d >= 0; --d) {
          v.shape[d] = r.in[k].shape[d];
          v.strides[d] = acc;
          acc *= std::max<int64_t>(1, v.shape[d]);
        }
        v.finish();
        RInstr cp;
        cp.op = VBE_OP_COPY;
        cp.nin = 1;
        cp.has_out = true;
        cp.out = v;
        cp.in[0] = r.in[k];
        cp.dt_out = cp.dt_in[0] = r.dt_in[k];
        out.push_back(cp);
        r.in[k] = v;
        r.h_in[k] = 0;
        RInstr fr;
        fr.op = VBE_OP_FREE;
        fr.has_out = true;
        fr.out = v;
        fr.dt_out = b.dtype;
        frees.push_back(fr);
        plan->staging.push_back({h, (int64_t)i});
      }
    }
    out.push_back(r);
    for (auto& f : frees) out.push_back(f);
  }
  return out;
}

Plan make_plan(Ctx* c, std::vector<RInstr>& prog, bool fuse, bool pack) {
  (void)pack;
  Plan pre;
  std::vector<RInstr> staged = stage_partial_overlaps(c, prog, &pre);
  prog.swap(staged);
  const LiveIndex live(prog);
  Builder b(c, prog, live, fuse);
  b.plan.staging = pre.staging;
  b.run_all();
  if (fuse && !(c->cfg.flags & VBE_NO_TILE_FUSION)) form_groups(c, prog, live, &b.plan);
  return std::move(b.plan);
}

// ------------------------------------------------------------------- JSON

static void json_str(std::ostringstream& os, const std::string& s) {
  os << '"';
  for (char ch : s) {
    switch (ch) {
      case '"': os << "\\\""; break;
      case '\\': os << "\\\\"; break;
      case '\n': os << "\\n"; break;
      case '\t': os << "\\t"; break;
      default:
        if ((unsigned char)ch < 0x20) {
          char buf[8];
          snprintf(buf, sizeof buf, "\\u%04x", ch);
          os << buf;
        } else {
          os << ch;
        }
    }
  }
  os << '"';
}

std::string plan_json(Ctx* c, const std::vector<RInstr>& prog, const Plan& p, bool want_source) {
  std::ostringstream os;
  os << "{\"items\":[";
  bool first = true;
  for (auto& it : p.items) {
    if (!first) os << ",";
    first = false;
    if (it.kind == 1) {
      static const char* names[] = {"FREE", "DISCARD", "SYNC"};
      os << "{\"action\":\"" << names[it.act.kind] << "\",\"base\":" << it.act.base << "}";
      continue;
    }
    if (it.kind == 2) {
      const Group& g = *it.group;
      os << "{\"group\":{\"runs\":[";
      for (size_t k = 0; k < g.runs.size(); ++k) {
        const Run& r = g.runs[k];
        os << (k ? "," : "") << "{\"shape\":[" << r.shape[0] << "," << r.shape[1] << "],\"instrs\":[";
        for (size_t q = 0; q < r.instrs.size(); ++q) os << (q ? "," : "") << r.instrs[q];
        os << "],\"box\":[" << g.box[k][0] << "," << g.box[k][1] << "," << g.box[k][2] << "," << g.box[k][3]
           << "],\"loads\":[";
        for (size_t q = 0; q < r.loads.size(); ++q) {
          const GroupLoad& ld = g.lds[k][q];
          os << (q ? "," : "") << "{\"base\":" << r.loads[q].base << ",\"from\":" << ld.prod;
          if (ld.prod >= 0) os << ",\"shift\":[" << ld.dr << "," << ld.dc << "]";
          os << "}";
        }
        os << "],\"stores\":[";
        for (size_t q = 0; q < r.stores.size(); ++q)
          os << (q ? "," : "") << "{\"base\":" << r.stores[q].base << ",\"shared\":"
             << (g.consumed[k][q] ? "true" : "false") << "}";
        os << "]}";
      }
      os << "],\"renamed\":[";
      for (size_t q = 0; q < g.renamed.size(); ++q) os << (q ? "," : "") << g.renamed[q];
      os << "]";
      if (want_source) {
        os << ",\"source\":";
        json_str(os, generate_group_source(g, nullptr, nullptr));
      }
      os << "}}";
      continue;
    }
    const Run& r = it.run;
    os << "{\"run\":{\"shape\":[";
    for (size_t k = 0; k < r.shape.size(); ++k) os << (k ? "," : "") << r.shape[k];
    os << "],\"instrs\":[";
    for (size_t k = 0; k < r.instrs.size(); ++k) os << (k ? "," : "") << r.instrs[k];
    os << "],\"ops\":[";
    for (size_t k = 0; k < r.steps.size(); ++k) os << (k ? "," : "") << "\"" << op_name(r.steps[k].op) << "\"";
    os << "],\"loads\":[";
    for (size_t k = 0; k < r.loads.size(); ++k) os << (k ? "," : "") << r.loads[k].base;
    os << "],\"stores\":[";
    for (size_t k = 0; k < r.stores.size(); ++k) os << (k ? "," : "") << r.stores[k].base;
    os << "]";
    if (r.has_red) {
      os << ",\"reduce\":{\"op\":\"" << op_name(r.red_op) << "\",\"axes\":[";
      for (size_t k = 0; k < r.red_axes.size(); ++k) os << (k ? "," : "") << r.red_axes[k];
      os << "],\"out\":" << r.red_out.base << "}";
    }
    if (r.has_red2) os << ",\"reduce2\":{\"op\":\"" << op_name(r.red2_op) << "\",\"out\":" << r.red2_out.base << "}";
    std::vector<uintptr_t> lp(r.loads.size(), 0), sp(r.stores.size(), 0);
    Canon cn = canonicalize(r, true, lp, sp, 0);
    static const char* modes[] = {"elementwise", "full_reduce", "axis_thread", "axis_block"};
    os << ",\"mode\":\"" << modes[(int)cn.spec.mode] << "\",\"dims\":[";
    for (size_t k = 0; k < cn.dims.size(); ++k) os << (k ? "," : "") << cn.dims[k];
    os << "],\"vector\":" << (cn.spec.vec ? "true" : "false");
    if (want_source) {
      os << ",\"source\":";
      json_str(os, generate_source(r, cn, nullptr));
    }
    os << "}}";
  }
  os << "],\"staged\":" << p.staging.size() << "}";
  (void)prog;
  (void)c;
  return os.str();
}

}  // namespace vbe
