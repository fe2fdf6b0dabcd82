// Tile fusion of stencil runs.
//
// The paper's array views let one instruction read several shifted windows
// of a base (section "Array Views"; the Jacobi stencil of its example reads
// up/down/left/right views of one grid), and its kernel formation stops at
// every instruction whose views overlap the kernel's outputs without being
// identical (section "Vector Engine"). A stencil program therefore becomes
// a chain of runs of different shapes that hand temporaries to each other
// through memory: in a Lax-Wendroff step, cell fluxes on the whole grid,
// half steps on the x and y faces, and the full step on the interior.
//
// On the GPU that chain is fused by tiles instead. The last run of the
// chain (the anchor) is cut into TH x TW tiles, one per block; every earlier
// run is evaluated over the anchor tile grown by the halo that its
// consumers read (margins found by walking the chain backwards), and its
// values stay in shared memory. Only the anchor writes memory. Points in a
// halo are computed by every block that needs them, with the same
// operations in the same order, so the result is the sequential one.
//
// A group is formed from consecutive runs when:
//   * every run is elementwise over a two-dimensional shape;
//   * a value a run stores is read only by later runs of the group, at a
//     constant shift (dr, dc) of at most kMaxHalo, within the region the
//     producer writes, and is dead after the anchor (DISCARD / FREE before
//     any later read), so it never needs to reach memory;
//   * every base is stored by at most one run of the group.
// If the anchor stores into a base that the group also reads through any
// other view (an in-place update read around by the earlier runs), blocks
// would race: a block could overwrite values its neighbour still has to
// read. Such a base is renamed: the anchor writes a second buffer, the
// elements it does not write are copied across in the same launch, and the
// second buffer becomes the base after the launch.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <map>

#include "vbe_core.h"

namespace vbe {

namespace {

constexpr int kMaxHalo = 8;         // largest shift between a producer and a consumer
constexpr int kMaxMargin = 16;      // largest halo of a run around the tile
constexpr int kMaxGroupRuns = 8;
constexpr int kMaxGroupSteps = 600;
constexpr int64_t kGroupSmemMax = 200 * 1024;  // shared memory of the smallest tile shape (8 x 16)
constexpr int64_t kMaxStride = 1 << 24;          // element strides of the group's views

int64_t last_instr(const Run& r) {
  int64_t m = -1;
  for (int i : r.instrs) m = std::max<int64_t>(m, i);
  return m;
}

// loader point + (dr, dc) = producer point, from the two views' offsets.
// With row stride P and 0 <= dc < P there is one decomposition of the
// offset difference; it is the only one that can satisfy the containment
// test the caller applies (producer columns stay below the row stride).
bool shift_of(const Slot& st, const Slot& ld, int64_t* dr, int64_t* dc) {
  if (st.st.size() != 2 || ld.st.size() != 2) return false;
  if (st.st[1] != 1 || ld.st[1] != 1 || st.st[0] != ld.st[0] || st.dtype != ld.dtype) return false;
  const int64_t P = st.st[0];
  if (P <= 0) return false;
  const int64_t delta = ld.offset - st.offset;
  int64_t r = delta / P;
  if (delta % P < 0) --r;
  const int64_t c = delta - r * P;
  if (std::llabs(r) > kMaxHalo || c > kMaxHalo) return false;
  *dr = r;
  *dc = c;
  return true;
}

bool same_slot(const Slot& a, const Slot& b) { return a.base == b.base && a.offset == b.offset && a.st == b.st; }

std::shared_ptr<Group> try_group(Ctx* c, const std::vector<RInstr>& prog, const LiveIndex& live, const Plan& plan,
                                 const std::vector<size_t>& items) {
  const int m = (int)items.size();
  if (m < 2 || m > kMaxGroupRuns) return nullptr;
  auto g = std::make_shared<Group>();
  int steps = 0;
  for (size_t i : items) {
    const Run& r = plan.items[i].run;
    if (r.shape.size() != 2 || r.shape[0] <= 0 || r.shape[1] <= 0) return nullptr;
    // a reduction over the whole run (both dims) can stay: each of its
    // points must then belong to exactly one tile (checked with the margins)
    if (r.has_red && r.red_axes != std::vector<int>{0, 1}) return nullptr;
    if (r.has_red2) return nullptr;
    // two strides per view, small enough for 32-bit offsets inside a tile
    for (auto* v : {&r.loads, &r.stores})
      for (auto& s : *v)
        if (s.st.size() != 2 || std::llabs(s.st[0]) > kMaxStride || std::llabs(s.st[1]) > kMaxStride) return nullptr;
    steps += (int)r.steps.size();
    g->runs.push_back(r);
  }
  if (steps > kMaxGroupSteps) return nullptr;
  const int anchor = m - 1;
  const int64_t last = last_instr(g->runs[anchor]);
  // producers
  std::map<int64_t, std::pair<int, int>> prod;
  for (int k = 0; k < m; ++k)
    for (int s = 0; s < (int)g->runs[k].stores.size(); ++s) {
      int64_t b = g->runs[k].stores[s].base;
      if (prod.count(b)) return nullptr;
      prod[b] = {k, s};
      if (k < anchor && live.live_after(b, (size_t)last)) return nullptr;
    }
  // loads served by earlier runs of the group
  g->lds.resize(m);
  g->consumed.resize(m);
  for (int k = 0; k < m; ++k) {
    g->lds[k].resize(g->runs[k].loads.size());
    g->consumed[k].assign(g->runs[k].stores.size(), 0);
  }
  for (int l = 0; l < m; ++l) {
    const Run& rl = g->runs[l];
    for (int s = 0; s < (int)rl.loads.size(); ++s) {
      auto it = prod.find(rl.loads[s].base);
      if (it == prod.end() || it->second.first >= l) continue;  // read from memory
      const int k = it->second.first, ss = it->second.second;
      const Run& rk = g->runs[k];
      int64_t dr = 0, dc = 0;
      if (!shift_of(rk.stores[ss], rl.loads[s], &dr, &dc)) return nullptr;
      if (dr < 0 || dc < 0 || rl.shape[0] + dr > rk.shape[0] || rl.shape[1] + dc > rk.shape[1]) return nullptr;
      g->lds[l][s] = GroupLoad{k, ss, (int)dr, (int)dc};
      g->consumed[k][ss] = 1;
    }
  }
  for (int k = 0; k < anchor; ++k) {
    if (g->runs[k].stores.empty()) return nullptr;
    for (char x : g->consumed[k])
      if (!x) return nullptr;
  }
  // margins, from the anchor backwards
  g->box.assign(m, {0, 0, 0, 0});
  for (int k = anchor - 1; k >= 0; --k) {
    int lo_r = INT_MAX, hi_r = INT_MIN, lo_c = INT_MAX, hi_c = INT_MIN;
    for (int l = k + 1; l < m; ++l)
      for (auto& ld : g->lds[l]) {
        if (ld.prod != k) continue;
        lo_r = std::min(lo_r, g->box[l][0] + ld.dr);
        hi_r = std::max(hi_r, g->box[l][1] + ld.dr);
        lo_c = std::min(lo_c, g->box[l][2] + ld.dc);
        hi_c = std::max(hi_c, g->box[l][3] + ld.dc);
      }
    if (lo_r == INT_MAX) return nullptr;
    for (int v : {lo_r, hi_r, lo_c, hi_c})
      if (std::abs(v) > kMaxMargin) return nullptr;
    g->box[k] = {lo_r, hi_r, lo_c, hi_c};
  }
  for (int k = 0; k < m; ++k) {
    const Run& r = g->runs[k];
    if (!r.has_red) continue;
    if (g->box[k] != std::array<int, 4>{0, 0, 0, 0}) return nullptr;
    // nothing in the group may touch the reduction's output
    for (auto& rr : g->runs) {
      for (auto& l : rr.loads)
        if (l.base == r.red_out.base) return nullptr;
      for (auto& st : rr.stores)
        if (st.base == r.red_out.base) return nullptr;
      if (&rr != &r && rr.has_red && rr.red_out.base == r.red_out.base) return nullptr;
    }
  }
  // renaming of bases the anchor updates while the group reads them around
  const Run& ra = g->runs[anchor];
  for (int ss = 0; ss < (int)ra.stores.size(); ++ss) {
    const Slot& st = ra.stores[ss];
    bool need = false;
    for (int l = 0; l < m; ++l)
      for (int s = 0; s < (int)g->runs[l].loads.size(); ++s) {
        const Slot& ld = g->runs[l].loads[s];
        if (ld.base != st.base || g->lds[l][s].prod >= 0) continue;
        if (l == anchor && same_slot(ld, st)) continue;  // each point reads only itself
        need = true;
      }
    if (!need) continue;
    auto bit = c->bases.find(st.base);
    if (bit == c->bases.end() || bit->second.external) return nullptr;
    if (st.st[1] != 1 || st.offset < 0) return nullptr;
    const int64_t P = st.st[0];
    if (P < ra.shape[1] || st.offset % P + ra.shape[1] > P) return nullptr;
    g->renamed.push_back(st.base);
    g->renamed_slot.push_back(ss);
    g->renamed_nelem.push_back(bit->second.nelem);
  }
  for (auto& r : g->runs)
    for (auto& l : r.loads) {
      auto bit = c->bases.find(l.base);
      if (bit != c->bases.end()) g->base_nelem[l.base] = bit->second.nelem;
    }
  // shared memory of the smallest tile shape
  int64_t smem = 0;
  for (int k = 0; k < anchor; ++k) {
    int64_t pts = (int64_t)(8 + g->box[k][1] - g->box[k][0]) * (16 + g->box[k][3] - g->box[k][2]);
    for (auto& s : g->runs[k].stores) smem += (pts * itemsize(s.dtype) + 15) / 16 * 16;
  }
  if (smem > kGroupSmemMax) return nullptr;
  return g;
}

}  // namespace

void form_groups(Ctx* c, const std::vector<RInstr>& prog, const LiveIndex& live, Plan* plan) {
  std::vector<PlanItem>& items = plan->items;
  std::vector<PlanItem> rev;  // output, back to front
  int64_t j = (int64_t)items.size() - 1;
  while (j >= 0) {
    if (items[j].kind != 0) {
      rev.push_back(std::move(items[j]));
      --j;
      continue;
    }
    // grow a window of runs backwards from run j while it stays a valid group
    std::vector<size_t> win{(size_t)j};
    std::shared_ptr<Group> best;
    int64_t p = j - 1;
    for (;;) {
      while (p >= 0 && items[p].kind == 1 && items[p].act.kind != 2) --p;  // DISCARD / FREE in between
      if (p < 0 || items[p].kind != 0) break;
      std::vector<size_t> cand{(size_t)p};
      cand.insert(cand.end(), win.begin(), win.end());
      auto g = try_group(c, prog, live, *plan, cand);
      if (!g) break;
      best = g;
      win = cand;
      --p;
    }
    if (!best) {
      rev.push_back(std::move(items[j]));
      --j;
      continue;
    }
    // host actions between the group's runs run after it
    std::vector<PlanItem> acts;
    for (size_t k = win.front(); k <= (size_t)j; ++k)
      if (items[k].kind == 1) acts.push_back(std::move(items[k]));
    for (auto it = acts.rbegin(); it != acts.rend(); ++it) rev.push_back(std::move(*it));
    PlanItem gi;
    gi.kind = 2;
    gi.group = best;
    rev.push_back(std::move(gi));
    j = (int64_t)win.front() - 1;
  }
  items.assign(std::make_move_iterator(rev.rbegin()), std::make_move_iterator(rev.rend()));
}

}  // namespace vbe
