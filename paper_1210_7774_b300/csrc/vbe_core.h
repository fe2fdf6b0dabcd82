// Internal declarations of libvbe (see include/vbe.h for the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/vbe.h"

namespace vbe {

// ----------------------------------------------------------------- errors
struct Error {
  int code;
  std::string msg;
};
[[noreturn]] void fail(int code, const std::string& msg);
void cuda_check(cudaError_t e, const char* what);

// ----------------------------------------------------------------- dtypes
int itemsize(int dtype);
const char* ctype(int dtype);
const char* dtype_name(int dtype);
bool is_float(int dtype);

// ------------------------------------------------------------------ views
struct ViewDesc {
  int64_t base = 0;
  int64_t offset = 0;
  int ndim = 0;
  int64_t shape[VBE_MAX_NDIM] = {};
  int64_t strides[VBE_MAX_NDIM] = {};
  int64_t lo = 0, hi = -1;  // reachable element range; hi < lo when empty

  int64_t size() const;
  bool same_shape(const ViewDesc& o) const;
  // identical element mapping: same base, offset, shape and strides
  bool identical(const ViewDesc& o) const;
  void finish();  // computes lo/hi
  bool self_overlapping() const;
};

// false only when the two views provably reach no common element (the
// cheap tests inline: analysis calls this for every pair it considers)
bool may_overlap_same_base(const ViewDesc& a, const ViewDesc& b);
inline bool may_overlap(const ViewDesc& a, const ViewDesc& b) {
  if (a.base != b.base) return false;
  if (a.hi < a.lo || b.hi < b.lo) return false;
  if (a.hi < b.lo || b.hi < a.lo) return false;
  return may_overlap_same_base(a, b);
}

// ------------------------------------------------------------ instructions
enum OpKind { K_ARITH, K_DIV, K_FUNARY, K_SUNARY, K_CMP, K_SELECT, K_CAST, K_COPY, K_RANDOM,
              K_REDUCE, K_CONTROL, K_USER };
OpKind op_kind(int op);
int op_arity(int op);
const char* op_name(int op);

// user-defined elementwise operations (process-wide table, vbe_op_register)
struct UserOp {
  std::string name, body;
  int nin = 0, dtype = 0;
};
const UserOp* user_op(int op);  // nullptr when op is not a registered user opcode
int register_user_op(const std::string& name, const std::string& body, int nin, int dtype);

struct RInstr {  // a validated, resolved instruction
  int op = 0;
  int nin = 0;
  int const_slot = -1;
  bool has_out = false;
  ViewDesc out;
  ViewDesc in[3];
  int64_t h_out = 0, h_in[3] = {0, 0, 0};  // view handles
  double kf = 0;
  int64_t ki = 0;
  int axis = 0;
  uint64_t seed = 0, key = 0;
  int64_t step = 0;
  int dt_out = 0;
  int dt_in[3] = {0, 0, 0};
  int dt_const = 0;
};

// -------------------------------------------------------------- run plan
enum class Mode { ELEM = 0, FULL = 1, AXIS_THREAD = 2, AXIS_BLOCK = 3 };

struct Slot {  // a view over the run's iteration space
  int64_t base = 0;
  int64_t offset = 0;
  int dtype = 0;
  std::vector<int64_t> st;  // stride per run dimension (kept dims only for reduction outputs)
};

struct Operand {
  int kind = 0;  // 0: load slot, 1: constant, 2: value
  int idx = 0;
  double f = 0;
  int64_t i = 0;
  int dtype = 0;
};

struct Step {
  int op = 0;
  int dt_out = 0;
  int dt_in = 0;
  int nin = 0;
  Operand a[3];
  int value = 0;  // SSA id of the result
  uint64_t seed = 0, key = 0;
  int64_t rstep = 0;
  int random_idx = -1;  // index among the run's RANDOM steps
  int instr = 0;
};

struct Run {
  std::vector<int64_t> shape;
  std::vector<Slot> loads;
  std::vector<Slot> stores;
  std::vector<int> store_value;
  std::vector<Step> steps;
  std::vector<int> value_dtype;
  bool has_red = false;
  int red_op = 0, red_dtype = 0, red_value = -1;
  std::vector<int> red_axes;  // run dims that are reduced (sorted)
  Slot red_out;               // strides over the kept dims, in order
  // MIN_REDUCE (MAX_REDUCE) followed by ARGMIN_REDUCE (ARGMAX_REDUCE) of the
  // same view over the same axis: one pass writes both (red2_out: int64)
  bool has_red2 = false;
  int red2_op = 0;
  Slot red2_out;
  std::vector<int> instrs;    // batch indices
  int nrandom = 0;
  std::vector<Operand> consts;  // constant operands, passed as parameter words
  bool soft_f64 = false;        // float64 divide/sqrt/exp/log on the integer pipes (sf64.cuh)
  int64_t elements() const;
};

// host-side effects between runs
struct HostAction {
  int kind = 0;  // 0 FREE, 1 DISCARD, 2 SYNC
  int64_t base = 0;
};

// Tile fusion: consecutive two-dimensional runs that communicate through
// temporaries read at small shifts become one kernel. Each block owns a
// TH x TW tile of the last run (the anchor); every earlier run is computed
// over the tile grown by the halo its consumers need, into shared memory.
struct GroupLoad {
  int prod = -1;        // producing run in the group (-1: read from memory)
  int prod_store = -1;  // the producer's store slot
  int dr = 0, dc = 0;   // producer point = loader point + (dr, dc)
};

struct GroupSource;  // generated source of a group (codegen), shared by identical groups

struct Group {
  std::vector<Run> runs;                     // program order; the last is the anchor
  std::vector<std::array<int, 4>> box;       // per run: row lo/hi, col lo/hi margins around the tile
  std::vector<std::vector<GroupLoad>> lds;   // per run, per load slot
  std::vector<std::vector<char>> consumed;   // per run, per store slot: kept in shared memory
  // bases the anchor stores that other views of the group read: the anchor
  // writes them into a second buffer that replaces the base after the
  // launch (elements the anchor does not write are copied across)
  std::vector<int64_t> renamed;
  std::vector<int> renamed_slot;             // the anchor's store slot of each renamed base
  std::vector<int64_t> renamed_nelem;        // element count of each renamed base
  std::map<int64_t, int64_t> base_nelem;     // element count of every base the group reads
  int64_t rows(int k) const { return runs[k].shape[0]; }
  int64_t cols(int k) const { return runs[k].shape[1]; }
  // its source, once looked up (a batch asks for it when it compiles and
  // again when it launches)
  mutable std::shared_ptr<const GroupSource> source;
};

struct PlanItem {
  int kind = 0;  // 0 run, 1 host action, 2 tile-fused group
  Run run;
  HostAction act;
  int pack_with_next = 0;  // >0: this run starts a pack of that many runs
  std::shared_ptr<Group> group;
};

struct Plan {
  std::vector<PlanItem> items;
  std::vector<std::pair<int64_t, int64_t>> staging;  // internal temps: (base handle, src instr)
};

// --------------------------------------------------------------- codegen
struct Spec {  // the launch-independent shape of a generated kernel
  Mode mode = Mode::ELEM;
  int nd = 0;         // ELEM/FULL: iteration dims after coalescing
  int ndk = 0, ndr = 0;
  bool vec = false;   // 1-D contiguous path with vector loads
  int E = 1;          // elements per vector chunk
  std::vector<int> load_cls, store_cls;  // inner-dim stride class: 0 zero, 1 unit, 2 general
  int red_cls = 0;
  bool packed = false;
};

struct Canon {  // a run in the form the generated kernel consumes
  Spec spec;
  std::vector<int64_t> dims;          // ELEM/FULL dims, or kept dims then reduced dims
  std::vector<std::vector<int64_t>> lst, sst;  // per slot strides over dims
  std::vector<int64_t> red_st;        // reduction output strides over kept dims
  std::vector<int64_t> red2_st;       // the paired index output's strides over kept dims
  std::vector<int64_t> idx_st;        // RANDOM linear index strides over dims
  int64_t total = 0;
};

Canon canonicalize(const Run& r, bool allow_vec, const std::vector<uintptr_t>& load_ptrs,
                   const std::vector<uintptr_t>& store_ptrs, uintptr_t red_ptr);
// key_out: the source's cache key (src_key), kept with the memoised source
std::string generate_source(const Run& r, const Canon& c, std::string* entry_prefix, std::string* key_out = nullptr);
// The memoised source of a run's signature, shared (nothing copied; the memo's
// lock is held only to look the entry up).
struct RunSource {
  std::string src, prefix, key;
};
std::shared_ptr<const RunSource> run_source(const Run& r, const Canon& c);
std::string src_key(const std::string& src);  // two 64-bit hashes of the source text
std::vector<std::pair<const char*, const char*>> nvrtc_headers();  // (include name, text)

// words of the kernel parameter block, in the order the generated code reads them
struct LaunchArgs {
  std::vector<int64_t> w;
};
void fill_words(const Run& r, const Canon& c, const std::vector<uintptr_t>& load_ptrs,
                const std::vector<uintptr_t>& store_ptrs, uintptr_t red_ptr, uintptr_t partials,
                uintptr_t counter, int64_t block, int64_t U, LaunchArgs* out, int64_t chunk = 0,
                uintptr_t err = 0, uintptr_t red2_ptr = 0);
int words_count(const Run& r, const Canon& c);

// tensor-copy boxes of a group's staged inputs for one tile shape: per staged
// input the base, its element size, row stride (elements), rows of the base
// and the box (columns, rows)
struct TmaBox {
  int64_t base = 0;
  int isz = 0;
  int64_t pitch = 0, rows = 0;
  int box_cols = 0, box_rows = 0;
  int ref_k = 0, ref_s = 0;  // the view whose pointer word addresses the base
};


// tile-fused groups: source with one kernel per tile shape, and its words
struct TileShape {
  int th = 0, tw = 0, block = 0;
  bool staged = false;  // stencil inputs copied to shared memory first (else read through L1)
  bool tma = false;     // persistent form: inputs prefetched by tensor copies, two stages
  // row-sweep form: one warp per strip of tw anchor columns walks th rows,
  // values kept in registers across rows and exchanged by warp shuffles
  bool sweep = false;
  int64_t smem = 0;     // dynamic shared memory bytes
  std::string suffix() const {
    return std::string(sweep ? "_rs" : (tma ? "_tm" : (staged ? "_ss" : "_sg"))) + std::to_string(th) + "x" +
           std::to_string(tw);
  }
  // the form's letter in VBE_TILE / VBE_RECORD_TILE: "r" sweep, "t" tensor copies, "s" staged
  const char* letter() const { return sweep ? "r" : (tma ? "t" : (staged ? "s" : "")); }
  int form() const { return sweep ? 3 : (tma ? 2 : (int)staged); }
};
struct GroupSource {
  std::string src, prefix, key;  // CUDA source, entry prefix, source key
  std::vector<TileShape> shapes;  // one kernel per shape
};
// A group's source, generated once per distinct group (process-wide memo)
// and kept on the group; nothing is copied.
std::shared_ptr<const GroupSource> group_source(const Group& g);
std::string generate_group_source(const Group& g, std::string* entry_prefix, std::vector<TileShape>* shapes,
                                  std::string* key_out = nullptr);
std::vector<TmaBox> group_tma_boxes(const Group& g, const TileShape& ts);
// tensor maps go first in a tensor-copy kernel's parameters: 16 words each
void fill_group_words(const Group& g, const TileShape& ts, const std::vector<std::vector<uintptr_t>>& load_ptrs,
                      const std::vector<std::vector<uintptr_t>>& store_ptrs,
                      const std::vector<std::pair<uintptr_t, uintptr_t>>& renamed_ptrs,
                      const std::vector<uintptr_t>& red_ptrs, uintptr_t partials, uintptr_t counters, LaunchArgs* out,
                      uintptr_t err_word = 0);

// ----------------------------------------------------------------- context
struct BaseRec {
  int dtype = 0;
  int64_t nelem = 0;
  void* dptr = nullptr;
  void* shadow = nullptr;  // second buffer of a base renamed by tile-fused groups
  bool external = false;
  bool written = false;
  bool internal = false;  // created by the library (staging)
  // host mirror (vbe_mirror_attach): the caller's copy of the base in host
  // memory, kept in step with the device copy by the sync / release /
  // discard rules of the ownership scheme
  void* mirror = nullptr;
  bool dev_valid = true;    // the device copy holds the base's current value
  bool host_valid = false;  // the host mirror holds it
  bool host_write = false;  // the host holds write access (it owns the base)
  std::vector<int64_t> views;  // handles of the views on this base (erased with it)
  int64_t bytes() const { return nelem * itemsize(dtype); }
};

// A loaded module. Modules are context-independent (cudaLibrary), so the
// contexts of a process share one per source: a scheduler thread meeting a
// kernel that another one loaded does not load it again (loading can wait
// for the device work in flight). Unloaded when its last user goes.
struct Kernel {
  cudaLibrary_t lib = nullptr;
  std::mutex mu;  // fn is filled lazily, from any context's thread
  std::map<std::string, cudaKernel_t> fn;
  ~Kernel();
};

// Long runs (many fused bytecodes) also get tile kernels compiled under a
// per-thread register cap, as tuning candidates: more resident warps to hide
// the latency of their long dependency chains, against some spilling
// (float64 Black-Scholes: 32 registers 1.766 ms against 1.795 ms at 40 and
// above on one B300; 24 measured no better than 32).
constexpr int kRegCapMinSteps = 24;
constexpr int kRegCaps[3] = {32, 40, 48};
inline bool reg_cap_variants(const Run& r) { return (int)r.steps.size() >= kRegCapMinSteps; }

struct TuneChoice {
  int block = 256;
  int U = 2;
  int maxreg = 0;      // > 0: the tile kernel compiled with this register cap (U = 1 or 2)
  int bulk_chunk = 0;  // > 0: stage unit-stride inputs through shared memory in chunks of this many elements
  int grid_mult = 0;  // 0: enough CTAs for the work (capped by residency)
};

struct Scratch {  // per stream: reduction partials and counters
  void* partials = nullptr;
  unsigned int* counters = nullptr;
  int64_t n_partials = 0, n_counters = 0;
};

struct Exec {
  cudaStream_t stream = nullptr;
  Scratch scratch;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

struct Launch;  // a recorded kernel launch (runtime.cpp)

// one way a batch ran: the launches are valid for the base addresses in
// the fingerprint (and leave the renamed bases as in `after`)
struct CachedVariant {
  std::vector<std::pair<int64_t, uintptr_t>> fingerprint;  // (base, address), (-base, second buffer)
  int seen = 0;
  bool has_eager = false;
  std::vector<std::shared_ptr<Launch>> eager;  // replayed one by one (no VBE_GRAPHS)
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  std::vector<void*> keep;  // device buffers the graph references
  int64_t launches = 0;
  int64_t packed_launches = 0;  // of which packed (several independent runs in one launch)
  std::vector<std::pair<int64_t, std::pair<void*, void*>>> after;  // renamed base -> (buffer, second buffer)
  uint64_t last_use = 0;
};

struct CachedBatch {
  uint64_t key = 0;
  // the batch's validated instructions, reused while no view or base has
  // been removed from the context since (epoch unchanged)
  std::vector<RInstr> rp;
  uint64_t rp_epoch = ~0ull;
  // a batch whose groups rename bases alternates between two address sets
  std::vector<CachedVariant> v;
};

void release_variant(CachedVariant& v);

struct Ctx {
  vbe_config cfg{};
  std::string cache_dir_s;
  bool host_only = false;
  int device = 0;
  int sm_count = 148;
  Exec exec;
  bool own_stream = false;
  std::mutex mu;  // guards handles and caches when a server thread shares the context
  std::unordered_map<int64_t, BaseRec> bases;
  std::unordered_map<int64_t, ViewDesc> views;
  int64_t next_handle = 1;
  uint64_t epoch = 0;  // advanced whenever a view or base is removed
  std::string last_error;
  // caches
  std::unordered_map<std::string, std::shared_ptr<Kernel>> kernels;  // by source hash
  std::unordered_map<std::string, TuneChoice> tune;                  // by source hash
  std::string tune_file;    // tuning choices kept across processes (in the cache directory), or empty
  std::string tune_device;  // the device model and SM count the choices are keyed by (empty: host only)
  std::unordered_map<uint64_t, CachedBatch> batches;
  // tickets: ticket t is recorded in ring slot t mod kTicketRing; a slot
  // reused by a later submit holds a later point of the same stream, so
  // waiting on it also covers the older ticket
  static constexpr int64_t kTicketRing = 1024;
  std::vector<cudaEvent_t> ticket_ring;
  int64_t next_ticket = 1;
  vbe_stats stats{};
  cudaMemPool_t pool = nullptr;
  // VBE_RECORD: host allocations and recorded launches
  bool record = false;
  int rec_block = 64, rec_U = 1;
  std::map<uintptr_t, size_t> host_allocs;
  std::vector<std::string> rec_launches;
  std::unordered_map<std::string, std::string> rec_sources;
  std::unordered_map<std::string, std::string> rec_alias;  // source key -> key with the test wait limit
  int force_bulk = 0;  // VBE_STAGING: stage every eligible run in chunks of this many elements
  // vbe_debug_set_wait_polls: >= 0 replaces the compute threads' wait limit
  // (VBE_CWAIT) in every kernel this context compiles from then on
  int64_t cwait = -1;
  std::string force_tile;  // VBE_TILE: tile shape of every tile-fused group ("32x32", "s32x32", "t32x32"), never split
  // per mirrored base, in instruction order: whether each in-batch SYNC of
  // the current batch copies the device copy back to the mirror
  std::unordered_map<int64_t, std::deque<bool>> mirror_syncs;
  int64_t n_mirrors = 0;  // bases given a host mirror so far (0: submits skip the mirror rules)
  // set by staged kernels whose bounded waits ran out (mapped host memory)
  unsigned* err_word = nullptr;
  unsigned* err_word_dev = nullptr;
};

// analysis
bool live_after(const std::vector<RInstr>& prog, int64_t base, size_t idx);
// The same question answered from an index built once per batch: per base,
// the positions of the instructions that read it or control it (SYNC,
// DISCARD, FREE), so each answer is a binary search instead of a scan of
// the rest of the batch.
struct LiveIndex {
  // position, and 0 a read, 1 a SYNC, 2 a DISCARD or FREE
  std::unordered_map<int64_t, std::vector<std::pair<int64_t, int>>> ev;
  explicit LiveIndex(const std::vector<RInstr>& prog);
  bool live_after(int64_t base, size_t idx) const;
};
void form_groups(Ctx* c, const std::vector<RInstr>& prog, const LiveIndex& live, Plan* plan);  // tile fusion (groups.cpp)
std::vector<RInstr> resolve_batch(Ctx* c, const vbe_instr* prog, int64_t n);
Plan make_plan(Ctx* c, std::vector<RInstr>& prog, bool fuse, bool pack);
std::string plan_json(Ctx* c, const std::vector<RInstr>& prog, const Plan& p, bool want_source);

// runtime
void exec_batch(Ctx* c, Exec* ex, const vbe_instr* prog, int64_t n, bool allow_graph);
// key: the source's src_key when the caller has it (saves hashing the text again)
std::shared_ptr<Kernel> get_kernel(Ctx* c, const std::string& src, const std::string* key = nullptr);
void precompile(Ctx* c, const std::vector<std::string>& srcs, const std::vector<std::string>* keys = nullptr);
void* dev_alloc(Ctx* c, Exec* ex, int64_t bytes);
void dev_free(Ctx* c, Exec* ex, void* p, int64_t bytes);
void ensure_scratch(Ctx* c, Exec* ex, int64_t partials, int64_t counters);
void release_exec(Ctx* c, Exec* ex);
void init_error_word(Ctx* c);
// views by base: a new view is listed under its base, and freeing a base
// erases its views without looking at any other
void add_view(Ctx* c, int64_t handle, const ViewDesc& v);
void erase_views_of(Ctx* c, BaseRec& br);
// Tuning choices are shared by the contexts of a process and persist in the
// cache directory, one file per device model: load_tune reads it when a
// context is created, recall_tune finds a choice (this context's, another
// context's, or the file's), remember_tune records a new one and appends it
// to the file.
void load_tune(Ctx* c);
bool recall_tune(Ctx* c, const std::string& key, TuneChoice* out);
void remember_tune(Ctx* c, const std::string& key, const TuneChoice& tc);
void release_error_word(Ctx* c);
bool take_error_word(Ctx* c);  // true (and cleared) when a staged kernel reported a failed wait
void check_error_word(Ctx* c);  // fails with VBE_ERR_TIMEOUT when take_error_word is true
// a host <-> device copy in stream order (recorded as a copy on VBE_RECORD contexts)
void stream_copy(Ctx* c, Exec* ex, void* dst, const void* src, int64_t bytes, bool to_host);
uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull);
uint64_t hash64(const void* data, size_t n, uint64_t seed);
std::string hex64(uint64_t v);

}  // namespace vbe

// the opaque handle of the public ABI
struct vbe_ctx {
  vbe::Ctx c;
};
