/*
 * vbe.h -- C ABI of libvbe, a single-GPU executor for vector bytecode.
 *
 * The interface follows the paper's component protocol (Kristensen et al.,
 * "cphVB: A System for Automated Runtime Optimization and Parallelization of
 * Vectorized Applications", SciPy 2012):
 *
 *   - section "Interface": the Vector Engine and its manager expose
 *     initialisation, finalisation, execution of a list of bytecodes, and
 *     creation of arrays           -> vbe_init, vbe_finalize, vbe_submit,
 *                                     vbe_base_create / vbe_view_create;
 *   - section "Numerical Python": an array-base is a contiguous allocation,
 *     an array-view selects / re-orders its elements -> vbe_view_create;
 *   - section "Bytecode": one opcode per mnemonic, the opcode fixes the
 *     operand count, operands are multidimensional arrays -> vbe_instr;
 *   - section "Vector Engine Manager": late allocation (metadata first,
 *     memory on first write) and the sync / discard / release ownership
 *     instructions -> vbe_base_create, vbe_sync, vbe_discard, vbe_free and
 *     the SYNC / DISCARD / FREE opcodes;
 *   - section "Vector Engine" (implementation): instructions are grouped
 *     into kernels while they are "blockable" (they share no data with the
 *     kernel, or exactly the same data) -> the fusion analysis behind
 *     vbe_submit (VBE_FUSE), described by vbe_plan.
 *
 * Conventions. Every call returns VBE_OK (0) or a negative VBE_ERR_* code;
 * no C++ exception crosses the boundary. vbe_last_error() gives a message
 * for the most recent failure on a context. Handles (vbe_base, vbe_view,
 * vbe_ticket) are opaque positive 64-bit ids; 0 means "none". Offsets,
 * shapes and strides count ELEMENTS, not bytes. Host pointers passed in are
 * only read during the call unless stated otherwise. The library owns the
 * device memory it allocates; memory registered with vbe_base_register
 * stays owned by the caller. A context is not thread-safe: use one context
 * per client thread, or lock around calls (the server API below does this
 * internally).
 */
#ifndef VBE_H
#define VBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
enum {
  VBE_OK = 0,
  VBE_ERR_INVALID = -1,      /* bad argument, unknown handle or opcode      */
  VBE_ERR_OUT_OF_BOUNDS = -2,/* a view reaches outside its base             */
  VBE_ERR_DTYPE = -3,        /* dtype rule of an opcode violated            */
  VBE_ERR_SHAPE = -4,        /* operand shapes disagree                     */
  VBE_ERR_OOM = -5,          /* device allocation failed                    */
  VBE_ERR_ADMISSION = -6,    /* request larger than the memory cap          */
  VBE_ERR_COMPILE = -7,      /* NVRTC rejected a generated kernel           */
  VBE_ERR_TIMEOUT = -8,      /* a wait ran out of time                      */
  VBE_ERR_CUDA = -9,         /* a CUDA runtime call failed                  */
  VBE_ERR_UNINIT = -10,      /* read of a base that was never written       */
  VBE_ERR_NO_DEVICE = -11,   /* call needs a device; context is host-only   */
  VBE_ERR_OVERLAP = -12,     /* an output view overlaps itself              */
  VBE_ERR_BUSY = -13         /* server queue full / shutting down           */
};

/* --------------------------------------------------------------- dtypes */
enum { VBE_BOOL = 0, VBE_INT64 = 1, VBE_FLOAT32 = 2, VBE_FLOAT64 = 3 };

/* -------------------------------------------------------------- opcodes */
/* Arity in brackets. Elementwise ops require every view operand to have
 * the output's shape (broadcasting is expressed by stride-0 views).
 * Arithmetic inputs share one dtype equal to the output's.               */
enum {
  VBE_OP_ADD = 1,         /* [2] int64/f32/f64; int64 wraps modulo 2^64   */
  VBE_OP_SUBTRACT = 2,    /* [2]                                          */
  VBE_OP_MULTIPLY = 3,    /* [2]                                          */
  VBE_OP_DIVIDE = 4,      /* [2] f32/f64 only, IEEE round-to-nearest (f64:
                             integer-pipe routine, correctly rounded, or
                             the FP64 pipe under VBE_NATIVE_F64)          */
  VBE_OP_MAXIMUM = 5,     /* [2] a if (a > b or a is NaN) else b          */
  VBE_OP_MINIMUM = 6,     /* [2] a if (a < b or a is NaN) else b          */
  VBE_OP_SQRT = 7,        /* [1] f32/f64, correctly rounded (f64: integer-
                             pipe routine, or the FP64 pipe under
                             VBE_NATIVE_F64)                              */
  VBE_OP_EXP = 8,         /* [1] f32: CUDA expf; f64: the library's own
                             table-driven exp on the integer pipes (within
                             1 ulp), or CUDA exp under VBE_NATIVE_F64      */
  VBE_OP_LOG = 9,         /* [1] f32: CUDA logf; f64: the library's own
                             table-driven log (within 1 ulp), or CUDA log
                             under VBE_NATIVE_F64                         */
  VBE_OP_ABSOLUTE = 10,   /* [1] int64/f32/f64                            */
  VBE_OP_NEGATIVE = 11,   /* [1] int64/f32/f64                            */
  VBE_OP_LESS = 12,       /* [2] same-dtype inputs, bool output           */
  VBE_OP_LESS_EQUAL = 13,
  VBE_OP_GREATER = 14,
  VBE_OP_GREATER_EQUAL = 15,
  VBE_OP_EQUAL = 16,
  VBE_OP_NOT_EQUAL = 17,
  VBE_OP_SELECT = 18,     /* [3] out = in0 ? in1 : in2; in0 bool          */
  VBE_OP_CAST = 19,       /* [1] any -> any; float->int64 truncates; ->bool is (x != 0) */
  VBE_OP_COPY = 20,       /* [1] same dtype; with a constant: fill        */
  VBE_OP_RANDOM = 21,     /* [0] f64 out; element m (row-major index over the
                             output view) = splitmix64 finaliser of
                             seed + (key + step*m + 1) * 0x9e3779b97f4a7c15,
                             top 53 bits scaled by 2^-53                  */
  VBE_OP_ADD_REDUCE = 22, /* [1] out = in with dimension `axis` summed    */
  VBE_OP_MIN_REDUCE = 23, /* [1] NaN propagates; empty axis is an error   */
  VBE_OP_MAX_REDUCE = 24,
  VBE_OP_SYNC = 25,       /* [0] out's base must hold its current value in
                             device memory here (a fusion barrier)        */
  VBE_OP_DISCARD = 26,    /* [0] out's base contents are dead until written
                             again; the handle stays valid                */
  VBE_OP_FREE = 27,       /* [0] out's base is released after the batch   */
  VBE_OP_ARGMIN_REDUCE = 28, /* [1] int64 out = index along `axis` of the first
                             minimum (a NaN counts as the minimum: index of
                             the first NaN); empty axis is an error       */
  VBE_OP_ARGMAX_REDUCE = 29, /* [1] likewise for the first maximum          */
  VBE_OP_USER_BASE = 64   /* opcodes from here on are user-defined (vbe_op_register) */
};
#define VBE_MAX_NDIM 8

/* ------------------------------------------------------------- handles */
typedef int64_t vbe_base;
typedef int64_t vbe_view;
typedef int64_t vbe_ticket;
typedef struct vbe_ctx vbe_ctx;

/* ----------------------------------------------------------- instruction */
typedef struct vbe_instr {
  int32_t op;          /* VBE_OP_*                                          */
  int32_t const_slot;  /* -1, or k: input k is the scalar `konst` instead of
                          in[k]; the constant takes the dtype of the other
                          inputs (SELECT: bool for slot 0, else the output's) */
  vbe_view out;        /* output view (SYNC/DISCARD/FREE: any view of the base) */
  vbe_view in[3];      /* input views; unused slots 0                        */
  int32_t axis;        /* reductions: dimension of in[0] to reduce           */
  int32_t reserved;
  union { double f64; int64_t i64; } konst; /* int64/bool constants use i64 */
  uint64_t seed;       /* RANDOM */
  uint64_t key;        /* RANDOM */
  int64_t step;        /* RANDOM */
} vbe_instr;

/* ---------------------------------------------------------------- config */
enum {
  VBE_FUSE = 1u << 0,      /* form kernels from blockable runs (else one launch per bytecode) */
  VBE_GRAPHS = 1u << 1,    /* capture repeated identical batches of three or more launches as
                              CUDA graphs (a batch of one or two launches replays its launch
                              list: with programmatic dependent launch that costs less than a
                              graph launch)                                                  */
  VBE_AUTOTUNE = 1u << 2,  /* time launch shapes per kernel signature and keep the fastest  */
  VBE_PACK = 1u << 3,      /* pack consecutive independent same-signature runs in one launch */
  VBE_HOST_ONLY = 1u << 4, /* no device: analysis, planning and code generation only        */
  VBE_NATIVE_F64 = 1u << 6,/* float64 divide/sqrt/exp/log on the FP64 pipe; by default they run
                              as integer arithmetic (correctly rounded divide and sqrt, exp/log
                              within 1 ulp), because B300's FP64 pipe is 1/64 of its FP32 rate */
  VBE_NO_TILE_FUSION = 1u << 7, /* with VBE_FUSE: keep two-dimensional runs that exchange
                              temporaries at small shifts as separate kernels (by default they
                              become one tile-fused kernel: temporaries in shared memory with
                              recomputed halos; a base the group both reads around and updates
                              gets a second buffer that replaces it after the launch, so
                              vbe_base_device_ptr of a library-owned base is valid only until
                              the next submit) */
  VBE_RECORD = 1u << 5     /* host-only context whose bases live in host memory and whose
                              launches are recorded (vbe_debug_take_launches) instead of run,
                              so tests can execute the generated kernels on a CPU; implies
                              VBE_HOST_ONLY. Not an execution path: nothing runs the kernels. */
};

typedef struct vbe_config {
  int32_t device;          /* CUDA device ordinal                                   */
  uint32_t flags;          /* VBE_* flags above                                     */
  uint64_t mem_cap_bytes;  /* 0 = unlimited; library allocations beyond it fail OOM */
  void* stream;            /* cudaStream_t to launch on, or NULL for a private one   */
  const char* cache_dir;   /* directory for compiled kernels and tuning choices, or NULL */
} vbe_config;

/* Create a context. On VBE_HOST_ONLY no CUDA call is made.
 * Errors: VBE_ERR_INVALID (null args), VBE_ERR_CUDA (device unusable). */
int vbe_init(const vbe_config* cfg, vbe_ctx** out);
/* Wait for all work, release every library allocation, destroy the context. */
int vbe_finalize(vbe_ctx* ctx);

/* Array-base creation: metadata only; device memory is allocated when the
 * base is first written (late allocation, section "Vector Engine Manager").
 * nelem >= 0. Errors: VBE_ERR_INVALID (dtype, nelem). */
int vbe_base_create(vbe_ctx* ctx, int32_t dtype, int64_t nelem, vbe_base* out);
/* Wrap caller-owned device memory (e.g. a framework tensor) as a base.
 * device_ptr must hold nelem elements and stay valid until vbe_free. The
 * library never frees it. */
int vbe_base_register(vbe_ctx* ctx, int32_t dtype, int64_t nelem, void* device_ptr, vbe_base* out);
/* Copy nbytes (== nelem * itemsize) from host into the base, allocating it
 * if needed. Ordered after all earlier submits; returns when the copy has
 * been read from host memory. */
int vbe_base_upload(vbe_ctx* ctx, vbe_base base, const void* host, int64_t nbytes);
/* Device address of the base, or NULL if it has no memory yet. */
int vbe_base_device_ptr(vbe_ctx* ctx, vbe_base base, void** out);

/* Describe a view: element (i_0..i_{ndim-1}) is base[offset + sum i_k*strides[k]].
 * ndim in [0, VBE_MAX_NDIM]; shape[k] >= 0; strides may be 0 or negative.
 * Every reachable element must lie in the base (VBE_ERR_OUT_OF_BOUNDS). */
int vbe_view_create(vbe_ctx* ctx, vbe_base base, int64_t offset, int32_t ndim,
                    const int64_t* shape, const int64_t* strides, vbe_view* out);
int vbe_view_destroy(vbe_ctx* ctx, vbe_view view);

/* Execute a batch of n bytecodes, in order semantics (section "Vector
 * Engine": the engine obeys the serialisation dependencies). Returns after
 * the work is enqueued on the context's stream; *ticket identifies it.
 * The batch is validated first; on any error nothing is enqueued. */
int vbe_submit(vbe_ctx* ctx, const vbe_instr* prog, int64_t n, vbe_ticket* ticket);
/* Wait for a ticket. timeout_ns < 0 waits forever; VBE_ERR_TIMEOUT when the
 * limit passes (the work continues). A ticket may be waited on any number
 * of times. Tickets share a ring of 1024 events: waiting on a ticket more
 * than 1024 submits old also waits for the later submit that reused its
 * event (later work on the same stream), never for less. VBE_ERR_INVALID for
 * a ticket this context never issued. */
int vbe_wait(vbe_ctx* ctx, vbe_ticket ticket, int64_t timeout_ns);
/* Read access (section "Vector Engine Manager", sync): wait for all work
 * enqueued so far, then copy nbytes of the base into host_dst. */
int vbe_sync(vbe_ctx* ctx, vbe_base base, void* host_dst, int64_t nbytes);
/* Mark a base's contents dead (discard); its memory may be reused. */
int vbe_discard(vbe_ctx* ctx, vbe_base base);
/* Release a base (and its views) after the work enqueued so far. */
int vbe_free(vbe_ctx* ctx, vbe_base base);

/* ------------------------------------------------------- host mirrors */
/* The data-ownership scheme of section "Vector Engine Manager" for a base
 * that also has a copy in host memory (the paper's "shared memory" copy):
 * the library keeps track of which copies hold the base's current value and
 * who may write it. Rules, as this library applies them:
 *  1. The host asks for access: vbe_mirror_sync for read access,
 *     vbe_mirror_release for write access (vbe_mirror_discard when it has
 *     already overwritten its copy). It keeps no ownership state itself.
 *  2. A submitted batch may read every input and write every output it
 *     names: before it runs, a mirrored base whose current value only the
 *     mirror holds is copied to the device (unless the batch's first use of
 *     it overwrites every element); afterwards the mirror of a base the batch
 *     wrote is stale, and the host holds write access to no base it named.
 *  3. An in-batch SYNC of a mirrored base copies the device copy back to the
 *     mirror at that point (the mirror is current once the batch completes);
 *     an in-batch DISCARD drops the device copy (the mirror, if current,
 *     then holds the value; otherwise no copy does). Such a batch is executed
 *     afresh at every submit (never replayed from a graph). A batch that
 *     reads a mirrored base after discarding it, while the mirror holds its
 *     value, is rejected (VBE_ERR_INVALID): write it first. A batch that
 *     reads a mirrored base whose value no copy holds is rejected
 *     (VBE_ERR_UNINIT).
 *  4. The library tracks ownership (vbe_mirror_state); it reads and writes
 *     the mirror only in the calls above and in rule 2 and 3 copies.
 * The mirror is caller-owned memory of exactly the base's size; it must stay
 * valid until vbe_free (or vbe_finalize). The host must not write it without
 * write access, nor read it without read access: the library cannot see such
 * accesses. vbe_base_upload into a mirrored base makes the device copy
 * current and the mirror stale. */
enum {
  VBE_MIRROR_DEVICE = 1,     /* the device copy holds the current value      */
  VBE_MIRROR_HOST = 2,       /* the mirror holds the current value            */
  VBE_MIRROR_HOST_WRITE = 4  /* the host holds write access (owns the base)   */
};
/* Attach host memory `host` (nbytes == the base's size) as the base's mirror.
 * It declares that the mirror holds the base's current value and that the
 * host has write access (as after a discard); the device copy, if any, is
 * no longer current. Waits for work already enqueued. Errors:
 * VBE_ERR_INVALID (size, null pointer, a registered base, a second mirror). */
int vbe_mirror_attach(vbe_ctx* ctx, vbe_base base, void* host, int64_t nbytes);
/* Read access (sync): waits for all enqueued work; on return the mirror holds
 * the base's current value (copied from the device if it did not). Errors:
 * VBE_ERR_INVALID (no mirror), VBE_ERR_UNINIT (no copy holds a value: the
 * base was discarded). */
int vbe_mirror_sync(vbe_ctx* ctx, vbe_base base);
/* Write access (release): as vbe_mirror_sync, then the device copy is no
 * longer current and the host owns the base; the next batch that uses it
 * reads the mirror. */
int vbe_mirror_release(vbe_ctx* ctx, vbe_base base);
/* Discard: the host declares that its mirror holds the base's current value
 * (it has overwritten it) and that every other copy is invalid; no copy is
 * made. Waits for enqueued work first, so no copy back is still in flight. */
int vbe_mirror_discard(vbe_ctx* ctx, vbe_base base);
/* *state = VBE_MIRROR_* bits of the base as of the calls made so far. */
int vbe_mirror_state(vbe_ctx* ctx, vbe_base base, int32_t* state);

/* Describe, as JSON, how vbe_submit would execute a batch: the kernels
 * (runs) it forms, the instructions of each, which values stay in registers
 * and which are stored, and the generated CUDA source when
 * want_source != 0. Writes at most cap bytes (NUL-terminated) and the full
 * length to *needed. Works on host-only contexts. */
int vbe_plan(vbe_ctx* ctx, const vbe_instr* prog, int64_t n, int32_t want_source,
             char* buf, int64_t cap, int64_t* needed);

/* Generate and compile (without loading) every kernel the batch would
 * use: a host-side check of the code generator. *nkernels = runs compiled. */
int vbe_plan_compile(vbe_ctx* ctx, const vbe_instr* prog, int64_t n, int64_t* nkernels);
/* Diagnostic: *out = 0 when the two views provably share no element, else
 * 1. This is the overlap test the fusion analysis uses (exact for views
 * whose strides form a divisibility chain, conservative otherwise). */
int vbe_views_may_overlap(vbe_ctx* ctx, vbe_view a, vbe_view b, int32_t* out);

/* VBE_RECORD contexts: move the launches recorded so far into buf as JSON
 * {"allocs": [[addr, bytes], ...], "launches": [...], "sources": {key: text}}
 * (addresses are host addresses of the context's allocations). Same size
 * protocol as vbe_plan. */
int vbe_debug_take_launches(vbe_ctx* ctx, char* buf, int64_t cap, int64_t* needed);

/* Test hook for failure detection (no counterpart in the paper): from now
 * on, kernels this context compiles give their compute threads at most
 * `polls` polls (0: none) when they wait for data staged by bulk or tensor
 * copies, so that those waits run out and the kernel takes its failure
 * path: it sets the context's error word, stops computing, lets its
 * producer and drain waits (which keep their full limit) see every copy it
 * issued land, and exits; the next vbe_wait / vbe_sync returns
 * VBE_ERR_TIMEOUT and the batch's results are invalid. polls < 0 restores
 * the normal limit (2^24 polls). Waits for enqueued work first and drops
 * the context's cached launches. VBE_ERR_INVALID if polls > 2^24. */
int vbe_debug_set_wait_polls(vbe_ctx* ctx, int64_t polls);

typedef struct vbe_stats {
  int64_t kernel_launches;   /* launches of generated kernels                 */
  int64_t graph_launches;    /* CUDA graph replays                            */
  int64_t graph_captures;
  int64_t compiles;          /* NVRTC compilations (cache misses)             */
  int64_t autotunes;         /* signatures tuned                              */
  int64_t batches;
  int64_t bytes_allocated;   /* live library allocations                      */
  int64_t peak_bytes;
  int64_t list_replays;      /* repeated batches replayed from their cached
                                launch list (no analysis, no graph)          */
  int64_t tma_group_launches; /* tile-fused groups issued (or captured) in the
                                tensor-copy form, tuning trials included     */
  int64_t packed_launches;   /* launches (graph replays included) of packed
                                kernels: several independent runs executed by
                                one persistent launch (VBE_PACK)              */
  int64_t sweep_group_launches; /* tile-fused groups issued (or captured) in
                                the row-sweep form (one warp per column strip
                                walking the rows), tuning trials included    */
} vbe_stats;
int vbe_get_stats(vbe_ctx* ctx, vbe_stats* out);

const char* vbe_strerror(int code);
const char* vbe_last_error(vbe_ctx* ctx);

/* Register a user-defined elementwise operation (section "Interface": the
 * engine's API includes registration of a user-defined operation). `body`
 * is the body of a CUDA device function of nin (1..3) arguments named a, b,
 * c, all of `dtype` (VBE_FLOAT32, VBE_FLOAT64 or VBE_INT64), returning that
 * dtype, e.g. "return a * a + b;". It is compiled into every fused kernel
 * that uses the operation, so it fuses with the bytecodes around it; the
 * code generator compiles with IEEE arithmetic (no FMA contraction), so a
 * body of + - * / sqrt is evaluated exactly as written. `name` is an
 * identifier of at most 48 characters. *opcode receives the operation's
 * opcode (>= VBE_OP_USER_BASE) for vbe_instr.op; registering the same
 * (name, body, nin, dtype) again returns the same opcode, in any context.
 * Opcodes are process-wide; at most 1024 operations. Errors:
 * VBE_ERR_INVALID (name, arity, dtype, a name registered with another
 * definition, table full), VBE_ERR_COMPILE (the body does not compile; the
 * message holds the compiler log). Instructions using the opcode follow
 * the arithmetic rules: inputs and output of the registered dtype, one
 * input may be a constant. */
int vbe_op_register(vbe_ctx* ctx, const char* name, const char* body, int32_t nin, int32_t dtype,
                    int32_t* opcode);

/* Sum of n float64 values x[0..n) into *out (both device pointers), on
 * `stream` (a cudaStream_t, or NULL), allocating nothing. The paper has no
 * counterpart: this is for callers that must not let a library allocate
 * device memory (code captured into a CUDA graph by its caller, inference
 * plugin enqueue functions, real-time loops). The reduction's scratch (one
 * partial per 16,384 elements and a completion counter) is a fixed 512 KiB
 * array inside the library, held by every GPU that loads it until exit, so
 * n is limited to 2^30 (VBE_ERR_INVALID beyond, or for null pointers). The
 * first call on a device looks up the array's device address: make it
 * before any stream capture. Calls share the array: calls that overlap on
 * the GPU race; serialise them. Summation order depends only on n.
 * VBE_ERR_CUDA if a CUDA call fails: a CUDA error already pending on the
 * calling thread is reported before anything is enqueued and left pending;
 * a failure of this call's own launch is reported and cleared. No context
 * is needed. */
int vbe_reduce_add_f64_noalloc(const double* x, int64_t n, double* out, void* stream);

/* Measurement aid (no counterpart in the paper): the FP64 pipe's rate on
 * the current device, in float64 operations per second (one fused
 * multiply-add, add or multiply per lane per operation: op = 0, 1 or 2),
 * from a throughput kernel of `iters` rounds of 8 independent chains per
 * thread over 8 blocks of 256 threads per SM, timed with CUDA events on
 * `stream` (a cudaStream_t or NULL); waits for the kernel. `scratch` is
 * device memory for 2048 * SMs doubles, which the kernel overwrites. The
 * float64 workloads' ALU roofline divides by this rate. VBE_ERR_INVALID
 * for bad arguments, VBE_ERR_CUDA if a CUDA call fails. */
int vbe_measure_fp64_rate(int32_t op, int64_t iters, double* out_per_s, double* scratch, void* stream);

/* ------------------------------------------------------------ serving */
/* A request is a self-contained program executed by the server loop:
 * bases (with optional host input and result buffers), views over them
 * (base = index into bases[]), and instructions whose view fields hold
 * 1-based indices into views[] (0 = none). Host buffers must stay valid
 * until the request completes. */
typedef struct vbe_req_base {
  int32_t dtype;
  int32_t reserved;
  int64_t nelem;
  const void* init;   /* host data uploaded on admission, or NULL          */
  void* result;       /* host buffer receiving the final contents, or NULL */
} vbe_req_base;

typedef struct vbe_req_view {
  int32_t base;       /* index into bases[] */
  int32_t ndim;
  int64_t offset;
  int64_t shape[VBE_MAX_NDIM];
  int64_t strides[VBE_MAX_NDIM];
} vbe_req_view;

typedef struct vbe_request {
  const vbe_req_base* bases;
  int32_t nbases;
  int32_t nviews;
  const vbe_req_view* views;
  const vbe_instr* instrs;
  int64_t ninstrs;
} vbe_request;

typedef struct vbe_server_config {
  int32_t slots;          /* requests in flight at once (one stream each) */
  int32_t max_queue;      /* pending requests accepted before VBE_ERR_BUSY */
  uint64_t mem_cap_bytes; /* admission cap on the sum of request footprints */
  uint32_t flags;         /* VBE_FUSE etc. for request execution             */
  int32_t workers;        /* scheduler threads (0 means 1), each with its own
                             context on the same device and a share of the
                             slots; they plan and launch requests in parallel */
} vbe_server_config;

typedef struct vbe_request_result {
  int32_t status;         /* VBE_OK or the request's error code             */
  int32_t reserved;
  int64_t footprint_bytes;
  double t_arrive_ns;     /* submit time (steady clock)                     */
  double t_admit_ns;      /* admitted (slot + memory available)             */
  double t_done_ns;       /* results copied to the host buffers (by the
                             vbe_server_wait call that fetched them)       */
  double t_issued_ns;     /* the request's kernels and result copies were
                             enqueued (t_issued - t_admit: host planning)  */
  double t_ready_ns;      /* results in host memory: the stream's host
                             callback ran (t_ready - t_issued: device work
                             and copies; t_done - t_ready: waking the
                             client's thread and staging copies; 0 when
                             the request failed before that)               */
} vbe_request_result;

typedef struct vbe_server vbe_server;

/* Start a server on a context (which it then owns for execution; do not
 * submit on the context directly while the server runs). Scheduler threads
 * (`workers`; the first uses ctx, the others contexts of their own with
 * ctx's device, flags and cache directory) admit queued requests in
 * arrival order while one of their slots is free and the admitted
 * footprints fit mem_cap_bytes (continuous batching: a request is admitted
 * as soon as another completes), execute each on its slot's stream, and
 * complete it when its results are in pinned staging. Each worker holds the
 * server's lock only to move requests between the queue, its slots and the
 * finished state. */
int vbe_server_create(vbe_ctx* ctx, const vbe_server_config* cfg, vbe_server** out);
/* Enqueue a request; *id identifies it. Its footprint is the bytes of all
 * its bases plus those of every base it writes through some views and reads
 * through others (which may get a second buffer, see VBE_NO_TILE_FUSION).
 * VBE_ERR_ADMISSION if the footprint alone exceeds the cap, VBE_ERR_BUSY if
 * the queue is full. */
int vbe_server_submit(vbe_server* srv, const vbe_request* req, int64_t* id);
/* Wait for a request's results (timeout_ns < 0: forever) and fetch its
 * result record. A result buffer in page-locked host memory (cudaHostAlloc,
 * cudaHostRegister) receives its copy directly from the device; any other
 * is filled from pinned staging by this call, in the calling thread, so a
 * request's results are in its buffers when this call returns VBE_OK. The
 * request's device memory may be released after the call returns. */
int vbe_server_wait(vbe_server* srv, int64_t id, int64_t timeout_ns, vbe_request_result* out);
/* Drain, stop the scheduler, release everything. */
int vbe_server_destroy(vbe_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* VBE_H */
