"""ctypes binding of libvbe (include/vbe.h): argument marshalling only.

Every function here has the name of the C entry point it calls and raises
:class:`VbeError` when that call returns a negative code. Nothing is
computed on the Python side; if the shared library is missing the import
fails loudly (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, Union, byref, c_char_p, c_double, c_int32, c_int64, c_uint32,
                    c_uint64, c_void_p)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvbe.so")

# dtypes
VBE_BOOL, VBE_INT64, VBE_FLOAT32, VBE_FLOAT64 = 0, 1, 2, 3
DTYPE_CODE = {"bool": VBE_BOOL, "int64": VBE_INT64, "float32": VBE_FLOAT32, "float64": VBE_FLOAT64}

# opcodes (same numbering as vbe.h)
OPCODES = {name: i + 1 for i, name in enumerate([
    "ADD", "SUBTRACT", "MULTIPLY", "DIVIDE", "MAXIMUM", "MINIMUM", "SQRT", "EXP", "LOG", "ABSOLUTE",
    "NEGATIVE", "LESS", "LESS_EQUAL", "GREATER", "GREATER_EQUAL", "EQUAL", "NOT_EQUAL", "SELECT", "CAST",
    "COPY", "RANDOM", "ADD_REDUCE", "MIN_REDUCE", "MAX_REDUCE", "SYNC", "DISCARD", "FREE", "ARGMIN_REDUCE",
    "ARGMAX_REDUCE"])}
VBE_OP_USER_BASE = 64

# config flags
VBE_FUSE, VBE_GRAPHS, VBE_AUTOTUNE, VBE_PACK, VBE_HOST_ONLY, VBE_RECORD = 1, 2, 4, 8, 16, 32
VBE_NATIVE_F64, VBE_NO_TILE_FUSION = 64, 128
VBE_MAX_NDIM = 8

ERRORS = {0: "VBE_OK", -1: "VBE_ERR_INVALID", -2: "VBE_ERR_OUT_OF_BOUNDS", -3: "VBE_ERR_DTYPE",
          -4: "VBE_ERR_SHAPE", -5: "VBE_ERR_OOM", -6: "VBE_ERR_ADMISSION", -7: "VBE_ERR_COMPILE",
          -8: "VBE_ERR_TIMEOUT", -9: "VBE_ERR_CUDA", -10: "VBE_ERR_UNINIT", -11: "VBE_ERR_NO_DEVICE",
          -12: "VBE_ERR_OVERLAP", -13: "VBE_ERR_BUSY"}


class _Konst(Union):
    _fields_ = [("f64", c_double), ("i64", c_int64)]


class vbe_instr(Structure):
    _fields_ = [("op", c_int32), ("const_slot", c_int32), ("out", c_int64), ("in_", c_int64 * 3),
                ("axis", c_int32), ("reserved", c_int32), ("konst", _Konst), ("seed", c_uint64),
                ("key", c_uint64), ("step", c_int64)]


class vbe_config(Structure):
    _fields_ = [("device", c_int32), ("flags", c_uint32), ("mem_cap_bytes", c_uint64),
                ("stream", c_void_p), ("cache_dir", c_char_p)]


class vbe_stats(Structure):
    _fields_ = [(n, c_int64) for n in ("kernel_launches", "graph_launches", "graph_captures", "compiles",
                                       "autotunes", "batches", "bytes_allocated", "peak_bytes",
                                       "list_replays", "tma_group_launches", "packed_launches",
                                       "sweep_group_launches")]


class vbe_req_base(Structure):
    _fields_ = [("dtype", c_int32), ("reserved", c_int32), ("nelem", c_int64), ("init", c_void_p),
                ("result", c_void_p)]


class vbe_req_view(Structure):
    _fields_ = [("base", c_int32), ("ndim", c_int32), ("offset", c_int64),
                ("shape", c_int64 * VBE_MAX_NDIM), ("strides", c_int64 * VBE_MAX_NDIM)]


class vbe_request(Structure):
    _fields_ = [("bases", POINTER(vbe_req_base)), ("nbases", c_int32), ("nviews", c_int32),
                ("views", POINTER(vbe_req_view)), ("instrs", POINTER(vbe_instr)), ("ninstrs", c_int64)]


class vbe_server_config(Structure):
    _fields_ = [("slots", c_int32), ("max_queue", c_int32), ("mem_cap_bytes", c_uint64), ("flags", c_uint32),
                ("workers", c_int32)]


class vbe_request_result(Structure):
    _fields_ = [("status", c_int32), ("reserved", c_int32), ("footprint_bytes", c_int64),
                ("t_arrive_ns", c_double), ("t_admit_ns", c_double), ("t_done_ns", c_double),
                ("t_issued_ns", c_double), ("t_ready_ns", c_double)]


assert ctypes.sizeof(vbe_instr) == 80 and ctypes.sizeof(vbe_config) == 32
assert ctypes.sizeof(vbe_req_view) == 144 and ctypes.sizeof(vbe_request) == 40

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libvbe.so is not built ({LIB_PATH}); run paper_1210_7774_b300.build.build()")
lib = ctypes.CDLL(LIB_PATH)

_P = c_void_p
_SIGS = {
    "vbe_init": [POINTER(vbe_config), POINTER(_P)],
    "vbe_finalize": [_P],
    "vbe_base_create": [_P, c_int32, c_int64, POINTER(c_int64)],
    "vbe_base_register": [_P, c_int32, c_int64, c_void_p, POINTER(c_int64)],
    "vbe_base_upload": [_P, c_int64, c_void_p, c_int64],
    "vbe_base_device_ptr": [_P, c_int64, POINTER(c_void_p)],
    "vbe_view_create": [_P, c_int64, c_int64, c_int32, POINTER(c_int64), POINTER(c_int64), POINTER(c_int64)],
    "vbe_view_destroy": [_P, c_int64],
    "vbe_submit": [_P, POINTER(vbe_instr), c_int64, POINTER(c_int64)],
    "vbe_wait": [_P, c_int64, c_int64],
    "vbe_sync": [_P, c_int64, c_void_p, c_int64],
    "vbe_discard": [_P, c_int64],
    "vbe_free": [_P, c_int64],
    "vbe_plan": [_P, POINTER(vbe_instr), c_int64, c_int32, ctypes.c_char_p, c_int64, POINTER(c_int64)],
    "vbe_plan_compile": [_P, POINTER(vbe_instr), c_int64, POINTER(c_int64)],
    "vbe_views_may_overlap": [_P, c_int64, c_int64, POINTER(c_int32)],
    "vbe_get_stats": [_P, POINTER(vbe_stats)],
    "vbe_debug_take_launches": [_P, ctypes.c_char_p, c_int64, POINTER(c_int64)],
    "vbe_strerror": [c_int32],
    "vbe_last_error": [_P],
    "vbe_server_create": [_P, POINTER(vbe_server_config), POINTER(_P)],
    "vbe_server_submit": [_P, POINTER(vbe_request), POINTER(c_int64)],
    "vbe_server_wait": [_P, c_int64, c_int64, POINTER(vbe_request_result)],
    "vbe_server_destroy": [_P],
    "vbe_op_register": [_P, ctypes.c_char_p, ctypes.c_char_p, c_int32, c_int32, POINTER(c_int32)],
    "vbe_reduce_add_f64_noalloc": [c_void_p, c_int64, c_void_p, c_void_p],
    "vbe_measure_fp64_rate": [c_int32, c_int64, POINTER(ctypes.c_double), c_void_p, c_void_p],
    "vbe_mirror_attach": [_P, c_int64, c_void_p, c_int64],
    "vbe_mirror_sync": [_P, c_int64],
    "vbe_mirror_release": [_P, c_int64],
    "vbe_mirror_discard": [_P, c_int64],
    "vbe_mirror_state": [_P, c_int64, POINTER(c_int32)],
    "vbe_debug_set_wait_polls": [_P, c_int64],
}
EXPORTED = tuple(_SIGS)
for _name, _args in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = c_char_p if _name in ("vbe_strerror", "vbe_last_error") else c_int32


class VbeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _check(code: int, ctx=None) -> None:
    if code < 0:
        msg = lib.vbe_last_error(ctx)
        raise VbeError(code, msg.decode(errors="replace") if msg else "")


# ------------------------------------------------------------------ calls

def vbe_init(device: int = 0, flags: int = VBE_FUSE, mem_cap_bytes: int = 0, stream: int | None = None,
             cache_dir: str | None = None):
    cfg = vbe_config(device, flags, mem_cap_bytes, stream or None,
                     cache_dir.encode() if cache_dir else None)
    ctx = c_void_p()
    _check(lib.vbe_init(byref(cfg), byref(ctx)))
    return ctx


def vbe_finalize(ctx) -> None:
    _check(lib.vbe_finalize(ctx))


def vbe_base_create(ctx, dtype: int, nelem: int) -> int:
    h = c_int64()
    _check(lib.vbe_base_create(ctx, dtype, nelem, byref(h)), ctx)
    return h.value


def vbe_base_register(ctx, dtype: int, nelem: int, device_ptr: int) -> int:
    h = c_int64()
    _check(lib.vbe_base_register(ctx, dtype, nelem, device_ptr, byref(h)), ctx)
    return h.value


def vbe_base_upload(ctx, base: int, host_ptr: int, nbytes: int) -> None:
    _check(lib.vbe_base_upload(ctx, base, host_ptr, nbytes), ctx)


def vbe_base_device_ptr(ctx, base: int) -> int:
    p = c_void_p()
    _check(lib.vbe_base_device_ptr(ctx, base, byref(p)), ctx)
    return p.value or 0


def vbe_view_create(ctx, base: int, offset: int, shape, strides) -> int:
    nd = len(shape)
    sh = (c_int64 * max(nd, 1))(*shape)
    st = (c_int64 * max(nd, 1))(*strides)
    h = c_int64()
    _check(lib.vbe_view_create(ctx, base, offset, nd, sh, st, byref(h)), ctx)
    return h.value


def vbe_view_destroy(ctx, view: int) -> None:
    _check(lib.vbe_view_destroy(ctx, view), ctx)


def vbe_submit(ctx, prog, n: int) -> int:
    t = c_int64()
    _check(lib.vbe_submit(ctx, prog, n, byref(t)), ctx)
    return t.value


def vbe_wait(ctx, ticket: int, timeout_ns: int = -1) -> None:
    _check(lib.vbe_wait(ctx, ticket, timeout_ns), ctx)


def vbe_sync(ctx, base: int, host_ptr: int, nbytes: int) -> None:
    _check(lib.vbe_sync(ctx, base, host_ptr, nbytes), ctx)


def vbe_discard(ctx, base: int) -> None:
    _check(lib.vbe_discard(ctx, base), ctx)


def vbe_free(ctx, base: int) -> None:
    _check(lib.vbe_free(ctx, base), ctx)


def vbe_plan(ctx, prog, n: int, want_source: bool = False) -> str:
    need = c_int64()
    _check(lib.vbe_plan(ctx, prog, n, int(want_source), None, 0, byref(need)), ctx)
    buf = ctypes.create_string_buffer(need.value)
    _check(lib.vbe_plan(ctx, prog, n, int(want_source), buf, need.value, byref(need)), ctx)
    return buf.value.decode()


def vbe_plan_compile(ctx, prog, n: int) -> int:
    k = c_int64()
    _check(lib.vbe_plan_compile(ctx, prog, n, byref(k)), ctx)
    return k.value


def vbe_op_register(ctx, name: str, body: str, nin: int, dtype: int) -> int:
    code = c_int32()
    _check(lib.vbe_op_register(ctx, name.encode(), body.encode(), nin, dtype, byref(code)), ctx)
    return code.value


def vbe_views_may_overlap(ctx, a: int, b: int) -> bool:
    o = c_int32()
    _check(lib.vbe_views_may_overlap(ctx, a, b, byref(o)), ctx)
    return bool(o.value)


def vbe_debug_take_launches(ctx) -> str:
    need = c_int64()
    _check(lib.vbe_debug_take_launches(ctx, None, 0, byref(need)), ctx)
    buf = ctypes.create_string_buffer(need.value)
    _check(lib.vbe_debug_take_launches(ctx, buf, need.value, byref(need)), ctx)
    return buf.value.decode()


def vbe_get_stats(ctx) -> dict:
    s = vbe_stats()
    _check(lib.vbe_get_stats(ctx, byref(s)), ctx)
    return {n: getattr(s, n) for n, _ in vbe_stats._fields_}


def vbe_strerror(code: int) -> str:
    return lib.vbe_strerror(code).decode()


def vbe_server_create(ctx, slots: int, mem_cap_bytes: int, flags: int, max_queue: int = 0, workers: int = 1):
    cfg = vbe_server_config(slots, max_queue, mem_cap_bytes, flags, workers)
    s = c_void_p()
    _check(lib.vbe_server_create(ctx, byref(cfg), byref(s)), ctx)
    return s


def vbe_server_submit(srv, req: vbe_request) -> int:
    i = c_int64()
    _check(lib.vbe_server_submit(srv, byref(req), byref(i)))
    return i.value


def vbe_server_wait(srv, req_id: int, timeout_ns: int = -1) -> vbe_request_result:
    r = vbe_request_result()
    _check(lib.vbe_server_wait(srv, req_id, timeout_ns, byref(r)))
    return r


def vbe_server_destroy(srv) -> None:
    _check(lib.vbe_server_destroy(srv))


def vbe_reduce_add_f64_noalloc(x_ptr: int, n: int, out_ptr: int, stream: int | None = None) -> None:
    code = lib.vbe_reduce_add_f64_noalloc(x_ptr, n, out_ptr, stream or None)
    if code < 0:
        raise VbeError(code, "vbe_reduce_add_f64_noalloc")


FP64_RATE_OPS = {"dfma": 0, "dadd": 1, "dmul": 2}


def vbe_measure_fp64_rate(op: str, iters: int, scratch_ptr: int, stream: int | None = None) -> float:
    """float64 operations per second of the FP64 pipe (throughput kernel)."""
    out = ctypes.c_double(0.0)
    code = lib.vbe_measure_fp64_rate(FP64_RATE_OPS[op], iters, byref(out), scratch_ptr, stream or None)
    if code < 0:
        raise VbeError(code, "vbe_measure_fp64_rate")
    return out.value


MIRROR_DEVICE, MIRROR_HOST, MIRROR_HOST_WRITE = 1, 2, 4


def vbe_mirror_attach(ctx, base: int, host_ptr: int, nbytes: int) -> None:
    _check(lib.vbe_mirror_attach(ctx, base, host_ptr, nbytes), ctx)


def vbe_mirror_sync(ctx, base: int) -> None:
    _check(lib.vbe_mirror_sync(ctx, base), ctx)


def vbe_mirror_release(ctx, base: int) -> None:
    _check(lib.vbe_mirror_release(ctx, base), ctx)


def vbe_mirror_discard(ctx, base: int) -> None:
    _check(lib.vbe_mirror_discard(ctx, base), ctx)


def vbe_mirror_state(ctx, base: int) -> int:
    st = c_int32(0)
    _check(lib.vbe_mirror_state(ctx, base, byref(st)), ctx)
    return st.value


def vbe_debug_set_wait_polls(ctx, polls: int) -> None:
    """Test hook: compute threads' staged-data waits allow ``polls`` polls in
    kernels compiled from now on (negative: the normal limit)."""
    _check(lib.vbe_debug_set_wait_polls(ctx, polls), ctx)
