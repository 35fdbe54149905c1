"""ctypes binding of libkl (include/kl.h): the same entry points, argument
marshalling only.  Every step of the stencil path runs in the library's CUDA
kernels; nothing here computes a tendency, and there is no CPU fallback: if
the shared library is missing or fails to load, every call raises.

PyTorch is used only for device memory and streams (`torch.Tensor.data_ptr()`,
`torch.cuda.current_stream().cuda_stream`).
"""

from __future__ import annotations

import ctypes
import os

from . import build as _build

KL_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "CUDA", -3: "NVRTC", -4: "IO", -5: "WISDOM_PARSE",
          -6: "UNSUPPORTED", -7: "BOUNDS", -8: "TIMEOUT", -9: "OOM"}
DTYPES = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}


class KLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"kl status {status} ({ERRORS.get(status, '?')}): {msg}")
        self.status = status


class Op(ctypes.Structure):
    _fields_ = [("adv", ctypes.c_int32), ("diff", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("accumulate", ctypes.c_int32), ("out_f32", ctypes.c_int32)]


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("g", ctypes.c_int32), ("sj", ctypes.c_int64), ("sk", ctypes.c_int64),
                ("origin", ctypes.c_int64), ("extent", ctypes.c_int64),
                ("zbc", ctypes.c_int32), ("xybc", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("nu", ctypes.c_double), ("zh", ctypes.POINTER(ctypes.c_double))]


class Fields(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("nu", ctypes.c_void_p), ("ut", ctypes.c_void_p), ("vt", ctypes.c_void_p),
                ("wt", ctypes.c_void_p)]


# every symbol include/kl.h declares, with ctypes signatures
_P = ctypes.c_void_p
_I32, _I64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_S = ctypes.c_char_p
SIGNATURES = {
    "kl_create": ([ctypes.POINTER(_P), ctypes.c_int, _S], ctypes.c_int),
    "kl_destroy": ([_P], None),
    "kl_last_error": ([], _S),
    "kl_layout": ([_I32, _I32, _I32, _I32, _I32] + [ctypes.POINTER(_I64)] * 4, ctypes.c_int),
    "kl_fill_ghosts": ([_P, _I32, ctypes.POINTER(Grid), _P, _P, _P, _P, _P], ctypes.c_int),
    "kl_launch": ([_P, ctypes.POINTER(Op), ctypes.POINTER(Grid), ctypes.POINTER(Fields), _P],
                  ctypes.c_int),
    "kl_step": ([_P, ctypes.POINTER(Op), ctypes.POINTER(Grid), ctypes.POINTER(Fields), _P],
                ctypes.c_int),
    "kl_fill_ghosts_op": ([_P, ctypes.POINTER(Op), ctypes.POINTER(Grid),
                           ctypes.POINTER(Fields), _P], ctypes.c_int),
    "kl_launch_with_config": ([_P, ctypes.POINTER(Op), _S, ctypes.POINTER(Grid),
                               ctypes.POINTER(Fields), _P], ctypes.c_int),
    "kl_launch_batched": ([_P, ctypes.POINTER(Op), _I32, ctypes.POINTER(Grid),
                           ctypes.POINTER(Fields), _P], ctypes.c_int),
    "kl_capture": ([_P, ctypes.POINTER(Op), ctypes.POINTER(Grid), ctypes.POINTER(Fields), _S, _P],
                   ctypes.c_int),
    "kl_tune": ([_P, _S, _S, _S], ctypes.c_int),
    "kl_diag": ([_P, _I32, ctypes.POINTER(Grid), _I32, _P, _P, ctypes.POINTER(_D), _P],
                ctypes.c_int),
    "kl_dot": ([_P, _I32, ctypes.POINTER(Grid), _I32, _P, _P, ctypes.POINTER(_D), _P],
               ctypes.c_int),
    "kl_check": ([_P, _P], ctypes.c_int),
    "kl_set_wait_limit": ([_P, _I64], ctypes.c_int),
    "kl_diag_noalloc": ([_I32, ctypes.POINTER(Grid), _P, _P, _P, ctypes.POINTER(_D), _P],
                        ctypes.c_int),
    "kl_stats": ([_P, ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
    "kl_config_normalize": ([ctypes.POINTER(Op), _S, ctypes.c_char_p, ctypes.c_size_t],
                            ctypes.c_int),
    "kl_space_size": ([ctypes.POINTER(Op), _I32, ctypes.POINTER(_I64)], ctypes.c_int),
    "kl_space_config": ([ctypes.POINTER(Op), _I32, _I64, ctypes.c_char_p, ctypes.c_size_t],
                        ctypes.c_int),
    "kl_compile_only": ([ctypes.POINTER(Op), _S, _I32, _I32, ctypes.c_char_p, ctypes.c_size_t],
                        ctypes.c_int),
    "kl_wisdom_select": ([_S, _S, _I32, _I32, _I32, _I32, _I32, _I32, ctypes.c_char_p,
                          ctypes.c_size_t, ctypes.POINTER(_I32)], ctypes.c_int),
    "kl_wisdom_select_points": ([_S, _S, _I32, _I32, _I32, _I64, ctypes.c_char_p, ctypes.c_size_t,
                                 ctypes.POINTER(_I32)], ctypes.c_int),
    "kl_wisdom_append": ([_S, _S, _I32, _I32, _I32, _I32, _I32, _I32, _S, _D, _S], ctypes.c_int),
    "kl_bo_posterior": ([_I32, _I32, _P, _P, _I32, _P, _D, _D, _P, _P, ctypes.POINTER(_D)],
                        ctypes.c_int),
    "kl_bo_suggest": ([_I32, _I32, _P, _P, _I32, _P, _I32, _P, _D, _D, _D,
                       ctypes.POINTER(_I32), _P], ctypes.c_int),
    "kl_set_cache_dir": ([_P, _S], ctypes.c_int),
    "kl_cache_prepare": ([_S, ctypes.POINTER(Op), _S, _I32, _I32, ctypes.POINTER(_I32)],
                         ctypes.c_int),
    "kl_def_create": ([ctypes.POINTER(_P), _S, _S, _S], ctypes.c_int),
    "kl_def_destroy": ([_P], None),
    "kl_def_param": ([_P, _S, _I32, ctypes.POINTER(_I64), _I64], ctypes.c_int),
    "kl_def_restrict": ([_P, _S], ctypes.c_int),
    "kl_def_geometry": ([_P, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_char_p), _S],
                        ctypes.c_int),
    "kl_def_options": ([_P, _S], ctypes.c_int),
    "kl_def_space_size": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)], ctypes.c_int),
    "kl_def_config_at": ([_P, _I64, ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
    "kl_def_normalize": ([_P, _S, ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
    "kl_def_launch_geometry": ([_P, _S, ctypes.POINTER(_I64), ctypes.POINTER(_I64)], ctypes.c_int),
    "kl_def_compile_only": ([_P, _S, ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
    "kl_def_launch": ([_P, _P, ctypes.POINTER(_I64), _I32, _P, _P], ctypes.c_int),
    "kl_def_launch_config": ([_P, _P, _S, ctypes.POINTER(_I64), _I32, _P, _P], ctypes.c_int),
    "kl_def_selected": ([_P, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(_I32)], ctypes.c_int),
    "kl_def_capture": ([_P, _P, ctypes.POINTER(_I64), _I32, _P, _S, _P], ctypes.c_int),
    "kl_def_tune": ([_P, _P, _S, _S, _S], ctypes.c_int),
    "kl_smagorinsky": ([_P, _I32, ctypes.POINTER(Grid), _D, _P, _P, _P, _P, _I32, _P],
                       ctypes.c_int),
    "kl_copy_in": ([_I32, ctypes.POINTER(Grid), _P, _P, _P], ctypes.c_int),
    "kl_copy_out": ([_I32, ctypes.POINTER(Grid), _P, _P, _P], ctypes.c_int),
    "kl_halo_bytes": ([ctypes.POINTER(Grid), _I32, _I32, _I32, ctypes.POINTER(_I64)], ctypes.c_int),
    "kl_halo_pack": ([_P, _I32, ctypes.POINTER(Grid), _I32, _I32, _I32, ctypes.POINTER(_P), _P, _P],
                     ctypes.c_int),
    "kl_halo_unpack": ([_P, _I32, ctypes.POINTER(Grid), _I32, _I32, _I32, ctypes.POINTER(_P), _P,
                        _P], ctypes.c_int),
    "kl_batch_shard": ([_I32, ctypes.POINTER(_I64), _I32, _I32, ctypes.POINTER(_I32),
                        ctypes.POINTER(_I32), ctypes.POINTER(_I64)], ctypes.c_int),
    "kl_version": ([], _S),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libkl.so (building it first if needed); raises if that fails."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libkl.so not found at {path}; run build() first")
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def last_error() -> str:
    return load().kl_last_error().decode()


def check(status: int) -> None:
    if status != KL_OK:
        raise KLError(status, last_error())


def _b(s):
    return None if s is None else (s.encode() if isinstance(s, str) else s)


# ----------------------------------------------------------- entry points

def kl_create(device: int = 0, wisdom_dir: str | None = None) -> int:
    ctx = ctypes.c_void_p()
    check(load().kl_create(ctypes.byref(ctx), device, _b(wisdom_dir)))
    return ctx.value


def kl_destroy(ctx: int) -> None:
    load().kl_destroy(ctx)


def kl_layout(nx, ny, nz, g, dtype):
    out = [ctypes.c_int64() for _ in range(4)]
    check(load().kl_layout(nx, ny, nz, g, dtype, *[ctypes.byref(o) for o in out]))
    return tuple(o.value for o in out)   # sj, sk, origin, extent


def kl_fill_ghosts(ctx, dtype, grid: Grid, u, v, w, nu=None, stream=None) -> None:
    check(load().kl_fill_ghosts(ctx, dtype, ctypes.byref(grid), u, v, w, nu, stream))


def kl_copy_in(dtype, grid: Grid, host, dev, stream=None) -> None:
    """host: address of a contiguous nz x ny x nx host array; dev: the padded device field."""
    check(load().kl_copy_in(dtype, ctypes.byref(grid), host, dev, stream))


def kl_copy_out(dtype, grid: Grid, dev, host, stream=None) -> None:
    check(load().kl_copy_out(dtype, ctypes.byref(grid), dev, host, stream))


def kl_halo_bytes(grid: Grid, dtype, axis, nf) -> int:
    out = ctypes.c_int64()
    check(load().kl_halo_bytes(ctypes.byref(grid), dtype, axis, nf, ctypes.byref(out)))
    return out.value


def kl_halo_pack(ctx, dtype, grid: Grid, axis, side, fields, buf, stream=None) -> None:
    arr = (_P * len(fields))(*fields)
    check(load().kl_halo_pack(ctx, dtype, ctypes.byref(grid), axis, side, len(fields), arr, buf,
                              stream))


def kl_halo_unpack(ctx, dtype, grid: Grid, axis, side, fields, buf, stream=None) -> None:
    arr = (_P * len(fields))(*fields)
    check(load().kl_halo_unpack(ctx, dtype, ctypes.byref(grid), axis, side, len(fields), arr, buf,
                                stream))


def kl_launch(ctx, op: Op, grid: Grid, fields: Fields, stream=None) -> None:
    check(load().kl_launch(ctx, ctypes.byref(op), ctypes.byref(grid), ctypes.byref(fields), stream))


def kl_fill_ghosts_op(ctx, op: Op, grid: Grid, fields: Fields, stream=None) -> None:
    check(load().kl_fill_ghosts_op(ctx, ctypes.byref(op), ctypes.byref(grid), ctypes.byref(fields),
                                   stream))


def kl_step(ctx, op: Op, grid: Grid, fields: Fields, stream=None) -> None:
    check(load().kl_step(ctx, ctypes.byref(op), ctypes.byref(grid), ctypes.byref(fields), stream))


def kl_launch_with_config(ctx, op: Op, config: str, grid: Grid, fields: Fields,
                          stream=None) -> None:
    check(load().kl_launch_with_config(ctx, ctypes.byref(op), _b(config), ctypes.byref(grid),
                                       ctypes.byref(fields), stream))


def kl_launch_batched(ctx, op: Op, grids, fields, stream=None) -> None:
    n = len(grids)
    ga = (Grid * n)(*grids)
    fa = (Fields * n)(*fields)
    check(load().kl_launch_batched(ctx, ctypes.byref(op), n, ga, fa, stream))


def kl_capture(ctx, op: Op, grid: Grid, fields: Fields, path: str, stream=None) -> None:
    check(load().kl_capture(ctx, ctypes.byref(op), ctypes.byref(grid), ctypes.byref(fields),
                            _b(path), stream))


def kl_tune(ctx, capture_path: str, opts: str, wisdom_path: str) -> None:
    check(load().kl_tune(ctx, _b(capture_path), _b(opts), _b(wisdom_path)))


def kl_diag(ctx, dtype, grid: Grid, level, t, ref=None, stream=None):
    out = (ctypes.c_double * 6)()
    check(load().kl_diag(ctx, dtype, ctypes.byref(grid), level, t, ref, out, stream))
    return list(out)


def kl_dot(ctx, dtype, grid: Grid, level, a, b, stream=None) -> float:
    """FP64 sum over the interior of a*b, weighted per level (0: dz, 1: dzh, -1: none)."""
    out = ctypes.c_double()
    check(load().kl_dot(ctx, dtype, ctypes.byref(grid), level, a, b, ctypes.byref(out), stream))
    return out.value


def kl_check(ctx, stream=None) -> None:
    """Raise KLError(KL_ERR_TIMEOUT) if a device wait gave up since the last check."""
    check(load().kl_check(ctx, stream))


def kl_set_wait_limit(ctx, cycles: int) -> None:
    check(load().kl_set_wait_limit(ctx, cycles))


def kl_diag_noalloc(dtype, grid: Grid, t, ref=None, wz=None, stream=None):
    """kl_diag without a context and without any allocation (static scratch)."""
    out = (ctypes.c_double * 6)()
    check(load().kl_diag_noalloc(dtype, ctypes.byref(grid), t, ref, wz, out, stream))
    return list(out)


def kl_stats(ctx) -> str:
    buf = ctypes.create_string_buffer(8192)
    check(load().kl_stats(ctx, buf, len(buf)))
    return buf.value.decode()


def kl_config_normalize(op: Op, config: str) -> str:
    buf = ctypes.create_string_buffer(1024)
    check(load().kl_config_normalize(ctypes.byref(op), _b(config), buf, len(buf)))
    return buf.value.decode()


def kl_space_size(op: Op, family: int) -> int:
    n = ctypes.c_int64()
    check(load().kl_space_size(ctypes.byref(op), family, ctypes.byref(n)))
    return n.value


def kl_space_config(op: Op, family: int, idx: int):
    """(config text, valid?) of the idx-th point of the raw space."""
    buf = ctypes.create_string_buffer(1024)
    st = load().kl_space_config(ctypes.byref(op), family, idx, buf, len(buf))
    if st not in (KL_OK, -1) or not buf.value:
        check(st)
    return buf.value.decode(), st == KL_OK


def kl_compile_only(op: Op, config: str, zbc: int = 0, zuni: int = 1) -> str:
    buf = ctypes.create_string_buffer(65536)
    check(load().kl_compile_only(ctypes.byref(op), _b(config), zbc, zuni, buf, len(buf)))
    return buf.value.decode()


def kl_smagorinsky(ctx, dtype, grid: Grid, cs, u, v, w, nu, fill_ghosts=True, stream=None) -> None:
    check(load().kl_smagorinsky(ctx, dtype, ctypes.byref(grid), cs, u, v, w, nu,
                                1 if fill_ghosts else 0, stream))


def kl_batch_shard(points, world: int, rank: int):
    """(indices of the grids `rank` owns, their total points) under LPT bin packing."""
    n = len(points)
    pts = (ctypes.c_int64 * max(1, n))(*points)
    out = (ctypes.c_int32 * max(1, n))()
    count, load_ = ctypes.c_int32(), ctypes.c_int64()
    check(load().kl_batch_shard(n, pts, world, rank, out, ctypes.byref(count),
                                ctypes.byref(load_)))
    return list(out[:count.value]), load_.value


def kl_set_cache_dir(ctx, path) -> None:
    check(load().kl_set_cache_dir(ctx, _b(path)))


def kl_cache_prepare(path: str, op: Op, config: str, zbc: int = 0, zuni: int = 1) -> bool:
    """Compile config into the cubin cache at path; True if it was already there."""
    hit = ctypes.c_int32()
    check(load().kl_cache_prepare(_b(path), ctypes.byref(op), _b(config), zbc, zuni,
                                  ctypes.byref(hit)))
    return bool(hit.value)


def _f64(a, cols=None):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float64)
    if cols is not None:
        a = a.reshape(-1, cols)
    return a


def kl_bo_posterior(X, y, Xq, length_scale: float = 0.0, noise: float = 0.0):
    """(mean, var, length scale used) of the surrogate at the rows of Xq."""
    import numpy as np
    X = _f64(X)
    n, d = X.shape
    y, Xq = _f64(y), _f64(Xq, d)
    m = Xq.shape[0]
    mean, var, ls = np.zeros(m), np.zeros(m), ctypes.c_double()
    check(load().kl_bo_posterior(n, d, X.ctypes.data, y.ctypes.data, m, Xq.ctypes.data,
                                 length_scale, noise, mean.ctypes.data, var.ctypes.data,
                                 ctypes.byref(ls)))
    return mean, var, ls.value


def kl_bo_suggest(X, y, C, pending=None, xi: float = 0.0, length_scale: float = 0.0,
                  noise: float = 0.0):
    """(index of the candidate row of C with the largest expected improvement, EI of every row)."""
    import numpy as np
    X = _f64(X)
    n, d = X.shape
    y, C = _f64(y), _f64(C, d)
    P = _f64(np.zeros((0, d)) if pending is None else pending, d)
    ei = np.zeros(C.shape[0])
    choice = ctypes.c_int32()
    check(load().kl_bo_suggest(n, d, X.ctypes.data, y.ctypes.data, P.shape[0],
                               P.ctypes.data if P.shape[0] else None, C.shape[0], C.ctypes.data,
                               xi, length_scale, noise, ctypes.byref(choice), ei.ctypes.data))
    return choice.value, ei


def kl_wisdom_select(path, device, cc_major, cc_minor, zbc, nx, ny, nz):
    buf = ctypes.create_string_buffer(1024)
    rule = ctypes.c_int32()
    check(load().kl_wisdom_select(_b(path), _b(device), cc_major, cc_minor, zbc, nx, ny, nz, buf,
                                  len(buf), ctypes.byref(rule)))
    return buf.value.decode(), rule.value


def kl_wisdom_select_points(path, device, cc_major, cc_minor, zbc, points):
    buf = ctypes.create_string_buffer(1024)
    rule = ctypes.c_int32()
    check(load().kl_wisdom_select_points(_b(path), _b(device), cc_major, cc_minor, zbc, points, buf,
                                         len(buf), ctypes.byref(rule)))
    return buf.value.decode(), rule.value


def kl_wisdom_append(path, device, cc_major, cc_minor, zbc, nx, ny, nz, config, time_us,
                     extra: str = "") -> None:
    check(load().kl_wisdom_append(_b(path), _b(device), cc_major, cc_minor, zbc, nx, ny, nz,
                                  _b(config), time_us, _b(extra)))


def kl_version() -> str:
    return load().kl_version().decode()


# ------------------------------------------------------------ user-defined kernels

class Arg(ctypes.Structure):
    """kl_arg: kind 0 scalar (ptr to the host value), 1 in, 2 out, 3 in/out device buffer."""
    _fields_ = [("ptr", ctypes.c_void_p), ("bytes", ctypes.c_int64), ("kind", ctypes.c_int32),
                ("dtype", ctypes.c_int32)]


_SCALARS = {"i32": ctypes.c_int32, "i64": ctypes.c_int64, "u32": ctypes.c_uint32,
            "f32": ctypes.c_float, "f64": ctypes.c_double}
_KINDS = {"in": 1, "out": 2, "inout": 3}


def _buffer_dtype(t) -> int:
    import torch
    return {torch.float64: 0, torch.float32: 1, torch.bfloat16: 2, torch.float16: 3,
            torch.int32: 4}.get(t.dtype, 5)


def make_args(args):
    """kl_arg array from [(kind, value)]: kind "i32"/"i64"/"u32"/"f32"/"f64" with a
    Python number, or "in"/"out"/"inout" with a contiguous device tensor.
    Returns (array, keep-alive list)."""
    keep, out = [], []
    for kind, v in args:
        if kind in _SCALARS:
            c = _SCALARS[kind](v)
            keep.append(c)
            out.append(Arg(ctypes.addressof(c), ctypes.sizeof(c), 0, 0))
        elif kind in _KINDS:
            assert v.is_contiguous()
            out.append(Arg(v.data_ptr(), v.numel() * v.element_size(), _KINDS[kind],
                           _buffer_dtype(v)))
        else:
            raise ValueError(f"unknown argument kind {kind!r}")
    arr = (Arg * max(1, len(out)))(*out)
    return arr, keep


def _problem(p):
    p = list(p) + [1] * (3 - len(p))
    return (ctypes.c_int64 * 3)(*p)


class KernelDef:
    """A user-defined tunable kernel: argument marshalling over the kl_def_* calls."""

    def __init__(self, name: str, source: str, function: str):
        h = ctypes.c_void_p()
        check(load().kl_def_create(ctypes.byref(h), _b(name), _b(source), _b(function)))
        self.h = h.value

    def close(self):
        if getattr(self, "h", None):
            load().kl_def_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:       # interpreter shutdown: the library may be gone
            pass

    def param(self, name, values, default=None):
        vals = (ctypes.c_int64 * len(values))(*values)
        check(load().kl_def_param(self.h, _b(name), len(values), vals,
                                  values[0] if default is None else default))
        return self

    def restrict(self, expr):
        check(load().kl_def_restrict(self.h, _b(expr)))
        return self

    def geometry(self, block=(), grid=(), shared_memory=None):
        arr = lambda xs: (ctypes.c_char_p * 3)(*[_b(x) for x in (list(xs) + [None] * 3)[:3]])
        check(load().kl_def_geometry(self.h, arr(block), arr(grid), _b(shared_memory)))
        return self

    def options(self, opts):
        check(load().kl_def_options(self.h, _b(opts)))
        return self

    def space_size(self):
        raw, valid = ctypes.c_int64(), ctypes.c_int64()
        check(load().kl_def_space_size(self.h, ctypes.byref(raw), ctypes.byref(valid)))
        return raw.value, valid.value

    def config_at(self, idx):
        buf = ctypes.create_string_buffer(4096)
        st = load().kl_def_config_at(self.h, idx, buf, len(buf))
        if st not in (KL_OK, -1) or not buf.value:
            check(st)
        return buf.value.decode(), st == KL_OK

    def normalize(self, config):
        buf = ctypes.create_string_buffer(4096)
        check(load().kl_def_normalize(self.h, _b(config), buf, len(buf)))
        return buf.value.decode()

    def launch_geometry(self, config, problem):
        out = (ctypes.c_int64 * 7)()
        check(load().kl_def_launch_geometry(self.h, _b(config), _problem(problem), out))
        return list(out)

    def compile_only(self, config="default"):
        buf = ctypes.create_string_buffer(65536)
        check(load().kl_def_compile_only(self.h, _b(config), buf, len(buf)))
        return buf.value.decode()

    def launch(self, ctx, problem, args, stream=None):
        arr, keep = make_args(args)
        check(load().kl_def_launch(ctx, self.h, _problem(problem), len(args), arr, stream))

    def launch_config(self, ctx, config, problem, args, stream=None):
        arr, keep = make_args(args)
        check(load().kl_def_launch_config(ctx, self.h, _b(config), _problem(problem), len(args),
                                          arr, stream))

    def selected(self):
        buf = ctypes.create_string_buffer(4096)
        rule = ctypes.c_int32()
        check(load().kl_def_selected(self.h, buf, len(buf), ctypes.byref(rule)))
        return buf.value.decode(), rule.value

    def capture(self, ctx, problem, args, path, stream=None):
        arr, keep = make_args(args)
        check(load().kl_def_capture(ctx, self.h, _problem(problem), len(args), arr, _b(path),
                                    stream))

    def tune(self, ctx, capture_path, opts, wisdom_path):
        check(load().kl_def_tune(ctx, self.h, _b(capture_path), _b(opts), _b(wisdom_path)))
