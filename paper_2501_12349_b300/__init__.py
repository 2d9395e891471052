"""B300-native local findpts (arXiv 2501.12349): Python binding of libfindpts.

Thin ctypes marshalling over the C ABI declared in include/findpts.h: every
function below has the C function's name, passes device pointers of torch
CUDA tensors and the current CUDA stream, and raises FindptsError on a
non-zero status.  All arithmetic runs in the library's CUDA kernels; there is
no CPU fallback — importing works without a GPU, but calls need the built
libfindpts.so and a CUDA device.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libfindpts.so"

FP_OK, FP_EINVAL, FP_ENOMEM, FP_ELAUNCH, FP_EDEVICE, FP_ETIMEDOUT, FP_EBUSY, FP_EUNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6, -7)
FP_INTERIOR, FP_BORDER, FP_NOT_FOUND = 0, 1, 2
FP_F64, FP_MIXED = 0, 1
FP_ORDER_GIVEN, FP_ORDER_CELL = 0, 1
FP_MAX_N = 8
FP_NSTATS = 16
FP_TIME_ORDER, FP_TIME_FIND, FP_TIME_FOLLOW, FP_TIME_EVAL, FP_NTIMES = 0, 1, 2, 3, 4
FP_SCHED_SRPT, FP_SCHED_SLACK = 0, 1


class FindptsError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} failed: {status} ({fp_status_string(status)})")
        self.status = status


class FpOpts(ctypes.Structure):
    _fields_ = [("bbox_tol", ctypes.c_double), ("M", ctypes.c_int), ("n_grid", ctypes.c_int),
                ("newton_tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("dist_tol", ctypes.c_double), ("precision", ctypes.c_int), ("point_order", ctypes.c_int)]


class FpMeshInfo(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("dr", ctypes.c_int), ("N", ctypes.c_int), ("M", ctypes.c_int),
                ("n_grid", ctypes.c_int), ("NE", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("n_cell_entries", ctypes.c_int64), ("grid_lo", ctypes.c_double * 3),
                ("grid_hi", ctypes.c_double * 3), ("device_bytes", ctypes.c_size_t),
                ("setup_boxes_ms", ctypes.c_double), ("setup_grid_ms", ctypes.c_double)]


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int


def lib() -> ctypes.CDLL:
    """The loaded libfindpts.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2501_12349_b300._build`")
        L = ctypes.CDLL(str(LIB_PATH))
        sig = {
            "fp_opts_default": ([ctypes.POINTER(FpOpts)], None),
            "fp_setup": ([_vp, _int, _int, _int, _i64, ctypes.POINTER(FpOpts), _vp, ctypes.POINTER(_vp)], _int),
            "fp_free": ([_vp], _int),
            "fp_set_precision": ([_vp, _int], _int),
            "fp_set_point_order": ([_vp, _int], _int),
            "fp_findpts": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp], _int),
            "fp_findpts_stats": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp], _int),
            "fp_eval": ([_vp, _vp, _vp, _vp, _i64, _vp, _int, _vp, _vp], _int),
            "fp_eval_order": ([_vp, _vp, _vp, _vp, _i64, _vp, _int, _int, _vp, _vp], _int),
            "fp_findpts_host": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _int, _vp, _i64, _vp], _int),
            "fp_get_info": ([_vp, ctypes.POINTER(FpMeshInfo)], _int),
            "fp_get_boxes": ([_vp, _vp, _vp, _vp, _vp], _int),
            "fp_get_grid": ([_vp, _vp, _vp, _vp], _int),
            "fp_get_curvature": ([_vp, _vp, _vp], _int),
            "fp_device_status": ([_vp, ctypes.POINTER(_int), _vp], _int),
            "fp_status_string": ([_int], ctypes.c_char_p),
            "fp_alu_peak": ([_int, _int, ctypes.POINTER(ctypes.c_double), _vp], _int),
            "fp_set_timing": ([_vp, _int], _int),
            "fp_kernel_times": ([_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64)], _int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def fp_status_string(status: int) -> str:
    return lib().fp_status_string(int(status)).decode()


def _check(fn: str, status: int) -> None:
    if status != FP_OK:
        raise FindptsError(fn, status)


def _stream(stream):
    import torch
    if stream is None:
        return _vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _vp(stream)
    return _vp(stream.cuda_stream)


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return _vp(t.data_ptr())


def fp_opts_default() -> FpOpts:
    o = FpOpts()
    lib().fp_opts_default(ctypes.byref(o))
    return o


def fp_setup(coords, d: int, dr: int, order: int, opts: FpOpts | None = None, stream=None) -> _vp:
    """Setup (Sec. 3.1) from device coordinates [d][NE][N^dr] (float64)."""
    import torch
    NE = coords.numel() // (d * (order + 1) ** dr)
    h = _vp()
    rc = lib().fp_setup(_ptr(coords, torch.float64, "coords"), d, dr, order, NE,
                        ctypes.byref(opts) if opts is not None else None, _stream(stream), ctypes.byref(h))
    _check("fp_setup", rc)
    return h


def fp_free(mesh) -> None:
    _check("fp_free", lib().fp_free(mesh))


def fp_set_precision(mesh, precision: int) -> None:
    _check("fp_set_precision", lib().fp_set_precision(mesh, int(precision)))


def fp_set_point_order(mesh, order: int) -> None:
    _check("fp_set_point_order", lib().fp_set_point_order(mesh, int(order)))


def _find_shapes(mesh, pts, code, elem, r, dist2) -> int:
    """Checks the shapes of a find call's tensors against the mesh's d and
    dr (the C ABI sees only pointers and n, so a short output would be
    written past its end): pts [n][d]; code, elem, dist2 at least n entries;
    r [n][dr].  Returns n."""
    info = fp_get_info(mesh)
    if pts.dim() != 2 or pts.shape[1] != info.d:
        raise ValueError(f"pts must have shape (n, {info.d}), got {tuple(pts.shape)}")
    n = pts.shape[0]
    for name, t in (("code", code), ("elem", elem), ("dist2", dist2)):
        if t.numel() < n:
            raise ValueError(f"{name} has {t.numel()} entries, need {n}")
    if r.numel() < n * info.dr or (r.dim() == 2 and r.shape[1] != info.dr) or r.dim() > 2:
        raise ValueError(f"r must have shape (n, {info.dr}) with n >= {n}, got {tuple(r.shape)}")
    return n


def _eval_shapes(mesh, code, elem, r, field, nc: int, out, field_N: int | None = None) -> int:
    """As _find_shapes for an eval call: elem and r [n][dr] cover the n
    entries of code, field holds nc * NE * field_N^dr values and out nc * n."""
    info = fp_get_info(mesh)
    n = code.shape[0] if code.dim() > 0 else 0
    Nf = info.N if field_N is None else field_N
    if elem.numel() < n or r.numel() < n * info.dr:
        raise ValueError(f"elem and r must cover the {n} points of code")
    if field.numel() < nc * info.NE * Nf ** info.dr:
        raise ValueError(f"field has {field.numel()} values, need {nc} x {info.NE} x {Nf}^{info.dr}")
    if out.numel() < nc * n:
        raise ValueError(f"out has {out.numel()} values, need {nc} x {n}")
    return n


def fp_findpts(mesh, pts, code, elem, r, dist2, stream=None) -> None:
    import torch
    n = _find_shapes(mesh, pts, code, elem, r, dist2)
    _check("fp_findpts", lib().fp_findpts(
        mesh, _ptr(pts, torch.float64, "pts"), n, _ptr(code, torch.int32, "code"),
        _ptr(elem, torch.int32, "elem"), _ptr(r, torch.float64, "r"),
        _ptr(dist2, torch.float64, "dist2"), _stream(stream)))


def fp_findpts_stats(mesh, pts, code, elem, r, dist2, stats, stream=None) -> None:
    import torch
    n = _find_shapes(mesh, pts, code, elem, r, dist2)
    if stats.numel() < FP_NSTATS:
        raise ValueError(f"stats: need {FP_NSTATS} int64 values, got {stats.numel()}")
    _check("fp_findpts_stats", lib().fp_findpts_stats(
        mesh, _ptr(pts, torch.float64, "pts"), n, _ptr(code, torch.int32, "code"),
        _ptr(elem, torch.int32, "elem"), _ptr(r, torch.float64, "r"),
        _ptr(dist2, torch.float64, "dist2"), _ptr(stats, torch.int64, "stats"), _stream(stream)))


def fp_eval(mesh, code, elem, r, field, nc: int, out, stream=None) -> None:
    import torch
    n = _eval_shapes(mesh, code, elem, r, field, nc, out)
    _check("fp_eval", lib().fp_eval(
        mesh, _ptr(code, torch.int32, "code"), _ptr(elem, torch.int32, "elem"),
        _ptr(r, torch.float64, "r"), n, _ptr(field, torch.float64, "field"), int(nc),
        _ptr(out, torch.float64, "out"), _stream(stream)))


def fp_eval_order(mesh, code, elem, r, field, field_order: int, nc: int, out, stream=None) -> None:
    import torch
    n = _eval_shapes(mesh, code, elem, r, field, nc, out, field_N=int(field_order) + 1)
    _check("fp_eval_order", lib().fp_eval_order(
        mesh, _ptr(code, torch.int32, "code"), _ptr(elem, torch.int32, "elem"),
        _ptr(r, torch.float64, "r"), n, _ptr(field, torch.float64, "field"), int(field_order), int(nc),
        _ptr(out, torch.float64, "out"), _stream(stream)))


def fp_findpts_host(mesh, pts, code, elem, r, dist2, field=None, nc: int = 0, out=None, chunk: int = 0,
                    stream=None) -> None:
    """Host tensors (pinned CPU torch tensors for overlapped copies): pts
    [n][d] float64; outputs code, elem int32 [n], r [n][dr], dist2 [n]; field
    a device tensor [nc][NE][N^dr] or None, out [nc][n] host."""
    import torch

    def hp(t, dt, name):
        if t.device.type != "cpu" or t.dtype != dt or not t.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous CPU {dt} tensor")
        return ctypes.c_void_p(t.data_ptr())
    n = _find_shapes(mesh, pts, code, elem, r, dist2)
    if field is not None and (out is None or out.numel() < int(nc) * n):
        raise ValueError(f"out must hold {int(nc)} x {n} values")
    _check("fp_findpts_host", lib().fp_findpts_host(
        mesh, hp(pts, torch.float64, "pts"), n, hp(code, torch.int32, "code"), hp(elem, torch.int32, "elem"),
        hp(r, torch.float64, "r"), hp(dist2, torch.float64, "dist2"),
        None if field is None else _ptr(field, torch.float64, "field"), int(nc) if field is not None else 0,
        None if field is None else hp(out, torch.float64, "out"), int(chunk), _stream(stream)))


def fp_get_info(mesh) -> FpMeshInfo:
    info = FpMeshInfo()
    _check("fp_get_info", lib().fp_get_info(mesh, ctypes.byref(info)))
    return info


def fp_get_boxes(mesh, aabb, obb_c, obb_A, stream=None) -> None:
    import torch
    _check("fp_get_boxes", lib().fp_get_boxes(mesh, _ptr(aabb, torch.float64), _ptr(obb_c, torch.float64),
                                              _ptr(obb_A, torch.float64), _stream(stream)))


def fp_get_curvature(mesh, curv, stream=None) -> None:
    import torch
    _check("fp_get_curvature", lib().fp_get_curvature(mesh, _ptr(curv, torch.float64, "curv"), _stream(stream)))


def fp_get_grid(mesh, cell_start, cell_elems, stream=None) -> None:
    import torch
    _check("fp_get_grid", lib().fp_get_grid(mesh, _ptr(cell_start, torch.int32), _ptr(cell_elems, torch.int32),
                                            _stream(stream)))


def fp_device_status(mesh, stream=None) -> int:
    s = _int(0)
    _check("fp_device_status", lib().fp_device_status(mesh, ctypes.byref(s), _stream(stream)))
    return s.value


def fp_set_timing(mesh, on: bool) -> None:
    _check("fp_set_timing", lib().fp_set_timing(mesh, int(bool(on))))


def fp_kernel_times(mesh):
    """(ms, calls): per stage FP_TIME_* the summed kernel milliseconds and
    the number of intervals since the last read."""
    ms = (ctypes.c_double * FP_NTIMES)()
    calls = (_i64 * FP_NTIMES)()
    _check("fp_kernel_times", lib().fp_kernel_times(mesh, ms, calls))
    return list(ms), list(calls)


def fp_alu_peak(which: int, iters: int = 4000, stream=None) -> float:
    g = ctypes.c_double(0.0)
    _check("fp_alu_peak", lib().fp_alu_peak(int(which), int(iters), ctypes.byref(g), _stream(stream)))
    return g.value


class FpBatchItem(ctypes.Structure):
    _fields_ = [("mesh", ctypes.c_int), ("pts", _vp), ("n", ctypes.c_int64), ("code", _vp),
                ("elem", _vp), ("r", _vp), ("dist2", _vp), ("field", _vp), ("nc", ctypes.c_int),
                ("out", _vp)]


class FpBatchClassInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("d", ctypes.c_int), ("dr", ctypes.c_int), ("n_items", ctypes.c_int),
                ("n_points", ctypes.c_int64), ("ctas_per_sm", ctypes.c_int), ("chunk_points", ctypes.c_int),
                ("tuned_ms", ctypes.c_float)]


def _batch_sig():
    L = lib()
    if getattr(L, "_batch_sig", False):
        return L
    L.fp_batch_create.argtypes = [ctypes.POINTER(_vp), _int, ctypes.POINTER(FpBatchItem), _int, _int, _vp,
                                  ctypes.POINTER(_vp)]
    L.fp_batch_run.argtypes = [_vp, _vp]
    L.fp_batch_autotune.argtypes = [_vp, _vp]
    L.fp_batch_free.argtypes = [_vp]
    L.fp_batch_num_classes.argtypes = [_vp]
    L.fp_batch_describe.argtypes = [_vp, _int, ctypes.POINTER(FpBatchClassInfo)]
    L.fp_batch_set_fused.argtypes = [_vp, _int]
    for f in ("fp_batch_create", "fp_batch_run", "fp_batch_autotune", "fp_batch_free",
              "fp_batch_num_classes", "fp_batch_describe", "fp_batch_set_fused"):
        getattr(L, f).restype = _int
    L._batch_sig = True
    return L


def fp_batch_create(meshes, items, precision: int = FP_F64, stream=None) -> _vp:
    arr = (_vp * len(meshes))(*[m if isinstance(m, _vp) else _vp(m) for m in meshes])
    its = (FpBatchItem * len(items))(*items)
    h = _vp()
    _check("fp_batch_create", _batch_sig().fp_batch_create(arr, len(meshes), its, len(items), int(precision),
                                                           _stream(stream), ctypes.byref(h)))
    return h


def fp_batch_run(batch, stream=None) -> None:
    _check("fp_batch_run", _batch_sig().fp_batch_run(batch, _stream(stream)))


def fp_batch_set_fused(batch, on: bool) -> None:
    _check("fp_batch_set_fused", _batch_sig().fp_batch_set_fused(batch, int(bool(on))))


def fp_batch_autotune(batch, stream=None) -> None:
    _check("fp_batch_autotune", _batch_sig().fp_batch_autotune(batch, _stream(stream)))


def fp_batch_num_classes(batch) -> int:
    return _batch_sig().fp_batch_num_classes(batch)


def fp_batch_describe(batch, i: int) -> FpBatchClassInfo:
    info = FpBatchClassInfo()
    _check("fp_batch_describe", _batch_sig().fp_batch_describe(batch, int(i), ctypes.byref(info)))
    return info


def fp_batch_free(batch) -> None:
    _check("fp_batch_free", _batch_sig().fp_batch_free(batch))


class Batch:
    """Find (+ eval) for many (Mesh, points[, field]) items in one graph
    launch; allocates every item's outputs as torch tensors."""

    def __init__(self, entries, precision: int = FP_F64, stream=None):
        import torch
        meshes, idx = [], {}
        self.entries, self.outputs, items = entries, [], []
        for mesh, pts, field in entries:
            if id(mesh) not in idx:
                idx[id(mesh)] = len(meshes)
                meshes.append(mesh.handle)
            n = pts.shape[0]
            dev = pts.device
            code = torch.empty(n, dtype=torch.int32, device=dev)
            elem = torch.empty(n, dtype=torch.int32, device=dev)
            r = torch.empty((n, mesh.dr), dtype=torch.float64, device=dev)
            d2 = torch.empty(n, dtype=torch.float64, device=dev)
            nc = 0 if field is None else field.numel() // (mesh.NE * mesh.N ** mesh.dr)
            out = None if field is None else torch.empty((nc, n), dtype=torch.float64, device=dev)
            self.outputs.append((code, elem, r, d2, out))
            items.append(FpBatchItem(idx[id(mesh)], _ptr(pts, torch.float64, "pts"), n, _ptr(code), _ptr(elem),
                                     _ptr(r), _ptr(d2), _ptr(field, torch.float64, "field"), nc, _ptr(out)))
        self.handle = fp_batch_create(meshes, items, precision, stream)

    def run(self, stream=None):
        fp_batch_run(self.handle, stream)

    def autotune(self, stream=None):
        fp_batch_autotune(self.handle, stream)

    def set_fused(self, on: bool):
        """One persistent find launch over all element shapes (True) or one
        per shape (False, the default)."""
        fp_batch_set_fused(self.handle, on)

    def classes(self):
        return [fp_batch_describe(self.handle, i) for i in range(fp_batch_num_classes(self.handle))]

    def close(self):
        if self.handle is not None:
            fp_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


FP_ECANCELED = -8
FP_REQ_REMAP, FP_REQ_PARTICLE = 0, 1


class FpServerOpts(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_size_t), ("max_active", ctypes.c_int), ("precision", ctypes.c_int),
                ("tick_timeout_s", ctypes.c_double), ("tick_points", ctypes.c_int64), ("policy", ctypes.c_int),
                ("slack_base", ctypes.c_double), ("slack_factor", ctypes.c_double)]


class FpServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("cancelled", ctypes.c_int64), ("ticks", ctypes.c_int64), ("timeouts", ctypes.c_int64),
                ("active", ctypes.c_int64), ("queued", ctypes.c_int64), ("bytes_in_use", ctypes.c_size_t)]


def _server_sig():
    L = lib()
    if getattr(L, "_server_sig", False):
        return L
    P = ctypes.POINTER
    sig = {
        "fp_server_opts_default": ([P(FpServerOpts)], None),
        "fp_server_create": ([P(_vp), _int, P(_vp), P(_int), P(_vp), P(FpServerOpts), P(_vp)], _int),
        "fp_server_submit": ([_vp, _int, _int, _vp, _i64, _int, ctypes.c_double, _vp, _vp, _vp, _vp, _vp,
                              P(_i64)], _int),
        "fp_server_poll": ([_vp, _i64, P(_int), P(_int)], _int),
        "fp_server_wait": ([_vp, _i64, ctypes.c_double], _int),
        "fp_server_cancel": ([_vp, _i64], _int),
        "fp_server_timing": ([_vp, _i64, P(ctypes.c_double), P(ctypes.c_double)], _int),
        "fp_server_release": ([_vp, _i64], _int),
        "fp_server_get_stats": ([_vp, P(FpServerStats)], _int),
        "fp_server_destroy": ([_vp], _int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    L._server_sig = True
    return L


def fp_server_opts_default() -> FpServerOpts:
    o = FpServerOpts()
    _server_sig().fp_server_opts_default(ctypes.byref(o))
    return o


def _hptr(a):
    """Host pointer of a numpy array or a CPU torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return _vp(a.data_ptr())
    return _vp(a.ctypes.data)


class Server:
    """Continuous-batching server over resident meshes (see fp_server_*).
    entries: list of (Mesh, remap_field or None, velocity_field or None)
    with fields as device tensors [nc][NE][N^dr]."""

    def __init__(self, entries, mem_budget: int = 1 << 30, max_active: int = 64, precision: int = FP_MIXED,
                 tick_timeout_s: float = 30.0, tick_points: int = 1 << 19, policy: int | None = None,
                 slack_base: float | None = None, slack_factor: float | None = None):
        L = _server_sig()
        o = fp_server_opts_default()
        o.mem_budget, o.max_active, o.precision, o.tick_timeout_s = mem_budget, max_active, precision, tick_timeout_s
        o.tick_points = tick_points
        if policy is not None:
            o.policy = policy
        if slack_base is not None:
            o.slack_base = slack_base
        if slack_factor is not None:
            o.slack_factor = slack_factor
        n = len(entries)
        self.meshes = [e[0] for e in entries]
        self._keep = entries
        mh = (_vp * n)(*[e[0].handle for e in entries])
        rf = (_vp * n)(*[None if e[1] is None else e[1].data_ptr() for e in entries])
        nc = (_int * n)(*[0 if e[1] is None else e[1].numel() // (e[0].NE * e[0].N ** e[0].dr) for e in entries])
        vf = (_vp * n)(*[None if e[2] is None else e[2].data_ptr() for e in entries])
        self.handle = _vp()
        _check("fp_server_create", L.fp_server_create(mh, n, rf, nc, vf, ctypes.byref(o), ctypes.byref(self.handle)))
        self._bufs = {}

    def submit(self, mesh: int, kind: int, pts, rk_steps: int = 0, dt: float = 0.0, outputs=None) -> int:
        """pts: host float64 [n][d] (pinned torch tensor or numpy array);
        outputs: (code, elem, r, dist2, out) host arrays, allocated if None."""
        import numpy as np
        m = self.meshes[mesh]
        n = pts.shape[0]
        if outputs is None:
            ncomp = m.d if kind == FP_REQ_PARTICLE else max(1, self._nc(mesh))
            outputs = (np.empty(n, np.int32), np.empty(n, np.int32), np.empty((n, m.dr)), np.empty(n),
                       np.empty((n, m.d)) if kind == FP_REQ_PARTICLE else np.empty((ncomp, n)))
        rid = _i64(0)
        _check("fp_server_submit", _server_sig().fp_server_submit(
            self.handle, mesh, kind, _hptr(pts), n, rk_steps, dt, *[_hptr(a) for a in outputs], ctypes.byref(rid)))
        self._bufs[rid.value] = (pts, outputs)
        return rid.value

    def _nc(self, mesh):
        e = self._keep[mesh]
        return 0 if e[1] is None else e[1].numel() // (e[0].NE * e[0].N ** e[0].dr)

    def wait(self, rid: int, timeout_s: float = 60.0):
        """Returns the request's outputs; raises FindptsError on failure or timeout."""
        _check("fp_server_wait", _server_sig().fp_server_wait(self.handle, rid, timeout_s))
        return self._bufs[rid][1]

    def poll(self, rid: int):
        done, st = _int(0), _int(0)
        _check("fp_server_poll", _server_sig().fp_server_poll(self.handle, rid, ctypes.byref(done), ctypes.byref(st)))
        return bool(done.value), st.value

    def cancel(self, rid: int) -> int:
        return _server_sig().fp_server_cancel(self.handle, rid)

    def timing(self, rid: int):
        q, t = ctypes.c_double(0), ctypes.c_double(0)
        _check("fp_server_timing", _server_sig().fp_server_timing(self.handle, rid, ctypes.byref(q), ctypes.byref(t)))
        return q.value, t.value

    def release(self, rid: int) -> None:
        _check("fp_server_release", _server_sig().fp_server_release(self.handle, rid))
        self._bufs.pop(rid, None)

    def stats(self) -> FpServerStats:
        st = FpServerStats()
        _check("fp_server_get_stats", _server_sig().fp_server_get_stats(self.handle, ctypes.byref(st)))
        return st

    def close(self):
        if self.handle is not None:
            _check("fp_server_destroy", _server_sig().fp_server_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


FP_NOALLOC_MAX_POINTS = 1 << 20


def fp_findpts_mixed_noalloc(mesh, pts, code, elem, r, dist2, stream=None) -> None:
    """Mixed-precision find that allocates no device memory (at most
    FP_NOALLOC_MAX_POINTS points per call; calls that overlap on the GPU
    race on the library's one scratch array)."""
    import torch
    f = lib().fp_findpts_mixed_noalloc
    f.argtypes = [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp]
    f.restype = _int
    n = _find_shapes(mesh, pts, code, elem, r, dist2)
    _check("fp_findpts_mixed_noalloc", f(
        mesh, _ptr(pts, torch.float64, "pts"), n, _ptr(code, torch.int32, "code"),
        _ptr(elem, torch.int32, "elem"), _ptr(r, torch.float64, "r"),
        _ptr(dist2, torch.float64, "dist2"), _stream(stream)))


class Mesh:
    """Owns an fp_mesh handle; allocates outputs as torch tensors."""

    def __init__(self, coords, d: int, dr: int, order: int, stream=None, **opts):
        o = fp_opts_default()
        for k, v in opts.items():
            setattr(o, k, v)
        self.d, self.dr, self.order = d, dr, order
        self.N = order + 1
        self.NE = coords.numel() // (d * self.N ** dr)
        self.handle = fp_setup(coords, d, dr, order, o, stream)

    def close(self):
        if self.handle is not None:
            fp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, precision: int):
        fp_set_precision(self.handle, precision)

    def set_point_order(self, order: int):
        fp_set_point_order(self.handle, order)

    def find(self, pts, stream=None, stats=None):
        import torch
        n = pts.shape[0]
        dev = pts.device
        code = torch.empty(n, dtype=torch.int32, device=dev)
        elem = torch.empty(n, dtype=torch.int32, device=dev)
        r = torch.empty((n, self.dr), dtype=torch.float64, device=dev)
        dist2 = torch.empty(n, dtype=torch.float64, device=dev)
        if stats is None:
            fp_findpts(self.handle, pts, code, elem, r, dist2, stream)
        else:
            fp_findpts_stats(self.handle, pts, code, elem, r, dist2, stats, stream)
        return code, elem, r, dist2

    def eval(self, code, elem, r, field, stream=None, order=None):
        """Interpolates field ([nc][NE][(order+1)^dr]; order defaults to the
        mesh's) at the find output (code, elem, r)."""
        import torch
        Nf = self.N if order is None else order + 1
        nc = field.numel() // (self.NE * Nf ** self.dr)
        out = torch.empty((nc, code.shape[0]), dtype=torch.float64, device=code.device)
        if order is None:
            fp_eval(self.handle, code, elem, r, field, nc, out, stream)
        else:
            fp_eval_order(self.handle, code, elem, r, field, order, nc, out, stream)
        return out

    def find_host(self, pts, field=None, chunk: int = 0, stream=None):
        """fp_findpts_host: pts a CPU float64 tensor [n][d] (pinned for
        overlapped copies); returns pinned CPU tensors (code, elem, r, dist2)
        and, with a device field [nc][NE][N^dr], the values [nc][n]."""
        import torch
        n = pts.shape[0]
        pin = pts.is_pinned()
        code = torch.empty(n, dtype=torch.int32, pin_memory=pin)
        elem = torch.empty(n, dtype=torch.int32, pin_memory=pin)
        r = torch.empty((n, self.dr), dtype=torch.float64, pin_memory=pin)
        dist2 = torch.empty(n, dtype=torch.float64, pin_memory=pin)
        nc = 0 if field is None else field.numel() // (self.NE * self.N ** self.dr)
        out = None if field is None else torch.empty((nc, n), dtype=torch.float64, pin_memory=pin)
        fp_findpts_host(self.handle, pts, code, elem, r, dist2, field, nc, out, chunk, stream)
        return (code, elem, r, dist2) if field is None else (code, elem, r, dist2, out)

    def info(self) -> FpMeshInfo:
        return fp_get_info(self.handle)

    def boxes(self):
        import torch
        dev = torch.device("cuda")
        aabb = torch.empty((self.NE, 2 * self.d), dtype=torch.float64, device=dev)
        oc = torch.empty((self.NE, self.d), dtype=torch.float64, device=dev)
        oA = torch.empty((self.NE, self.d, self.d), dtype=torch.float64, device=dev)
        fp_get_boxes(self.handle, aabb, oc, oA)
        return aabb, oc, oA

    def curvature(self):
        """Per-element curvature bounds (fp_get_curvature), [NE] FP64 on the device."""
        import torch
        curv = torch.empty(self.NE, dtype=torch.float64, device="cuda")
        fp_get_curvature(self.handle, curv)
        return curv

    def grid(self):
        import torch
        info = self.info()
        cs = torch.empty(info.n_cells + 1, dtype=torch.int32, device="cuda")
        ce = torch.empty(max(info.n_cell_entries, 1), dtype=torch.int32, device="cuda")
        fp_get_grid(self.handle, cs, ce)
        return cs, ce[:info.n_cell_entries]

    def device_status(self) -> int:
        return fp_device_status(self.handle)
