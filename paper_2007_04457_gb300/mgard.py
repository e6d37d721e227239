"""ctypes binding of the C ABI in ``include/mgard.h``.

Argument marshalling only: every step of the decomposition runs in the CUDA
library.  The module-level functions carry the C names and take raw
integers (device pointers, byte counts, stream handles); ``Plan`` wraps them
for torch tensors, using torch only for device memory and streams.

Importing this module loads ``lib/libmgard_gb300.so`` and raises if it is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

F32, F64, F32_MIXED = 0, 1, 2
_DTYPE_CODES = {"f32": F32, "f64": F64, "f32_mixed": F32_MIXED}

STATUS = {
    0: "MGARD_OK",
    1: "MGARD_ERR_INVALID_ARG",
    2: "MGARD_ERR_UNSUPPORTED_SHAPE",
    3: "MGARD_ERR_WORKSPACE",
    4: "MGARD_ERR_CUDA",
    5: "MGARD_ERR_TIMEOUT",
    6: "MGARD_ERR_INTERNAL",
}


class MgardError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str):
        super().__init__(f"{what}: {STATUS.get(status, status)}: {detail}")
        self.status = status


def _load() -> ctypes.CDLL:
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA library {path} is not built; run paper_2007_04457_gb300.build.build() "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, sz, i64p = ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int64)
    dpp = ctypes.POINTER(ctypes.POINTER(ctypes.c_double))
    sigs = {
        "mgard_plan_create": ([ctypes.c_int, i64p, ctypes.c_int, dpp, ctypes.c_int,
                               ctypes.POINTER(vp)], ctypes.c_int),
        "mgard_plan_destroy": ([vp], ctypes.c_int),
        "mgard_plan_levels": ([vp], ctypes.c_int),
        "mgard_workspace_bytes": ([vp], sz),
        "mgard_plan_launches": ([vp, ctypes.c_int], ctypes.c_int),
        "mgard_decompose": ([vp, vp, vp, sz, vp], ctypes.c_int),
        "mgard_recompose": ([vp, vp, vp, sz, vp], ctypes.c_int),
        "mgard_recompose_classes": ([vp, ctypes.c_int, vp, vp, sz, vp], ctypes.c_int),
        "mgard_decompose_adjoint": ([vp, vp, vp, sz, vp], ctypes.c_int),
        "mgard_recompose_adjoint": ([vp, vp, vp, sz, vp], ctypes.c_int),
        "mgard_decompose_host": ([vp, vp, vp, vp, vp, sz, vp], ctypes.c_int),
        "mgard_recompose_host": ([vp, vp, vp, vp, vp, sz, vp], ctypes.c_int),
        "mgard_profile_enable": ([vp, ctypes.c_int], ctypes.c_int),
        "mgard_profile_read": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "mgard_plan_tune": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "mgard_plan_get_tune": ([vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "mgard_plan_check": ([vp, vp, vp], ctypes.c_int),
        "mgard_plan_create_per_dim": ([ctypes.c_int, i64p, ctypes.POINTER(ctypes.c_int), dpp, ctypes.c_int,
                                       ctypes.POINTER(vp)], ctypes.c_int),
        "mgard_batch_create": ([ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp)],
                               ctypes.c_int),
        "mgard_batch_destroy": ([vp], ctypes.c_int),
        "mgard_batch_workspace_bytes": ([vp], sz),
        "mgard_batch_decompose": ([vp, ctypes.POINTER(vp), vp, sz, vp], ctypes.c_int),
        "mgard_batch_recompose": ([vp, ctypes.POINTER(vp), vp, sz, vp], ctypes.c_int),
        "mgard_batch_tune": ([vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "mgard_batch_get": ([vp, ctypes.c_int], ctypes.c_longlong),
        "mgard_batch_check": ([vp, vp], ctypes.c_int),
        "mgard_batch_profile_read": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)],
                                     ctypes.c_int),
        "mgard_decompose_noalloc": ([ctypes.c_int, i64p, ctypes.c_int, ctypes.c_int, vp, vp], ctypes.c_int),
        "mgard_probe_fp64_peak": ([ctypes.POINTER(ctypes.c_double), vp], ctypes.c_int),
        "mgard_quantize": ([vp, ctypes.POINTER(ctypes.c_double), vp, vp, vp], ctypes.c_int),
        "mgard_dequantize": ([vp, ctypes.POINTER(ctypes.c_double), vp, vp, vp], ctypes.c_int),
        "mgard_decompose_quantize": ([vp, ctypes.POINTER(ctypes.c_double), vp, vp, vp, sz, vp], ctypes.c_int),
        "mgard_dequantize_recompose": ([vp, ctypes.POINTER(ctypes.c_double), vp, vp, vp, sz, vp], ctypes.c_int),
        "mgard_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "mgard_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


LIB = _load()
LIB_PATH = _build.LIB


def _check(status: int, what: str) -> None:
    if status != 0:
        raise MgardError(status, what, LIB.mgard_last_error().decode())


# --------------------------------------------------------------- C-named calls

def _coords_arg(ndim, coords, keep):
    if coords is None:
        return None
    import numpy as np
    arrs = [np.ascontiguousarray(c, dtype=np.float64) for c in coords]
    keep.extend(arrs)
    return (ctypes.POINTER(ctypes.c_double) * ndim)(
        *[a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in arrs])


def mgard_plan_create(ndim, dims, nlevels, coords, dtype) -> int:
    """Returns the plan handle (an integer).  coords: None or ndim float64
    numpy arrays."""
    d = (ctypes.c_int64 * ndim)(*[int(v) for v in dims])
    out = ctypes.c_void_p()
    keep = []
    cptr = _coords_arg(ndim, coords, keep)
    _check(LIB.mgard_plan_create(ndim, d, nlevels, cptr, dtype, ctypes.byref(out)),
           "mgard_plan_create")
    return out.value


def mgard_plan_create_per_dim(ndim, dims, levels, coords, dtype) -> int:
    """A plan with a level count per dimension (levels: None, or ndim ints,
    -1 = that dimension's maximum)."""
    d = (ctypes.c_int64 * ndim)(*[int(v) for v in dims])
    lv = None if levels is None else (ctypes.c_int * ndim)(*[int(v) for v in levels])
    out = ctypes.c_void_p()
    keep = []
    cptr = _coords_arg(ndim, coords, keep)
    _check(LIB.mgard_plan_create_per_dim(ndim, d, lv, cptr, dtype, ctypes.byref(out)),
           "mgard_plan_create_per_dim")
    return out.value


def mgard_plan_destroy(plan: int) -> None:
    _check(LIB.mgard_plan_destroy(plan), "mgard_plan_destroy")


def mgard_plan_levels(plan: int) -> int:
    return LIB.mgard_plan_levels(plan)


def mgard_workspace_bytes(plan: int) -> int:
    return LIB.mgard_workspace_bytes(plan)


def mgard_plan_launches(plan: int, recompose: int) -> int:
    return LIB.mgard_plan_launches(plan, recompose)


def mgard_decompose(plan: int, d_data: int, d_ws: int, ws_bytes: int, stream: int) -> None:
    _check(LIB.mgard_decompose(plan, d_data, d_ws, ws_bytes, stream), "mgard_decompose")


def mgard_recompose(plan: int, d_data: int, d_ws: int, ws_bytes: int, stream: int) -> None:
    _check(LIB.mgard_recompose(plan, d_data, d_ws, ws_bytes, stream), "mgard_recompose")


def mgard_recompose_classes(plan: int, nclasses: int, d_data: int, d_ws: int, ws_bytes: int,
                            stream: int) -> None:
    _check(LIB.mgard_recompose_classes(plan, nclasses, d_data, d_ws, ws_bytes, stream),
           "mgard_recompose_classes")


def mgard_decompose_adjoint(plan: int, d_data: int, d_ws: int, ws_bytes: int, stream: int) -> None:
    _check(LIB.mgard_decompose_adjoint(plan, d_data, d_ws, ws_bytes, stream), "mgard_decompose_adjoint")


def mgard_recompose_adjoint(plan: int, d_data: int, d_ws: int, ws_bytes: int, stream: int) -> None:
    _check(LIB.mgard_recompose_adjoint(plan, d_data, d_ws, ws_bytes, stream), "mgard_recompose_adjoint")


def mgard_decompose_host(plan: int, h_in: int, h_out: int, d_data: int, d_ws: int, ws_bytes: int,
                         stream: int) -> None:
    _check(LIB.mgard_decompose_host(plan, h_in, h_out, d_data, d_ws, ws_bytes, stream),
           "mgard_decompose_host")


def mgard_recompose_host(plan: int, h_in: int, h_out: int, d_data: int, d_ws: int, ws_bytes: int,
                         stream: int) -> None:
    _check(LIB.mgard_recompose_host(plan, h_in, h_out, d_data, d_ws, ws_bytes, stream),
           "mgard_recompose_host")


def mgard_profile_enable(plan: int, levels: int) -> None:
    _check(LIB.mgard_profile_enable(plan, levels), "mgard_profile_enable")


def mgard_profile_read(plan: int, cap: int = 64):
    """List of (kind, level, launches, ms) since the last read."""
    kinds = (ctypes.c_int * cap)()
    levels = (ctypes.c_int * cap)()
    launches = (ctypes.c_int * cap)()
    ms = (ctypes.c_double * cap)()
    n = LIB.mgard_profile_read(plan, cap, kinds, levels, launches, ms)
    if n < 0:
        raise MgardError(6, "mgard_profile_read", mgard_last_error())
    return [(kinds[i], levels[i], launches[i], ms[i]) for i in range(n)]


def mgard_plan_tune(plan: int, level: int, param: int, value: int) -> None:
    _check(LIB.mgard_plan_tune(plan, level, param, value), "mgard_plan_tune")


def mgard_plan_get_tune(plan: int, level: int, param: int) -> int:
    return LIB.mgard_plan_get_tune(plan, level, param)


def mgard_plan_check(plan: int, d_ws: int, stream: int) -> None:
    _check(LIB.mgard_plan_check(plan, d_ws, stream), "mgard_plan_check")


NOALLOC_SCRATCH_BYTES = 32 << 20


def mgard_decompose_noalloc(ndim, dims, nlevels, dtype, d_data: int, stream: int) -> None:
    """Uniform-grid decomposition with tables and workspace in the library's
    static scratch (no device allocation; calls must not overlap)."""
    d = (ctypes.c_int64 * ndim)(*[int(v) for v in dims])
    _check(LIB.mgard_decompose_noalloc(ndim, d, nlevels, dtype, d_data, stream), "mgard_decompose_noalloc")


def _bins_arg(bins):
    arr = (ctypes.c_double * len(bins))(*[float(b) for b in bins])
    return arr


def mgard_quantize(plan: int, bins, d_data: int, d_codes: int, stream: int) -> None:
    _check(LIB.mgard_quantize(plan, _bins_arg(bins), d_data, d_codes, stream), "mgard_quantize")


def mgard_dequantize(plan: int, bins, d_codes: int, d_data: int, stream: int) -> None:
    _check(LIB.mgard_dequantize(plan, _bins_arg(bins), d_codes, d_data, stream), "mgard_dequantize")


def mgard_decompose_quantize(plan: int, bins, d_data: int, d_codes: int, d_ws: int, ws_bytes: int,
                             stream: int) -> None:
    _check(LIB.mgard_decompose_quantize(plan, _bins_arg(bins), d_data, d_codes, d_ws, ws_bytes, stream),
           "mgard_decompose_quantize")


def mgard_dequantize_recompose(plan: int, bins, d_codes: int, d_data: int, d_ws: int, ws_bytes: int,
                               stream: int) -> None:
    _check(LIB.mgard_dequantize_recompose(plan, _bins_arg(bins), d_codes, d_data, d_ws, ws_bytes, stream),
           "mgard_dequantize_recompose")


def mgard_probe_fp64_peak(stream: int) -> float:
    """FP64 FMA rate of the current device in TFLOP/s (measurement support)."""
    out = ctypes.c_double(0.0)
    _check(LIB.mgard_probe_fp64_peak(ctypes.byref(out), stream), "mgard_probe_fp64_peak")
    return out.value


def mgard_status_string(status: int) -> str:
    return LIB.mgard_status_string(status).decode()


def mgard_last_error() -> str:
    return LIB.mgard_last_error().decode()


# --------------------------------------------------------------- torch wrapper

def _torch():
    import torch
    return torch


class Plan:
    """A plan for one shape / precision, bound to the current CUDA device.

    shape:   node counts, slowest first (1 to 3 dims after squeezing 1s)
    nlevels: number of levels, -1 for the maximum the shape allows
    coords:  None (uniform) or one increasing float64 array per dimension
    dtype:   "f32", "f64" or "f32_mixed"
    dim_levels: None, or a level count per dimension (-1 = that dimension's
             maximum; "max" = all maxima): each dimension coarsens in its
             first dim_levels[k] steps and then keeps its nodes
    """

    def __init__(self, shape, nlevels: int = -1, coords=None, dtype: str = "f32", dim_levels=None):
        if dtype not in _DTYPE_CODES:
            raise ValueError(f"dtype must be one of {sorted(_DTYPE_CODES)}")
        self.shape = tuple(int(n) for n in shape)
        self.dtype = dtype
        if dim_levels is None:
            self.handle = mgard_plan_create(len(self.shape), self.shape, nlevels, coords,
                                            _DTYPE_CODES[dtype])
        else:
            # a level count per dimension ("max" = every dimension its maximum)
            lv = None if dim_levels == "max" else list(dim_levels)
            self.handle = mgard_plan_create_per_dim(len(self.shape), self.shape, lv, coords,
                                                    _DTYPE_CODES[dtype])
        self.levels = mgard_plan_levels(self.handle)
        self.workspace_bytes = mgard_workspace_bytes(self.handle)
        self._ws = None

    @property
    def torch_dtype(self):
        torch = _torch()
        return torch.float64 if self.dtype == "f64" else torch.float32

    def launches(self, recompose: bool = False) -> int:
        return mgard_plan_launches(self.handle, int(recompose))

    def workspace(self, device=None):
        """A cached device workspace of the required size (torch allocator)."""
        torch = _torch()
        if self._ws is None or (device is not None and self._ws.device != torch.device(device)):
            self._ws = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8,
                                   device=device or "cuda")
        return self._ws

    def _args(self, data, workspace, stream):
        torch = _torch()
        if not data.is_cuda or not data.is_contiguous() or data.dtype != self.torch_dtype:
            raise ValueError(f"data must be a contiguous CUDA {self.torch_dtype} tensor")
        if tuple(n for n in data.shape if n != 1) != tuple(n for n in self.shape if n != 1):
            raise ValueError(f"data shape {tuple(data.shape)} does not match plan {self.shape}")
        ws = workspace if workspace is not None else self.workspace(data.device)
        s = stream if stream is not None else torch.cuda.current_stream(data.device)
        return data.data_ptr(), ws.data_ptr(), ws.numel() * ws.element_size(), s.cuda_stream

    def decompose(self, data, workspace=None, stream=None):
        """In-place decomposition of a CUDA tensor; returns it."""
        mgard_decompose(self.handle, *self._args(data, workspace, stream))
        return data

    def recompose(self, data, workspace=None, stream=None):
        """In-place recomposition of a CUDA tensor; returns it."""
        mgard_recompose(self.handle, *self._args(data, workspace, stream))
        return data

    def recompose_classes(self, data, nclasses: int, workspace=None, stream=None):
        """In place: rebuild the field from its first `nclasses` coefficient
        classes (1 .. levels + 1; the finer classes count as zero)."""
        mgard_recompose_classes(self.handle, int(nclasses), *self._args(data, workspace, stream))
        return data

    def decompose_adjoint(self, data, workspace=None, stream=None):
        """In place: data (a cotangent of the decomposition's output) becomes
        the cotangent of its input (transpose of decompose)."""
        mgard_decompose_adjoint(self.handle, *self._args(data, workspace, stream))
        return data

    def recompose_adjoint(self, data, workspace=None, stream=None):
        """In place transpose of recompose."""
        mgard_recompose_adjoint(self.handle, *self._args(data, workspace, stream))
        return data

    def _codes(self, data, codes):
        torch = _torch()
        if codes is None:
            codes = torch.empty(data.shape, dtype=torch.int32, device=data.device)
        if not codes.is_cuda or codes.dtype != torch.int32 or codes.numel() != data.numel() \
                or not codes.is_contiguous():
            raise ValueError("codes must be a contiguous CUDA int32 tensor of the field's size")
        return codes

    def quantize(self, data, bins, codes=None, stream=None):
        """int32 codes of a decomposed field, one bin width per coefficient
        class (levels + 1 of them, class 0 = coarsest values)."""
        codes = self._codes(data, codes)
        d, _, _, st = self._args(data, None, stream)
        mgard_quantize(self.handle, bins, d, codes.data_ptr(), st)
        return codes

    def dequantize(self, codes, bins, data, stream=None):
        """codes x bin width of each node's class, into the field `data`."""
        self._codes(data, codes)
        d, _, _, st = self._args(data, None, stream)
        mgard_dequantize(self.handle, bins, codes.data_ptr(), d, st)
        return data

    def decompose_quantize(self, data, bins, codes=None, workspace=None, stream=None):
        """Decompose `data` in place, then its int32 codes."""
        codes = self._codes(data, codes)
        d, w, wb, st = self._args(data, workspace, stream)
        mgard_decompose_quantize(self.handle, bins, d, codes.data_ptr(), w, wb, st)
        return codes

    def dequantize_recompose(self, codes, bins, data, workspace=None, stream=None):
        """The field rebuilt from codes (de-quantized into `data`, recomposed)."""
        self._codes(data, codes)
        d, w, wb, st = self._args(data, workspace, stream)
        mgard_dequantize_recompose(self.handle, bins, codes.data_ptr(), d, w, wb, st)
        return data

    def tune(self, level: int, param: int, value: int) -> None:
        """Launch-shape tuning of one level (see mgard_plan_tune)."""
        mgard_plan_tune(self.handle, level, param, value)

    def check(self, workspace=None, stream=None) -> None:
        """Raise MgardError (MGARD_ERR_TIMEOUT) if a grid-barrier wait of the
        last cooperative launch on this workspace ran out (mgard_plan_check)."""
        torch = _torch()
        ws = workspace if workspace is not None else self.workspace()
        s = stream if stream is not None else torch.cuda.current_stream(ws.device)
        mgard_plan_check(self.handle, ws.data_ptr(), s.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            mgard_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------- batches

def mgard_batch_create(plans, streams: int = 8) -> int:
    arr = (ctypes.c_void_p * len(plans))(*plans)
    out = ctypes.c_void_p()
    _check(LIB.mgard_batch_create(len(plans), arr, streams, ctypes.byref(out)), "mgard_batch_create")
    return out.value


def mgard_batch_destroy(batch: int) -> None:
    _check(LIB.mgard_batch_destroy(batch), "mgard_batch_destroy")


def mgard_batch_workspace_bytes(batch: int) -> int:
    return LIB.mgard_batch_workspace_bytes(batch)


def mgard_batch_decompose(batch: int, d_data, d_ws: int, ws_bytes: int, stream: int) -> None:
    arr = (ctypes.c_void_p * len(d_data))(*d_data)
    _check(LIB.mgard_batch_decompose(batch, arr, d_ws, ws_bytes, stream), "mgard_batch_decompose")


def mgard_batch_recompose(batch: int, d_data, d_ws: int, ws_bytes: int, stream: int) -> None:
    arr = (ctypes.c_void_p * len(d_data))(*d_data)
    _check(LIB.mgard_batch_recompose(batch, arr, d_ws, ws_bytes, stream), "mgard_batch_recompose")


def mgard_batch_tune(batch: int, param: int, value: int) -> None:
    _check(LIB.mgard_batch_tune(batch, param, value), "mgard_batch_tune")


def mgard_batch_get(batch: int, param: int) -> int:
    return int(LIB.mgard_batch_get(batch, param))


def mgard_batch_profile_read(batch: int, direction: int):
    """Per item kind (A, B, C, D, small, place): block-ms busy, block-ms
    waiting, items -- summed since the last read."""
    busy = (ctypes.c_double * 6)()
    wait = (ctypes.c_double * 6)()
    items = (ctypes.c_longlong * 6)()
    _check(LIB.mgard_batch_profile_read(batch, direction, busy, wait, items), "mgard_batch_profile_read")
    return list(busy), list(wait), list(items)


def mgard_batch_check(batch: int, stream: int) -> int:
    """The status code (0, or 5 = MGARD_ERR_TIMEOUT when a dependency wait of
    the persistent kernel ran out); does not raise."""
    return int(LIB.mgard_batch_check(batch, stream))


class Batch:
    """Independent fields (one Plan each) refactored by one CUDA-graph launch
    per call: the persistent kernel when every field fits it, else the graph
    of per-field launches.  The plans must outlive the batch."""

    # mgard_batch_get parameters
    GET = {"persistent": 0, "spin": 1, "stall": 2, "blocks_per_sm_req": 3, "eligible": 4, "grid": 5,
           "occupancy": 6, "items_dec": 7, "items_rec": 8, "model_us_dec": 9, "model_us_rec": 10,
           "smem": 11, "order": 12}

    def __init__(self, plans, streams: int = 8):
        self.plans = list(plans)
        self.handle = mgard_batch_create([p.handle for p in self.plans], streams)
        self.workspace_bytes = mgard_batch_workspace_bytes(self.handle)
        self._ws = None

    def workspace(self, device=None):
        torch = _torch()
        if self._ws is None:
            self._ws = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=device or "cuda")
        return self._ws

    def _args(self, fields, workspace, stream):
        torch = _torch()
        if len(fields) != len(self.plans):
            raise ValueError("one tensor per plan")
        for t, p in zip(fields, self.plans):
            if not t.is_cuda or not t.is_contiguous() or t.dtype != p.torch_dtype:
                raise ValueError("fields must be contiguous CUDA tensors of their plan's dtype")
        ws = workspace if workspace is not None else self.workspace(fields[0].device)
        s = stream if stream is not None else torch.cuda.current_stream(fields[0].device)
        return [t.data_ptr() for t in fields], ws.data_ptr(), ws.numel() * ws.element_size(), s.cuda_stream

    def decompose(self, fields, workspace=None, stream=None):
        mgard_batch_decompose(self.handle, *self._args(fields, workspace, stream))
        return fields

    def recompose(self, fields, workspace=None, stream=None):
        mgard_batch_recompose(self.handle, *self._args(fields, workspace, stream))
        return fields

    def tune(self, param: int, value: int) -> None:
        """0: 1 = persistent kernel, 0 = graph of per-field launches;
        1: dependency polls before a wait gives up; 2: test hook (1 = the
        first item waits for a count nothing reaches); 3: blocks per SM (0 =
        as many as fit); 4: 1 = record busy / waiting time per item kind;
        5: queue order (0 = fields by size, 1 = longest remaining path).
        The workspace size does not change."""
        mgard_batch_tune(self.handle, param, value)

    def get(self, name: str) -> int:
        return mgard_batch_get(self.handle, self.GET[name])

    KINDS = ("A", "B", "C", "D", "small", "place")

    def profile(self, direction: int) -> dict:
        """Block-ms busy / waiting and items per item kind since the last
        read (tuning param 4 = 1 records them)."""
        busy, wait, items = mgard_batch_profile_read(self.handle, direction)
        return {k: {"busy_ms": b, "wait_ms": w, "items": n} for k, b, w, n in zip(self.KINDS, busy, wait, items)}

    def check(self, stream=None) -> int:
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream()
        return mgard_batch_check(self.handle, s.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            mgard_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
