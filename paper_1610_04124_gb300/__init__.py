"""Python binding of the GB300 stixel library (include/stixels.h).

Argument marshalling only: every step of the stixel pipeline runs in the CUDA
kernels of libstixels.so.  PyTorch provides device memory and streams.  There
is no CPU fallback -- importing this package without the built library raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Dict, Optional

import numpy as np

from . import build as _build_mod

__all__ = ["Params", "Stixels", "Batch", "Server", "STIXEL_DTYPE", "StixelsError", "lib", "default_params",
           "model_tables", "lut_pitch", "OBJECT", "GROUND", "SKY"]

OBJECT, GROUND, SKY = 0, 1, 2
OK, E_INVALID_ARG, E_OOM, E_CUDA, E_CAPACITY, E_NOT_READY, E_TIMEOUT, E_REJECTED, E_DEVICE_FAULT = range(9)
ERR_CAPACITY, ERR_INFEASIBLE, ERR_TIMEOUT = 1, 2, 4
MAX_HEIGHT = 2048
NOALLOC_SCRATCH_BYTES = 48 << 20
N_SCALARS = 18
UNITS_PER_COST = 16384

STIXEL_DTYPE = np.dtype([("row_top", "<i2"), ("row_bottom", "<i2"), ("cls", "u1"), ("flags", "u1"),
                         ("reserved", "<i2"), ("disparity", "<f4")])
assert STIXEL_DTYPE.itemsize == 12


class Params(C.Structure):
    _fields_ = [
        ("focal_px", C.c_float), ("baseline_m", C.c_float), ("camera_height_m", C.c_float),
        ("pitch_rad", C.c_float),
        ("horizon_row", C.c_int32), ("stixel_width", C.c_int32), ("dmax", C.c_int32),
        ("p_out", C.c_float), ("sigma_ground", C.c_float), ("sigma_object", C.c_float),
        ("sigma_sky", C.c_float),
        ("prior_first", C.c_float * 3),
        ("prior_trans", (C.c_float * 3) * 3),
        ("cost_new_stixel", C.c_float),
        ("cost_gravity", C.c_float), ("eps_gravity", C.c_float),
        ("cost_diving", C.c_float), ("eps_diving", C.c_float),
        ("cost_order", C.c_float), ("eps_order", C.c_float),
        ("reduce_mode", C.c_int32), ("max_stixels_per_col", C.c_int32), ("pixel_grid", C.c_int32),
        ("sigma_gain", C.c_float), ("sigma_mid", C.c_float), ("sigma_width", C.c_float),
        ("ground_estimate", C.c_int32), ("global_map", C.c_int32),
    ]

    def to_dict(self) -> Dict[str, object]:
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            if name == "prior_first":
                v = tuple(v[i] for i in range(3))
            elif name == "prior_trans":
                v = tuple(tuple(v[i][j] for j in range(3)) for i in range(3))
            d[name] = v
        return d


class Output(C.Structure):
    _fields_ = [("stixels", C.c_void_p), ("counts", C.c_void_p), ("column_cost", C.c_void_p),
                ("column_cost_fixed", C.c_void_p), ("ncols", C.c_int32), ("capacity", C.c_int32)]


class FrameDesc(C.Structure):
    _fields_ = [("camera", C.c_void_p), ("H", C.c_int32), ("W", C.c_int32)]


class BatchConfig(C.Structure):
    _fields_ = [("dp_warps", C.c_int32), ("dp_ctas_per_sm", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("admitted", C.c_uint64), ("rejected", C.c_uint64),
                ("completed", C.c_uint64), ("iterations", C.c_uint64), ("frames_in_iterations", C.c_uint64),
                ("bytes_in_use", C.c_uint64), ("bytes_budget", C.c_uint64),
                ("slots_in_use", C.c_int32), ("max_slots", C.c_int32)]


class StixelsError(RuntimeError):
    def __init__(self, status: int, what: str):
        detail = ""
        if status in (E_CUDA, E_OOM):
            detail = f" [{lib().stixels_last_cuda_error().decode()}]"
        super().__init__(f"{what}: {lib().stixels_status_string(status).decode()} (status {status}){detail}")
        self.status = status


_lib = None


def lib():
    """The loaded libstixels.so (built in-tree on first use if missing or stale)."""
    global _lib
    if _lib is None:
        path = _build_mod.build()
        if not os.path.exists(path):
            raise RuntimeError("libstixels.so is missing; the CUDA library must be built (nvcc, sm_103a)")
        L = C.CDLL(path)
        P, V, I = C.POINTER, C.c_void_p, C.c_int
        L.stixels_params_default.argtypes = [P(Params)]
        L.stixels_create.argtypes = [P(Params), P(V)]
        L.stixels_destroy.argtypes = [V]
        L.stixels_output_shape.argtypes = [V, I, I, P(I), P(I)]
        L.stixels_reserve.argtypes = [V, I, I]
        L.stixels_compute.argtypes = [V, V, I, I, V, P(Output)]
        L.stixels_compute_host.argtypes = [V, V, I, I, V, V, V]
        L.stixels_get_error.argtypes = [V, V, P(C.c_uint32)]
        L.stixels_selftest_wait.argtypes = [V, I, V, P(C.c_uint32)]
        L.stixels_lut_pitch.argtypes = [I]
        L.stixels_reduce.argtypes = [V, V, I, I, V, V]
        L.stixels_build_luts.argtypes = [V, V, I, I, V, V, V, V, V]
        L.stixels_estimate_ground.argtypes = [V, V, I, I, V, V]
        L.stixels_solve.argtypes = [V, V, V, V, V, I, I, V, P(Output)]
        L.stixels_model_tables.argtypes = [P(Params), I, V, V, V, V, V, V, V]
        L.stixels_compute_noalloc.argtypes = [V, V, I, I, V, P(Output)]
        L.stixels_batch_create.argtypes = [P(FrameDesc), I, P(V)]
        L.stixels_batch_input.argtypes = [V, I, P(V)]
        L.stixels_batch_output.argtypes = [V, I, P(Output)]
        L.stixels_batch_set_input.argtypes = [V, I, V, V]
        L.stixels_batch_get_output.argtypes = [V, I, V, V, V, V, V]
        L.stixels_batch_launch.argtypes = [V, V]
        L.stixels_batch_set_config.argtypes = [V, P(BatchConfig)]
        L.stixels_batch_get_config.argtypes = [V, P(BatchConfig)]
        L.stixels_batch_tune.argtypes = [V, V, C.c_char_p, P(BatchConfig)]
        L.stixels_batch_destroy.argtypes = [V]
        L.stixels_server_create.argtypes = [C.c_size_t, I, P(V)]
        L.stixels_submit.argtypes = [V, V, V, I, I, P(C.c_uint64)]
        L.stixels_poll.argtypes = [V, C.c_uint64, P(Output), I]
        L.stixels_server_stats.argtypes = [V, P(ServerStats)]
        L.stixels_server_destroy.argtypes = [V]
        L.stixels_status_string.argtypes = [I]
        L.stixels_status_string.restype = C.c_char_p
        L.stixels_last_cuda_error.argtypes = []
        L.stixels_last_cuda_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc: int, what: str, allowed=(OK,)) -> int:
    if rc not in allowed:
        raise StixelsError(rc, what)
    return rc


def default_params(camera=None, **overrides) -> Params:
    """stixels_params_default(), then the fields of a scenes.Camera-like object, then overrides."""
    p = Params()
    _check(lib().stixels_params_default(C.byref(p)), "params_default")
    if camera is not None:
        for name in ("focal_px", "baseline_m", "camera_height_m", "pitch_rad", "horizon_row",
                     "stixel_width", "dmax"):
            setattr(p, name, getattr(camera, name))
    for name, v in overrides.items():
        if name == "prior_first":
            for i in range(3):
                p.prior_first[i] = float(v[i])
        elif name == "prior_trans":
            for i in range(3):
                for j in range(3):
                    p.prior_trans[i][j] = float(v[i][j])
        else:
            setattr(p, name, v)
    return p


def lut_pitch(H: int) -> int:
    return int(lib().stixels_lut_pitch(H))


def model_tables(params: Params, H: int) -> Dict[str, np.ndarray]:
    """Host-side fixed-point tables the library builds for `params` (no CUDA call)."""
    F, E = params.dmax + 1, 16 * params.dmax + 1
    n = max(H, 1)
    t = dict(k_obj=np.zeros(F, np.int32), g_obj=np.zeros(E, np.int32), g_sky=np.zeros(E, np.int32),
             fg=np.zeros(n, np.float64), k_ground=np.zeros(n, np.int32), thr=np.zeros(n, np.int32),
             scalars=np.zeros(N_SCALARS, np.int32))
    _check(lib().stixels_model_tables(C.byref(params), H, *(t[k].ctypes.data for k in
                                                             ("k_obj", "g_obj", "g_sky", "fg", "k_ground", "thr",
                                                              "scalars"))), "model_tables")
    for k in ("fg", "k_ground", "thr"):
        t[k] = t[k][:H]
    return t


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Stixels:
    """One handle (camera / parameter set) of the stixel library."""

    def __init__(self, params: Optional[Params] = None, **overrides):
        self.params = params if params is not None else default_params(**overrides)
        h = C.c_void_p()
        _check(lib().stixels_create(C.byref(self.params), C.byref(h)), "stixels_create")
        self._h = h

    def close(self):
        self.__dict__.pop("_host_ptrs", None)
        if getattr(self, "_h", None):
            lib().stixels_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def output_shape(self, H: int, W: int):
        # fixed for a handle and frame size: asked of the library once
        cache = self.__dict__.setdefault("_shapes", {})
        shape = cache.get((H, W))
        if shape is None:
            n, c = C.c_int(), C.c_int()
            _check(lib().stixels_output_shape(self._h, H, W, C.byref(n), C.byref(c)), "output_shape")
            shape = cache[(H, W)] = (n.value, c.value)
        return shape

    def reserve(self, H: int, W: int):
        _check(lib().stixels_reserve(self._h, H, W), "reserve")

    def alloc_output(self, H: int, W: int, device=None):
        """Device output buffers (torch tensors) for an H x W frame."""
        import torch
        ncols, cap = self.output_shape(H, W)
        dev = device or torch.device("cuda", torch.cuda.current_device())
        return dict(stixels=torch.zeros(max(ncols * cap, 1) * 3, dtype=torch.int32, device=dev),
                    counts=torch.zeros(max(ncols, 1), dtype=torch.int32, device=dev),
                    cost=torch.zeros(max(ncols, 1), dtype=torch.float32, device=dev),
                    cost_fixed=torch.zeros(max(ncols, 1), dtype=torch.int32, device=dev),
                    ncols=ncols, capacity=cap)

    @staticmethod
    def _out_struct(out) -> Output:
        return Output(_ptr(out["stixels"]), _ptr(out["counts"]), _ptr(out.get("cost")),
                      _ptr(out.get("cost_fixed")), out["ncols"], out["capacity"])

    def compute(self, disparity, out=None, stream=None):
        """Full pipeline on a CUDA float32 (H, W) tensor; returns the output dict (async on stream)."""
        assert disparity.is_cuda and disparity.dtype.is_floating_point and disparity.dim() == 2
        disparity = disparity.contiguous()
        H, W = disparity.shape
        if out is None:
            out = self.alloc_output(H, W, disparity.device)
        o = self._out_struct(out)
        _check(lib().stixels_compute(self._h, _ptr(disparity), H, W, _stream_ptr(stream), C.byref(o)),
               "stixels_compute")
        return out

    def alloc_host_output(self, H: int, W: int, pinned: bool = False):
        """Host output arrays (stixels, counts, cost) for compute_host, optionally page-locked."""
        ncols, cap = self.output_shape(H, W)
        if pinned:
            import torch
            st = torch.zeros(max(ncols * cap, 1) * 3, dtype=torch.int32, pin_memory=True).numpy().view(STIXEL_DTYPE)
            counts = torch.zeros(max(ncols, 1), dtype=torch.int32, pin_memory=True).numpy()
            cost = torch.zeros(max(ncols, 1), dtype=torch.float32, pin_memory=True).numpy()
        else:
            st = np.zeros(max(ncols * cap, 1), STIXEL_DTYPE)
            counts = np.zeros(max(ncols, 1), np.int32)
            cost = np.zeros(max(ncols, 1), np.float32)
        return st, counts, cost

    def compute_noalloc(self, disparity, out, stream=None):
        """stixels_compute_noalloc: same as compute(), intermediates in the library's
        fixed scratch array (no device allocation; call reserve(H, W) first)."""
        H, W = disparity.shape
        o = self._out_struct(out)
        _check(lib().stixels_compute_noalloc(self._h, _ptr(disparity), H, W, _stream_ptr(stream), C.byref(o)),
               "stixels_compute_noalloc")
        return out

    def compute_host(self, disparity: np.ndarray, out=None):
        """Host -> host pipeline (synchronous).  Returns (stixels, counts, cost, status)."""
        d = disparity if (isinstance(disparity, np.ndarray) and disparity.dtype == np.float32
                          and disparity.flags.c_contiguous) else np.ascontiguousarray(disparity, dtype=np.float32)
        H, W = d.shape
        ncols, cap = self.output_shape(H, W)
        st, counts, cost = out if out is not None else self.alloc_host_output(H, W)
        # the buffers' addresses, kept with references to the arrays they
        # belong to (so those arrays stay alive and the addresses valid) for
        # the next call with the same arrays
        last = self.__dict__.get("_host_ptrs")
        if last is not None and last[0] is d:
            dp = last[1]
        else:
            dp = d.ctypes.data
        if last is not None and last[2] is out and out is not None:
            sp, cp, kp = last[3]
        else:
            sp, cp, kp = st.ctypes.data, counts.ctypes.data, cost.ctypes.data
        self._host_ptrs = (d, dp, out, (sp, cp, kp))
        rc = lib().stixels_compute_host(self._h, dp, H, W, sp, cp, kp)
        _check(rc, "stixels_compute_host", (OK, E_CAPACITY))
        return st[:ncols * cap].reshape(ncols, cap), counts[:ncols], cost[:ncols], rc

    def get_error(self, stream=None) -> int:
        v = C.c_uint32()
        _check(lib().stixels_get_error(self._h, _stream_ptr(stream), C.byref(v)), "get_error")
        return v.value

    def selftest_wait(self, polls: int = 1000, stream=None) -> int:
        """Run the kernels' bounded wait on a flag nothing sets; returns the
        error word (ERR_TIMEOUT when the wait gave up as it should)."""
        v = C.c_uint32()
        _check(lib().stixels_selftest_wait(self._h, int(polls), _stream_ptr(stream), C.byref(v)),
               "stixels_selftest_wait")
        return v.value

    # ---- stages ----
    def reduce(self, disparity, q=None, stream=None):
        import torch
        H, W = disparity.shape
        ncols = W // self.params.stixel_width
        if q is None:
            q = torch.zeros((max(ncols, 1), max(H, 1)), dtype=torch.int16, device=disparity.device)
        _check(lib().stixels_reduce(self._h, _ptr(disparity), H, W, _stream_ptr(stream), _ptr(q)), "stixels_reduce")
        return q

    def estimate_ground(self, q, H: int, ncols: int, stream=None):
        """stixels_estimate_ground on reduced codes q: (k, horizon row, votes); slope k / 256 px per row."""
        import torch
        line = torch.zeros(3, dtype=torch.int32, device=q.device)
        _check(lib().stixels_estimate_ground(self._h, _ptr(q), H, ncols, _stream_ptr(stream), _ptr(line)),
               "stixels_estimate_ground")
        k, h, votes = (int(x) for x in line.cpu())
        return k, h, votes

    def build_luts(self, q, H: int, ncols: int, stream=None):
        import torch
        P, F = lut_pitch(H), self.params.dmax + 1
        dev = q.device
        pd = torch.zeros((max(ncols, 1), P), dtype=torch.int32, device=dev)
        pg = torch.zeros_like(pd)
        ps = torch.zeros_like(pd)
        po = torch.zeros((max(ncols, 1), F, P), dtype=torch.int32, device=dev)
        _check(lib().stixels_build_luts(self._h, _ptr(q), H, ncols, _stream_ptr(stream), _ptr(pd), _ptr(pg),
                                        _ptr(ps), _ptr(po)), "stixels_build_luts")
        return pd, pg, ps, po

    def solve(self, pd, pg, ps, po, H: int, ncols: int, out=None, stream=None):
        if out is None:
            out = self.alloc_output(H, ncols * self.params.stixel_width, pd.device)
        o = self._out_struct(out)
        _check(lib().stixels_solve(self._h, _ptr(pd), _ptr(pg), _ptr(ps), _ptr(po), H, ncols, _stream_ptr(stream),
                                   C.byref(o)), "stixels_solve")
        return out

    @staticmethod
    def to_host(out):
        """Copy an output dict to numpy: (stixels[ncols, cap], counts, cost, cost_fixed)."""
        ncols, cap = out["ncols"], out["capacity"]
        st = out["stixels"].cpu().numpy().view(STIXEL_DTYPE)[:ncols * cap].reshape(ncols, cap)
        return (st, out["counts"].cpu().numpy()[:ncols], out["cost"].cpu().numpy()[:ncols],
                out["cost_fixed"].cpu().numpy()[:ncols])


class Batch:
    """A fixed set of frames (camera handle, H, W) run by one graph-captured launch."""

    def __init__(self, frames):
        self.frames = [(h, int(H), int(W)) for h, H, W in frames]
        arr = (FrameDesc * len(self.frames))(*[FrameDesc(h.handle, H, W) for h, H, W in self.frames])
        b = C.c_void_p()
        _check(lib().stixels_batch_create(arr, len(self.frames), C.byref(b)), "stixels_batch_create")
        self._b = b

    def close(self):
        if getattr(self, "_b", None):
            lib().stixels_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_input(self, i, src, stream=None):
        """src: a CUDA tensor or a contiguous float32 numpy array (H, W)."""
        ptr = src.data_ptr() if hasattr(src, "data_ptr") else np.ascontiguousarray(src, np.float32).ctypes.data
        _check(lib().stixels_batch_set_input(self._b, i, ptr, _stream_ptr(stream)), "stixels_batch_set_input")

    def launch(self, stream=None):
        _check(lib().stixels_batch_launch(self._b, _stream_ptr(stream)), "stixels_batch_launch")

    def output(self, i, stream=None):
        """Frame i's results copied to host numpy: (stixels[ncols, cap], counts, cost, cost_fixed)."""
        o = Output()
        _check(lib().stixels_batch_output(self._b, i, C.byref(o)), "stixels_batch_output")
        st = np.zeros(max(o.ncols * o.capacity, 1), STIXEL_DTYPE)
        cnt = np.zeros(max(o.ncols, 1), np.int32)
        cost = np.zeros(max(o.ncols, 1), np.float32)
        fix = np.zeros(max(o.ncols, 1), np.int32)
        _check(lib().stixels_batch_get_output(self._b, i, st.ctypes.data, cnt.ctypes.data, cost.ctypes.data,
                                              fix.ctypes.data, _stream_ptr(stream)), "stixels_batch_get_output")
        import torch
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        n = o.ncols
        return st[:n * o.capacity].reshape(n, o.capacity), cnt[:n], cost[:n], fix[:n]

    @property
    def config(self):
        c = BatchConfig()
        _check(lib().stixels_batch_get_config(self._b, C.byref(c)), "stixels_batch_get_config")
        return (c.dp_warps, c.dp_ctas_per_sm)

    def set_config(self, dp_warps, dp_ctas_per_sm):
        c = BatchConfig(dp_warps, dp_ctas_per_sm)
        _check(lib().stixels_batch_set_config(self._b, C.byref(c)), "stixels_batch_set_config")

    def tune(self, cache_path=None, stream=None):
        c = BatchConfig()
        path = cache_path.encode() if cache_path else None
        _check(lib().stixels_batch_tune(self._b, _stream_ptr(stream), path, C.byref(c)), "stixels_batch_tune")
        return (c.dp_warps, c.dp_ctas_per_sm)


class Server:
    """Continuous-batching server over many camera handles (stixels_server_*)."""

    def __init__(self, mem_budget_bytes: int, max_slots: int = 256):
        s = C.c_void_p()
        _check(lib().stixels_server_create(int(mem_budget_bytes), int(max_slots), C.byref(s)),
               "stixels_server_create")
        self._s = s
        self._shape = {}                         # ticket -> (ncols, capacity)

    def close(self):
        if getattr(self, "_s", None):
            lib().stixels_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, camera: Stixels, disparity) -> Optional[int]:
        """Admit one frame (CUDA tensor or float32 numpy array); the ticket, or None if rejected."""
        if hasattr(disparity, "data_ptr"):
            assert disparity.dtype.is_floating_point and disparity.element_size() == 4 and disparity.is_contiguous()
            ptr, (H, W) = disparity.data_ptr(), disparity.shape
        else:
            assert isinstance(disparity, np.ndarray) and disparity.dtype == np.float32 and \
                disparity.flags.c_contiguous
            ptr, (H, W) = disparity.ctypes.data, disparity.shape
        t = C.c_uint64()
        rc = _check(lib().stixels_submit(self._s, camera.handle, ptr, H, W, C.byref(t)), "stixels_submit",
                    (OK, E_REJECTED))
        if rc != OK:
            return None
        self._shape[t.value] = camera.output_shape(H, W)
        return t.value

    def poll(self, ticket: int, out, timeout_us: int = 0) -> int:
        """Wait up to timeout_us for the ticket; fills `out` and returns OK / E_CAPACITY, or
        E_NOT_READY / E_TIMEOUT while the frame is not done.  `out` is a
        (stixels, counts, cost) host tuple as Stixels.alloc_host_output, or a device dict
        as Stixels.alloc_output."""
        ncols, cap = self._shape.get(int(ticket), (0, 0))
        if isinstance(out, dict):
            o = Stixels._out_struct(out)
        else:
            st, counts, cost = out
            o = Output(st.ctypes.data, counts.ctypes.data, cost.ctypes.data, 0, ncols, cap)
        rc = _check(lib().stixels_poll(self._s, int(ticket), C.byref(o), int(timeout_us)), "stixels_poll",
                    (OK, E_CAPACITY, E_NOT_READY, E_TIMEOUT))
        if rc in (OK, E_CAPACITY):
            self._shape.pop(int(ticket), None)
        return rc

    def stats(self) -> Dict[str, int]:
        st = ServerStats()
        _check(lib().stixels_server_stats(self._s, C.byref(st)), "stixels_server_stats")
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}
