"""CPU oracle for multi-stixel estimation -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and this
package imports nothing of it.

The arithmetic lives in ``oracle.c`` (plain FP64 C, optionally OpenMP across
columns); this module compiles it with gcc on first use and wraps it with
ctypes.  Every function cites the part of the paper it follows in oracle.c.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import tempfile
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

OBJECT, GROUND, SKY, NONE = 0, 1, 2, 3
INF = float("inf")

OK, E_ARG, E_MEM, E_INFEASIBLE, E_CAPACITY = 0, 1, 2, 3, 4


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
        ("reduce_mode", C.c_int32), ("quantize", C.c_int32), ("pixel_grid", C.c_int32),
        ("sigma_gain", C.c_float), ("sigma_mid", C.c_float), ("sigma_width", C.c_float),
        ("ground_estimate", C.c_int32), ("global_map", C.c_int32),
    ]


class ColumnResult(C.Structure):
    _fields_ = [("cost", C.c_double), ("gap_abs", C.c_double), ("gap_rel", C.c_double),
                ("n", C.c_int32)]


STIXEL_DTYPE = np.dtype([("v_bottom", "<i4"), ("v_top", "<i4"), ("cls", "<i4"), ("f", "<i4"),
                         ("sum_q", "<i8"), ("disparity", "<f8")])
COLUMN_DTYPE = np.dtype([("cost", "<f8"), ("gap_abs", "<f8"), ("gap_rel", "<f8"), ("n", "<i4"),
                         ("_pad", "<i4")])

# The prior and sensor-model defaults of this implementation.  The paper takes
# its values from Pfeiffer's thesis, which is not available; these are our own
# choice for the five constraints it names (Sec. 3).
DEFAULTS: Dict[str, object] = dict(
    focal_px=700.0, baseline_m=0.3, camera_height_m=1.2, pitch_rad=0.0,
    horizon_row=40, stixel_width=5, dmax=64,
    p_out=0.05, sigma_ground=1.0, sigma_object=1.0, sigma_sky=1.0,
    prior_first=(1.0, 0.2, 5.0),                 # object, ground, sky
    prior_trans=((1.5, 1.0, 4.0),                # object above object / ground / sky
                 (1.5, INF, INF),                # ground above ...
                 (0.5, 0.5, INF)),               # sky above ...
    cost_new_stixel=3.0,
    cost_gravity=2.0, eps_gravity=1.0, cost_diving=10.0, eps_diving=1.0,
    cost_order=2.0, eps_order=0.0,
    reduce_mode=0, quantize=1, pixel_grid=0,
    sigma_gain=0.0, sigma_mid=32.0, sigma_width=8.0, ground_estimate=0, global_map=0,
)


def _build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc, OpenMP, no FP contraction) and return the library path."""
    return _build(force)


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build())
        P = C.POINTER
        L.or_reduce.argtypes = [P(C.c_float), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P(C.c_int16)]
        L.or_ground_estimate.argtypes = [P(C.c_int16), C.c_int, C.c_int, C.c_int, P(C.c_int32)]
        L.or_pixel_cost.argtypes = [P(Params), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P(C.c_double)]
        L.or_gaussian_branch.argtypes = [P(Params), C.c_int, C.c_double, C.c_double, P(C.c_double)]
        L.or_model_constants.argtypes = [P(Params), C.c_int, P(C.c_double), P(C.c_double), P(C.c_double),
                                         P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double),
                                         P(C.c_double)]
        L.or_prefix.argtypes = [P(Params), P(C.c_int16), C.c_int, P(C.c_int64), P(C.c_double),
                                P(C.c_double), P(C.c_double)]
        L.or_column.argtypes = [P(Params), P(C.c_int16), C.c_int, C.c_int, C.c_void_p, P(ColumnResult)]
        L.or_frame.argtypes = [P(Params), P(C.c_float), C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                               P(C.c_int16), C.c_int]
        L.or_eval_segmentation.argtypes = [P(Params), P(C.c_int16), C.c_int, C.c_void_p, C.c_int,
                                           P(C.c_double)]
        L.or_eval_frame.argtypes = [P(Params), P(C.c_int16), C.c_int, C.c_int, C.c_void_p, C.c_int,
                                    P(C.c_int32), P(C.c_double)]
        L.or_brute_force.argtypes = [P(Params), P(C.c_int16), C.c_int, P(C.c_double), P(C.c_int64),
                                     C.c_void_p, P(C.c_int32)]
        L.or_max_threads.argtypes = []
        _lib = L
    return _lib


def make_params(camera=None, **overrides) -> Params:
    """Params from DEFAULTS, then the camera's fields (a scenes.Camera), then overrides."""
    d = dict(DEFAULTS)
    if camera is not None:
        d.update(focal_px=camera.focal_px, baseline_m=camera.baseline_m,
                 camera_height_m=camera.camera_height_m, pitch_rad=camera.pitch_rad,
                 horizon_row=camera.horizon_row, stixel_width=camera.stixel_width, dmax=camera.dmax)
    d.update(overrides)
    p = Params()
    for name, _ in Params._fields_:
        v = d[name]
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


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _check(rc: int, what: str, allowed=(OK,)):
    if rc not in allowed:
        raise RuntimeError(f"oracle {what} failed with status {rc}")
    return rc


def reduce(disp: np.ndarray, s: int, dmax: int, mode: int = 0, pixel_grid: int = 0) -> np.ndarray:
    """Column reduction + transpose (Sec. 5.1) -> (ncols, H) int16 Q4 codes, row 0 = bottom;
    with pixel_grid the codes are rounded to whole pixels (multiples of 16, halves up)."""
    disp = np.ascontiguousarray(disp, dtype=np.float32)
    H, W = disp.shape
    q = np.zeros((W // s, H), dtype=np.int16)
    _check(lib().or_reduce(_ptr(disp, C.c_float), H, W, s, dmax, mode, pixel_grid, _ptr(q, C.c_int16)), "reduce")
    return q


def ground_estimate(q: np.ndarray, dmax: int):
    """v-disparity ground line of reduced codes q (ncols, H), bottom-up: (k, horizon row, votes),
    slope k / 256 px of disparity per image row."""
    q = np.ascontiguousarray(q, dtype=np.int16)
    out = np.zeros(3, np.int32)
    _check(lib().or_ground_estimate(_ptr(q, C.c_int16), q.shape[0], q.shape[1], dmax, _ptr(out, C.c_int32)),
           "ground_estimate")
    return int(out[0]), int(out[1]), int(out[2])


def pixel_cost(params: Params, H: int, cls: int, v: int, q: int, f: int = 0) -> float:
    out = C.c_double()
    _check(lib().or_pixel_cost(C.byref(params), H, cls, v, q, f, C.byref(out)), "pixel_cost")
    return out.value


def gaussian_branch(params: Params, cls: int, f: float, d: float) -> float:
    out = C.c_double()
    _check(lib().or_gaussian_branch(C.byref(params), cls, f, d, C.byref(out)), "gaussian_branch")
    return out.value


def model_constants(params: Params, H: int) -> Dict[str, np.ndarray]:
    F = params.dmax + 1
    c_out, k_sky = C.c_double(), C.c_double()
    k_obj = np.zeros(F); fg = np.zeros(H); kg = np.zeros(H)
    first = np.zeros(3); trans = np.zeros(9); pens = np.zeros(3)
    d = C.POINTER(C.c_double)
    _check(lib().or_model_constants(C.byref(params), H, C.byref(c_out), _ptr(k_obj, C.c_double),
                                    C.byref(k_sky), _ptr(fg, C.c_double), _ptr(kg, C.c_double),
                                    _ptr(first, C.c_double), _ptr(trans, C.c_double),
                                    _ptr(pens, C.c_double)), "model_constants")
    return dict(c_out=c_out.value, k_obj=k_obj, k_sky=k_sky.value, fg=fg, k_ground=kg,
                first=first, trans=trans.reshape(3, 3), pens=pens)


def prefix(params: Params, q_col: np.ndarray):
    """Prefix LUTs of one column (Sec. 3.4): pd (int64), pg, ps (H+1), po ((dmax+1) x (H+1))."""
    q_col = np.ascontiguousarray(q_col, dtype=np.int16)
    H = q_col.shape[0]
    pd = np.zeros(H + 1, np.int64); pg = np.zeros(H + 1); ps = np.zeros(H + 1)
    po = np.zeros((params.dmax + 1, H + 1))
    _check(lib().or_prefix(C.byref(params), _ptr(q_col, C.c_int16), H, _ptr(pd, C.c_int64),
                           _ptr(pg, C.c_double), _ptr(ps, C.c_double), _ptr(po, C.c_double)), "prefix")
    return pd, pg, ps, po


@dataclass
class ColumnOut:
    stixels: np.ndarray      # STIXEL_DTYPE, bottom -> top
    cost: float
    gap_abs: float
    gap_rel: float
    n: int                   # stixels on the optimal path (may exceed len(stixels) on overflow)


def column(params: Params, q_col: np.ndarray, cap: int = 4096) -> ColumnOut:
    """The DP of Eq. 5-6 plus backtracking for one column of Q4 codes (bottom-up)."""
    q_col = np.ascontiguousarray(q_col, dtype=np.int16)
    H = q_col.shape[0]
    out = np.zeros(max(cap, 1), STIXEL_DTYPE)
    res = ColumnResult()
    _check(lib().or_column(C.byref(params), _ptr(q_col, C.c_int16), H, cap, out.ctypes.data,
                           C.byref(res)), "column", (OK, E_CAPACITY))
    return ColumnOut(out[:min(res.n, cap)].copy(), res.cost, res.gap_abs, res.gap_rel, res.n)


@dataclass
class FrameOut:
    q: np.ndarray            # (ncols, H) int16
    stixels: np.ndarray      # (ncols, cap) STIXEL_DTYPE
    counts: np.ndarray       # (ncols,) stixels on each column's path
    cost: np.ndarray         # (ncols,) float64
    gap_abs: np.ndarray
    gap_rel: np.ndarray
    status: int


def frame(params: Params, disp: np.ndarray, cap: int = 256, nthreads: int = 0) -> FrameOut:
    """Reduction then the DP on every column of a frame (OpenMP across columns)."""
    disp = np.ascontiguousarray(disp, dtype=np.float32)
    H, W = disp.shape
    ncols = W // params.stixel_width
    st = np.zeros((ncols, max(cap, 1)), STIXEL_DTYPE)
    res = np.zeros(ncols, COLUMN_DTYPE)
    q = np.zeros((ncols, H), np.int16)
    rc = lib().or_frame(C.byref(params), _ptr(disp, C.c_float), H, W, cap, st.ctypes.data,
                        res.ctypes.data, _ptr(q, C.c_int16), nthreads)
    _check(rc, "frame", (OK, E_CAPACITY))
    return FrameOut(q, st[:, :cap], res["n"].copy(), res["cost"].copy(), res["gap_abs"].copy(),
                    res["gap_rel"].copy(), rc)


def eval_segmentation(params: Params, q_col: np.ndarray, stixels: np.ndarray) -> float:
    """Direct re-evaluation (per-pixel sums + pairwise priors) of a bottom -> top stixel list."""
    q_col = np.ascontiguousarray(q_col, dtype=np.int16)
    st = np.ascontiguousarray(stixels, dtype=STIXEL_DTYPE)
    out = C.c_double()
    _check(lib().or_eval_segmentation(C.byref(params), _ptr(q_col, C.c_int16), q_col.shape[0],
                                      st.ctypes.data, len(st), C.byref(out)), "eval_segmentation")
    return out.value


def eval_frame(params: Params, q: np.ndarray, stixels: np.ndarray, counts: np.ndarray) -> np.ndarray:
    """Direct re-evaluation of one segmentation per column (stixels: ncols x cap,
    counts[c] used) under the frame's model (with ground_estimate, the line
    estimated from q); NaN where a list is incomplete (counts > cap)."""
    q = np.ascontiguousarray(q, dtype=np.int16)
    st = np.ascontiguousarray(stixels, dtype=STIXEL_DTYPE)
    cnt = np.ascontiguousarray(counts, dtype=np.int32)
    ncols, H = q.shape
    out = np.zeros(ncols)
    _check(lib().or_eval_frame(C.byref(params), _ptr(q, C.c_int16), ncols, H, st.ctypes.data, st.shape[1],
                               _ptr(cnt, C.c_int32), _ptr(out, C.c_double)), "eval_frame")
    return out


def brute_force(params: Params, q_col: np.ndarray):
    """Exhaustive minimum over all segmentations (H <= 14): (cost, count, first argmin)."""
    q_col = np.ascontiguousarray(q_col, dtype=np.int16)
    H = q_col.shape[0]
    best = C.c_double(); cnt = C.c_int64(); n = C.c_int32()
    out = np.zeros(H, STIXEL_DTYPE)
    _check(lib().or_brute_force(C.byref(params), _ptr(q_col, C.c_int16), H, C.byref(best), C.byref(cnt),
                                out.ctypes.data, C.byref(n)), "brute_force")
    return best.value, cnt.value, out[:n.value].copy()


def max_threads() -> int:
    return int(lib().or_max_threads())
