"""Seeded synthetic road scenes (FP32 disparity maps) for tests and benchmarks.

This module only draws inputs: a flat ground plane below the horizon, sky
(disparity 0) above it, rectangular fronto-parallel obstacles standing on the
ground, and a sensor-noise recipe (Gaussian jitter, uniform outliers, invalid
zeros).  It holds none of the stixel method's arithmetic (no cost model, no
reduction, no dynamic program); both the CUDA library and the CPU oracle take
its output as plain input.

Image row 0 is the top row.  The ground disparity at image row r is
alpha * (r - horizon) with alpha = baseline * cos(pitch) / camera_height, the
flat-ground geometry the paper assumes known for every image (Sec. 3, the
ground model of Sec. 3.1).

The five workloads are the ones the benchmark and the parity tests use; none
comes from a public dataset (the paper's SYNTHIA and labelled Daimler images
are not used), they only mimic their sizes and structure.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Camera", "Scene", "make_scene", "config_frames", "camera_for",
    "CONFIG1", "CONFIG2", "CONFIG3", "CONFIG4", "serving_cameras",
]


@dataclass(frozen=True)
class Camera:
    """Camera and stixel-model settings for one stream of frames."""
    width: int
    height: int
    stixel_width: int = 5
    dmax: int = 64
    focal_px: float = 700.0
    baseline_m: float = 0.3
    camera_height_m: float = 1.2
    pitch_rad: float = 0.0
    horizon_row: int = 40

    @property
    def alpha(self) -> float:
        return self.baseline_m * math.cos(self.pitch_rad) / self.camera_height_m

    @property
    def ncols(self) -> int:
        return self.width // self.stixel_width


@dataclass
class Scene:
    disparity: np.ndarray            # (H, W) float32, row 0 = top
    camera: Camera
    labels: np.ndarray               # (H, W) uint8: 0 object, 1 ground, 2 sky (noise-free truth)
    obj_disp: np.ndarray             # (H, W) float32 disparity of the painted obstacle, or -1
    obstacles: List[Tuple[float, int, int, int, int]] = field(default_factory=list)
    # (disparity, first column, span in columns, top row, bottom row)


def make_scene(cam: Camera, seed: int, *, n_obstacles: Tuple[int, int] = (3, 6),
               disp_range: Tuple[float, float] = (5.0, 60.0), integer_disp: bool = False,
               span_cols: Tuple[int, int] = (2, 40),
               height_frac: Tuple[float, float] = (1.0 / 8.0, 1.0 / 2.0),
               min_height: int = 1,
               noise_sigma: float = 1.0, p_outlier: float = 0.05, p_invalid: float = 0.02) -> Scene:
    """Draw one frame.  Same (cam, seed, keyword arguments) -> same bytes."""
    rng = np.random.default_rng(seed)
    H, W, s = cam.height, cam.width, cam.stixel_width
    C = max(1, W // s)
    alpha = cam.alpha
    rows = np.arange(H, dtype=np.float64)
    ground = np.where(rows > cam.horizon_row, alpha * (rows - cam.horizon_row), 0.0)
    D = np.repeat(ground[:, None], W, axis=1)
    labels = np.where(rows[:, None] > cam.horizon_row, 1, 2).astype(np.uint8).repeat(W, axis=1)
    obj = np.full((H, W), -1.0, dtype=np.float32)

    k = int(rng.integers(n_obstacles[0], n_obstacles[1] + 1))
    obstacles = []
    for _ in range(k):
        if integer_disp:
            d = float(rng.integers(int(disp_range[0]), int(disp_range[1]) + 1))
        else:
            d = float(rng.uniform(disp_range[0], disp_range[1]))
        span = int(rng.integers(span_cols[0], min(span_cols[1], C) + 1)) if C >= span_cols[0] else C
        c0 = int(rng.integers(0, C - span + 1))
        bottom = min(H - 1, int(round(cam.horizon_row + d / alpha))) if alpha > 0 else H - 1
        lo = max(min_height, int(math.ceil(H * height_frac[0])))
        hi = max(lo, int(math.floor(H * height_frac[1])))
        height = int(rng.integers(lo, hi + 1))
        top = max(0, bottom - height + 1)
        obstacles.append((d, c0, span, top, bottom))
    # paint far to near so that the nearer obstacle (larger disparity) occludes
    for d, c0, span, top, bottom in sorted(obstacles, key=lambda o: o[0]):
        x0, x1 = c0 * s, min(W, (c0 + span) * s)
        D[top:bottom + 1, x0:x1] = d
        labels[top:bottom + 1, x0:x1] = 0
        obj[top:bottom + 1, x0:x1] = d

    if noise_sigma > 0:
        D = D + rng.normal(0.0, noise_sigma, size=D.shape)
    if p_outlier > 0:
        m = rng.random(D.shape) < p_outlier
        D[m] = rng.uniform(0.0, cam.dmax, size=int(m.sum()))
    if p_invalid > 0:
        m = rng.random(D.shape) < p_invalid
        D[m] = 0.0
    D = np.clip(D, 0.0, cam.dmax).astype(np.float32)
    return Scene(D, cam, labels, obj, obstacles)


# --------------------------------------------------------------------------------------
# Workloads.  Seeds: workload n, frame i -> 1000 * n + i.

CONFIG1 = Camera(320, 120, stixel_width=5, dmax=64, focal_px=700.0, baseline_m=0.3,
                 camera_height_m=1.2, pitch_rad=0.0, horizon_row=40)
CONFIG2 = Camera(1024, 440, stixel_width=5, dmax=128, focal_px=700.0, baseline_m=0.3,
                 camera_height_m=1.2, pitch_rad=0.0, horizon_row=180)
# width / height sweep: 1024x440 at s = 3, 5, 7, 11 and 2048x880 at s = 5
CONFIG3 = [replace(CONFIG2, stixel_width=s) for s in (3, 5, 7, 11)] + [
    Camera(2048, 880, stixel_width=5, dmax=128, focal_px=1400.0, baseline_m=0.3,
           camera_height_m=1.2, pitch_rad=0.0, horizon_row=400)]
OBSTACLES = {1: (3, 6), 2: (8, 20), 3: (8, 20), 4: (8, 20), 5: (8, 20)}


def _batched_camera(i: int) -> Camera:
    """Frame i of the 64-frame mixed batch: 24 x 640x240, 32 x 1024x440, 8 x 2048x880;
    stixel width alternates 5 / 7 by frame index; dmax 64 only for 640x240 frames
    at even index, 128 otherwise."""
    s = 5 if i % 2 == 0 else 7
    if i < 24:
        return Camera(640, 240, stixel_width=s, dmax=64 if i % 2 == 0 else 128,
                      focal_px=700.0, baseline_m=0.3, camera_height_m=1.2, horizon_row=80)
    if i < 56:
        return replace(CONFIG2, stixel_width=s)
    return replace(CONFIG3[-1], stixel_width=s)


CONFIG4 = [_batched_camera(i) for i in range(64)]


def serving_cameras(seed: int = 5000) -> List[Camera]:
    """Eight cameras: 0-2 at 640x240, 3-5 at 1024x440, 6-7 at 2048x880, stixel width 5.
    Height 1.0-1.6 m, baseline 0.2-0.5 m, horizon 0.35-0.45 H, pitch 0-2 degrees,
    redrawn until the bottom-row ground disparity is at most 0.9 dmax."""
    rng = np.random.default_rng(seed)
    sizes = [(640, 240, 64)] * 3 + [(1024, 440, 128)] * 3 + [(2048, 880, 128)] * 2
    cams = []
    for (W, H, dmax) in sizes:
        while True:
            h = float(rng.uniform(1.0, 1.6))
            b = float(rng.uniform(0.2, 0.5))
            hz = int(round(float(rng.uniform(0.35, 0.45)) * H))
            pitch = math.radians(float(rng.uniform(0.0, 2.0)))
            cam = Camera(W, H, stixel_width=5, dmax=dmax, focal_px=700.0 * W / 1024,
                         baseline_m=b, camera_height_m=h, pitch_rad=pitch, horizon_row=hz)
            if cam.alpha * (H - 1 - hz) <= 0.9 * dmax:
                cams.append(cam)
                break
    return cams


def camera_for(config: int, frame: int = 0) -> Camera:
    if config == 1:
        return CONFIG1
    if config == 2:
        return CONFIG2
    if config == 3:
        return CONFIG3[frame % len(CONFIG3)]
    if config == 4:
        return CONFIG4[frame % 64]
    if config == 5:
        return serving_cameras()[frame % 8]
    raise ValueError(f"unknown workload {config}")


def config_frames(config: int, n: Optional[int] = None) -> List[Scene]:
    """The frames of workload `config` (all of them, or the first n)."""
    counts = {1: 1, 2: 1, 3: len(CONFIG3), 4: 64, 5: 8}
    n = counts[config] if n is None else n
    return [make_scene(camera_for(config, i), 1000 * config + i, n_obstacles=OBSTACLES[config])
            for i in range(n)]
