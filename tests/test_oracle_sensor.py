"""Pins of the oracle's sensor model (paper Eq. 3 and Eq. 4) against facts
that do not come from the oracle itself: probability normalisation, closed
forms evaluated at 40 digits, the geometry of the ground line, and the
resolution bound of the fixed cost grid."""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sensor_closed_forms.txt")


@pytest.mark.parametrize("dmax,p_out,sigma", [(64, 0.05, 1.0), (128, 0.2, 2.5), (32, 0.01, 0.5)])
@pytest.mark.parametrize("cls", [oracle.OBJECT, oracle.GROUND, oracle.SKY])
def test_gaussian_branch_carries_inlier_mass(dmax, p_out, sigma, cls):
    """Eq. 3: the Gaussian component, normalised by A_norm over [0, d_range],
    integrates to 1 - p_out for any model disparity f inside the range."""
    p = oracle.make_params(dmax=dmax, p_out=p_out, sigma_object=sigma, sigma_ground=sigma,
                           sigma_sky=sigma, quantize=0)
    p_out32 = float(np.float32(p_out))
    for f in [0.0, 0.3, dmax / 2.0, dmax - 0.7, float(dmax)]:
        val, _ = integrate.quad(lambda d: math.exp(-oracle.gaussian_branch(p, cls, f, d)), 0.0, float(dmax),
                                points=[f], limit=400, epsabs=1e-13, epsrel=1e-12)
        assert abs(val - (1.0 - p_out32)) < 1e-9, (f, val)


@pytest.mark.parametrize("dmax,p_out", [(64, 0.05), (128, 0.3)])
def test_outlier_branch_carries_outlier_mass(dmax, p_out):
    """Eq. 3-4: the uniform branch is p_out / d_range, so exp(-C_out) * d_range = p_out.
    A pixel far from the model disparity costs exactly that branch."""
    p = oracle.make_params(dmax=dmax, p_out=p_out, quantize=0)
    c = oracle.pixel_cost(p, 10, oracle.OBJECT, 0, 16 * dmax, 0)
    assert abs(math.exp(-c) * dmax - float(np.float32(p_out))) < 1e-12
    pq = oracle.make_params(dmax=dmax, p_out=p_out, quantize=1)
    cq = oracle.pixel_cost(pq, 10, oracle.OBJECT, 0, 16 * dmax, 0)
    assert abs(cq - c) <= 2.0 ** -13 and (cq * 4096.0).is_integer()


def test_closed_forms():
    """C_out and K(f) against 40-digit closed forms (tests/golden, written by a
    script that uses only mpmath)."""
    rows = [l.split() for l in open(GOLDEN) if not l.startswith("#")]
    assert len(rows) >= 8
    for dmax, p_out, sigma, f, c_out, k in rows:
        p = oracle.make_params(dmax=int(dmax), p_out=float(p_out), sigma_object=float(sigma), quantize=0)
        mc = oracle.model_constants(p, 4)
        assert abs(mc["c_out"] - float(c_out)) < 1e-13
        assert abs(mc["k_obj"][int(f)] - float(k)) < 1e-13, (dmax, p_out, sigma, f)
        if int(f) == 0:
            p2 = oracle.make_params(dmax=int(dmax), p_out=float(p_out), sigma_sky=float(sigma), quantize=0)
            assert abs(oracle.model_constants(p2, 4)["k_sky"] - float(k)) < 1e-13


def test_pixel_cost_is_min_of_branches_and_minimal_at_model():
    """Eq. 4: cost = min(outlier branch, Gaussian branch); the Gaussian branch is
    smallest at d = f, where it equals K(f)."""
    p = oracle.make_params(dmax=64, quantize=0)
    c_out = oracle.model_constants(p, 8)["c_out"]
    rng = np.random.default_rng(1)
    for _ in range(200):
        f = int(rng.integers(0, 65)); q = int(rng.integers(0, 16 * 64 + 1))
        c = oracle.pixel_cost(p, 8, oracle.OBJECT, 0, q, f)
        g = oracle.gaussian_branch(p, oracle.OBJECT, float(f), q / 16.0)
        assert abs(c - min(c_out, g)) < 1e-12
    for f in [0, 5, 30, 64]:
        costs = [oracle.pixel_cost(p, 8, oracle.OBJECT, 0, q, f) for q in range(0, 16 * 64 + 1)]
        assert int(np.argmin(costs)) == 16 * f


def test_ground_line_geometry_and_row_direction():
    """Sec. 3.1: ground disparity alpha (v_hor - v); with v = 0 the bottom row and
    image row r = H-1-v, the cheapest ground disparity at r is alpha (r - horizon),
    alpha = baseline cos(pitch) / height."""
    H, hz = 60, 20
    p = oracle.make_params(dmax=64, horizon_row=hz, baseline_m=0.5, camera_height_m=1.0,
                           pitch_rad=0.1, quantize=0)
    alpha = float(np.float32(0.5)) * math.cos(float(np.float32(0.1))) / 1.0
    for v in [0, 5, 17, 30, 39]:
        r = H - 1 - v
        costs = [oracle.pixel_cost(p, H, oracle.GROUND, v, q) for q in range(0, 16 * 64 + 1)]
        best = int(np.argmin(costs)) / 16.0
        assert abs(best - alpha * (r - hz)) <= 1.0 / 32 + 1e-12, (v, best)
    pq = oracle.make_params(dmax=64, horizon_row=hz, baseline_m=0.5, camera_height_m=1.0,
                            pitch_rad=0.1, quantize=1)
    fg = oracle.model_constants(pq, H)["fg"]
    # the cost grid leaves the ground model itself alone: the line is not rounded
    for v in range(H):
        assert abs(fg[v] - alpha * (H - 1 - v - hz)) <= 1e-12


def test_cost_grid_resolution():
    """The fixed-point reading: each of the two Gaussian-branch terms and C_out is
    rounded to the 2^-12 grid, so a pixel cost moves by at most 2^-12 and lands on
    the grid (object and sky models; the ground line's own 1/16-px grid is separate)."""
    pu = oracle.make_params(dmax=128, sigma_object=1.3, sigma_sky=0.8, p_out=0.07, quantize=0)
    pq = oracle.make_params(dmax=128, sigma_object=1.3, sigma_sky=0.8, p_out=0.07, quantize=1)
    rng = np.random.default_rng(2)
    for _ in range(300):
        q = int(rng.integers(0, 16 * 128 + 1)); f = int(rng.integers(0, 129))
        for cls in (oracle.OBJECT, oracle.SKY):
            a = oracle.pixel_cost(pu, 4, cls, 0, q, f)
            b = oracle.pixel_cost(pq, 4, cls, 0, q, f)
            assert abs(a - b) <= 2.0 ** -12 + 1e-15
            assert (b * 4096.0).is_integer()


# ---- disparity-dependent noise (Eq. 3's sigma^c(f, v), a logistic in the model disparity)

@pytest.mark.parametrize("cls", [oracle.OBJECT, oracle.GROUND])
@pytest.mark.parametrize("gain", [0.8, -0.4])
def test_variable_sigma_branch_still_carries_inlier_mass(cls, gain):
    """With sigma depending on f, A_norm must be evaluated at that same sigma:
    the Gaussian branch still integrates to 1 - p_out at every f."""
    p = oracle.make_params(dmax=64, p_out=0.05, quantize=0, sigma_gain=gain, sigma_mid=20.0, sigma_width=6.0)
    for f in [0.0, 7.0, 20.0, 41.5, 64.0]:
        val, _ = integrate.quad(lambda d: math.exp(-oracle.gaussian_branch(p, cls, f, d)), 0.0, 64.0,
                                points=[f], limit=400, epsabs=1e-13, epsrel=1e-12)
        assert abs(val - (1.0 - float(np.float32(0.05)))) < 1e-9, (f, val)


def test_variable_sigma_closed_form_at_the_midpoint_and_tails():
    """At f = mid the logistic is 1/2: sigma = base (1 + gain / 2).  The branch's
    curvature in d is 1 / sigma^2, read from three values; far below / above mid
    the sigma tends to base and base (1 + gain)."""
    base, gain, mid, width = 1.2, 1.5, 24.0, 4.0
    p = oracle.make_params(dmax=64, quantize=0, sigma_object=base, sigma_gain=gain, sigma_mid=mid,
                           sigma_width=width)

    def curvature(f):
        h = 0.25
        g = [oracle.gaussian_branch(p, oracle.OBJECT, f, f + x) for x in (-h, 0.0, h)]
        return (g[0] - 2 * g[1] + g[2]) / (h * h)

    b32 = float(np.float32(base))                      # parameters are single precision
    assert abs(curvature(mid) - 1.0 / (b32 * (1 + gain / 2)) ** 2) < 1e-9
    assert abs(curvature(0.0) - 1.0 / (b32 * (1 + gain / (1 + math.exp(mid / width)))) ** 2) < 1e-9
    assert abs(curvature(64.0) - 1.0 / (b32 * (1 + gain / (1 + math.exp(-(64 - mid) / width)))) ** 2) < 1e-9


def test_zero_gain_is_the_constant_sigma_model():
    cam = scenes.CONFIG1
    sc = scenes.make_scene(cam, 4400)
    a = oracle.frame(oracle.make_params(cam), sc.disparity, cap=64)
    b = oracle.frame(oracle.make_params(cam, sigma_gain=0.0, sigma_mid=3.0, sigma_width=1.0), sc.disparity, cap=64)
    assert np.array_equal(a.cost, b.cost) and np.array_equal(a.counts, b.counts)
