"""Host-side checks of the CUDA library that need no GPU: the shared object
loads and exports every entry point of include/stixels.h, its defaults and
its fixed-point model tables agree exactly with the oracle's (which computes
them independently), and invalid parameters are rejected."""
import math
import os
import re

import numpy as np
import pytest

import oracle
import paper_1610_04124_gb300 as S
import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stixels.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stixels_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 14
    L = S.lib()
    for n in names:
        assert hasattr(L, n), n


def test_defaults_match_oracle_defaults():
    d = S.default_params().to_dict()
    o = oracle.DEFAULTS
    for k, v in d.items():
        if k in ("max_stixels_per_col",):
            continue
        ov = o[k]
        if isinstance(v, tuple):
            assert np.allclose(np.array(v, dtype=np.float64), np.float32(np.array(ov, dtype=np.float64)),
                               rtol=0, atol=0, equal_nan=False) or np.array_equal(
                np.array(v), np.float32(np.array(ov))), k
        elif isinstance(v, float):
            assert v == float(np.float32(ov)), k
        else:
            assert v == ov, k


PARAM_SETS = [
    dict(camera=scenes.CONFIG1),
    dict(camera=scenes.CONFIG2),
    dict(camera=scenes.CONFIG3[-1]),
    dict(camera=scenes.CONFIG1, sigma_object=1.7, sigma_ground=0.6, sigma_sky=2.2, p_out=0.13),
    dict(camera=scenes.CONFIG2, pitch_rad=0.03, baseline_m=0.45, camera_height_m=1.55, horizon_row=200,
         eps_gravity=0.4, eps_diving=2.3, eps_order=-0.7, cost_new_stixel=1.25),
]


def _both(ps):
    cam = ps.get("camera")
    kw = {k: v for k, v in ps.items() if k != "camera"}
    return S.default_params(cam, **kw), oracle.make_params(cam, **kw)


@pytest.mark.parametrize("i", range(len(PARAM_SETS)))
def test_model_tables_equal_oracle_constants(i):
    lp, op = _both(PARAM_SETS[i])
    H = 97 if i != 2 else 880
    t = S.model_tables(lp, H)
    mc = oracle.model_constants(op, H)
    U = S.UNITS_PER_COST
    sc = t["scalars"]
    assert sc[0] == mc["c_out"] * U
    assert sc[1] == mc["k_sky"] * U
    assert np.array_equal(t["k_obj"], mc["k_obj"] * U)
    assert np.array_equal(t["k_ground"], mc["k_ground"] * U)
    assert np.array_equal(t["fg"], mc["fg"])
    big = 1 << 29
    first = np.where(np.isinf(mc["first"]), big, mc["first"] * U)
    trans = np.where(np.isinf(mc["trans"]), big, mc["trans"] * U)
    assert np.array_equal(sc[2:5], first)
    assert np.array_equal(sc[5:14], trans.reshape(-1))
    assert np.array_equal(sc[14:17], mc["pens"] * U)


def _decide(thr_word, f):
    """(gravity, diving) decisions of a packed threshold word for disparity f."""
    fhi = ((thr_word & 0xffff) ^ 0x8000) - 0x8000
    flo = thr_word >> 16
    return f > fhi, f < flo


@pytest.mark.parametrize("i", range(len(PARAM_SETS)))
def test_thresholds_decide_as_the_unrounded_rule(i):
    """The per-row gravity / diving thresholds and the ordering offset give, for
    every integer disparity, the decision of the paper's comparisons on the
    unrounded ground line (Sec. 3 constraints): 16 f > 16 (f_g + eps_gravity),
    16 f < 16 (f_g - eps_diving), 16 f > 16 f' + 16 eps_order."""
    lp, op = _both(PARAM_SETS[i])
    H = 97 if i != 2 else 880
    t = S.model_tables(lp, H)
    fg = oracle.model_constants(op, H)["fg"]
    eg, ed, eo = float(np.float32(lp.eps_gravity)), float(np.float32(lp.eps_diving)), float(np.float32(lp.eps_order))
    for v in range(H):
        for f in range(0, lp.dmax + 1):
            grav, div = _decide(int(t["thr"][v]), f)
            assert grav == (16.0 * f > 16.0 * (fg[v] + eg)), (v, f)
            assert div == (16.0 * f < 16.0 * (fg[v] - ed)), (v, f)
    off = int(t["scalars"][17])
    for d in range(-300, 301):
        assert (d > off) == (16.0 * d > 16.0 * eo), d


def _llround(x):
    """C's llround for x >= 0: nearest integer, halves away from zero (exact)."""
    n = math.floor(x)
    return n + 1 if x - n >= 0.5 else n


@pytest.mark.parametrize("i", [0, 3, 4])
def test_pixel_costs_from_tables_equal_oracle(i):
    """min(C_out, K + G[min(e, 16 dmax)]) from the library's tables equals the oracle's Eq. 4."""
    lp, op = _both(PARAM_SETS[i])
    H = 60
    t = S.model_tables(lp, H)
    U = S.UNITS_PER_COST
    c_out, k_sky = int(t["scalars"][0]), int(t["scalars"][1])
    emax = 16 * lp.dmax
    rng = np.random.default_rng(i)
    for _ in range(300):
        q = int(rng.integers(0, emax + 1)); f = int(rng.integers(0, lp.dmax + 1)); v = int(rng.integers(0, H))
        obj = min(c_out, int(t["k_obj"][f]) + int(t["g_obj"][min(abs(q - 16 * f), emax)]))
        # the ground residual at the unrounded line, in FP64 as the LUT kernel
        # evaluates it, rounded to the 2^-12 grid
        sg = float(np.float32(lp.sigma_ground))
        dpx = q / 16.0 - float(t["fg"][v])
        gres = 4 * _llround(4096.0 * min(dpx * dpx / (2.0 * sg * sg), 65536.0))
        gnd = min(c_out, int(t["k_ground"][v]) + gres)
        sky = min(c_out, k_sky + int(t["g_sky"][q]))
        assert obj == oracle.pixel_cost(op, H, oracle.OBJECT, v, q, f) * U
        assert gnd == oracle.pixel_cost(op, H, oracle.GROUND, v, q) * U
        assert sky == oracle.pixel_cost(op, H, oracle.SKY, v, q) * U


@pytest.mark.parametrize("bad", [
    dict(dmax=0), dict(dmax=256), dict(stixel_width=0), dict(stixel_width=17), dict(p_out=0.0), dict(p_out=1.0),
    dict(sigma_object=0.0), dict(sigma_ground=float("nan")), dict(camera_height_m=0.0),
    dict(prior_first=(1.0, -0.5, 1.0)), dict(cost_diving=float("inf")), dict(cost_new_stixel=float("inf")),
    dict(eps_gravity=-1.0), dict(eps_order=200.0), dict(reduce_mode=2), dict(max_stixels_per_col=0),
    dict(sigma_sky=900.0),            # residual table would not reach the outlier branch
    dict(pixel_grid=2), dict(sigma_gain=-1.0), dict(sigma_gain=11.0), dict(sigma_gain=float("nan")),
    dict(sigma_gain=0.5, sigma_width=0.0), dict(sigma_gain=0.5, sigma_mid=float("inf")),
    dict(sigma_gain=0.5),             # valid, but its per-disparity tables are not exported
])
def test_invalid_params_rejected(bad):
    p = S.default_params(**bad)
    with pytest.raises(S.StixelsError) as e:
        S.model_tables(p, 10)
    assert e.value.status == S.E_INVALID_ARG


def test_lut_pitch():
    for H in [0, 1, 2, 3, 4, 5, 119, 120, 440, 880, 2048]:
        P = S.lut_pitch(H)
        assert P % 4 == 0 and H + 1 <= P < H + 5
