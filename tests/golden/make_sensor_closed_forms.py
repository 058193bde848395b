"""Writes sensor_closed_forms.txt: closed-form values of the sensor model's
constants (Eq. 3 and Eq. 4 of the paper), evaluated with 40-digit mpmath.

This script uses neither the oracle nor the CUDA library: the values follow
from the definitions alone --
  C_out = ln(d_range / p_out)                      (uniform branch of Eq. 4)
  K(f)  = ln A_norm(f) + ln(sigma sqrt(2 pi)) - ln(1 - p_out)
  A_norm(f) = Phi((d_range - f) / sigma) - Phi(-f / sigma)
with d_range = dmax and Phi the standard normal CDF.  Run it from the
repository root:  python tests/golden/make_sensor_closed_forms.py
"""
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 40

CASES = [  # dmax, p_out, sigma, f
    (64, 0.05, 1.0, 0), (64, 0.05, 1.0, 1), (64, 0.05, 1.0, 32), (64, 0.05, 1.0, 64),
    (128, 0.05, 1.0, 0), (128, 0.05, 1.0, 17), (128, 0.2, 2.5, 3), (32, 0.01, 0.5, 0),
]


def phi(x):
    return mp.ncdf(x)


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sensor_closed_forms.txt")
    with open(out, "w") as fh:
        fh.write("# Closed forms of the sensor model (paper Eq. 3 / Eq. 4), 40-digit mpmath.\n")
        fh.write("# Parameters are single-precision values, as the library receives them.\n")
        fh.write("# columns: dmax p_out sigma f C_out K(f)\n")
        for dmax, p_out, sigma, f in CASES:
            p32 = mp.mpf(float(np.float32(p_out)))
            s32 = mp.mpf(float(np.float32(sigma)))
            d = mp.mpf(dmax)
            c_out = mp.log(d) - mp.log(p32)
            a = phi((d - f) / s32) - phi(-mp.mpf(f) / s32)
            k = mp.log(a) + mp.log(s32 * mp.sqrt(2 * mp.pi)) - mp.log(1 - p32)
            fh.write(f"{dmax} {p_out!r} {sigma!r} {f} {mp.nstr(c_out, 25)} {mp.nstr(k, 25)}\n")


if __name__ == "__main__":
    main()
