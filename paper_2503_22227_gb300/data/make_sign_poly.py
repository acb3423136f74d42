"""Writes sign_cheb63.txt: the Chebyshev coefficients c_0 .. c_63 of the
degree-63 interpolant of tanh(8x) on [-1, 1] (interpolation at the
Chebyshev points of the first kind; the even coefficients, zero by the
odd symmetry of tanh up to rounding, are set to exactly zero).  This is
the smooth sign approximation of the serving workload's range predicate.

    python -m paper_2503_22227_gb300.data.make_sign_poly
"""
import os

import numpy as np


def coefficients() -> np.ndarray:
    c = np.polynomial.chebyshev.Chebyshev.interpolate(lambda x: np.tanh(8.0 * x), 63).coef
    c = np.array(c, dtype=np.float64)
    c[0::2] = 0.0
    return c


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sign_cheb63.txt")
    with open(path, "w") as f:
        f.write("# Chebyshev coefficients c_0..c_63 of the degree-63 interpolant of tanh(8x)\n")
        f.write("# on [-1, 1]; written by make_sign_poly.py\n")
        for v in coefficients():
            f.write(repr(float(v)) + "\n")
    print(path)
