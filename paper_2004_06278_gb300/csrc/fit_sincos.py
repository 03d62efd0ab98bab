"""Coefficients of the sine and cosine polynomials in sq::box_muller
(include/squares_device.cuh).

The Box-Muller angle's remainder is theta' = (pi/4) t with t in [-1, 1).
sin(theta') is taken as t * P(t^2) and cos(theta') as Q(t^2), with P and Q
of degree 3 (so t^1..t^7 and t^0..t^6). Each is the least-squares fit, in
double precision, of sin((pi/4) t) / t and cos((pi/4) t) on 2000 Chebyshev
nodes of [-1, 1] (a near-minimax polynomial: least squares on Chebyshev
nodes approximates the Chebyshev interpolant, whose error is within a small
factor of the minimax error), then rounded to float32. The maximum error
of the double-precision fits over [-1, 1] is about 2.4e-9 for the sine and
2.8e-8 for the cosine; with the coefficients rounded to float32, about
2.4e-8 and 5.4e-8, at the float32 rounding of the evaluation itself.

Running this file prints the coefficients; tests/test_fit_sincos.py checks
that the constants in the header equal them.
"""
import numpy as np

NODES = 2000
DEGREE = 3  # in t^2


def fit():
    """(sin_coeffs, cos_coeffs) as float32 arrays, lowest power of t^2 first."""
    t = np.cos(np.pi * (np.arange(NODES) + 0.5) / NODES)
    u = t * t
    vander = np.vstack([u ** k for k in range(DEGREE + 1)]).T
    a = np.pi / 4
    sin_c, *_ = np.linalg.lstsq(vander, np.sin(a * t) / t, rcond=None)
    cos_c, *_ = np.linalg.lstsq(vander, np.cos(a * t), rcond=None)
    return sin_c.astype(np.float32), cos_c.astype(np.float32)


def max_errors():
    """Largest |fit - exact| over a fine grid of [-1, 1], in double precision
    with the float32 coefficients."""
    s, c = fit()
    t = np.linspace(-1.0, 1.0, 200001)
    u = t * t
    a = np.pi / 4
    ps = np.polyval(s.astype(np.float64)[::-1], u) * t
    pc = np.polyval(c.astype(np.float64)[::-1], u)
    return float(np.max(np.abs(ps - np.sin(a * t)))), float(np.max(np.abs(pc - np.cos(a * t))))


if __name__ == "__main__":
    s, c = fit()
    print("sin:", " ".join(f"{x:.8e}f" for x in s))
    print("cos:", " ".join(f"{x:.8e}f" for x in c))
    print("max errors (sin, cos):", max_errors())
