"""Coefficients of the polynomials in sq::box_muller
(include/squares_device.cuh).

Each polynomial is the least-squares fit, in double precision, of the target
function on 2000 Chebyshev nodes of its interval (a near-minimax
polynomial: least squares on Chebyshev nodes approximates the Chebyshev
interpolant, whose error is within a small factor of the minimax error),
then rounded to float32.

* Angle. The remainder is theta' = (pi/4) t with t in [-1, 1).
  sin(theta') = t * P(t^2) and cos(theta') = Q(t^2), P and Q of degree 3
  (t^1..t^7 and t^0..t^6), fitted to sin((pi/4) t) / t and cos((pi/4) t).
  Errors with the float32 coefficients: about 2.4e-8 and 5.4e-8.
* Log. ln(1 + f) = 2 atanh(s) with |s| <= 0.1716 (plus a little when the
  rounding of float(k) moves the exponent split); atanh(s) = s * A(s^2),
  A of degree 2 (s, s^3, s^5), fitted to atanh(s) / s on |s| <= 0.18. Error
  about 3.6e-8 (Taylor to s^7: 2.3e-8). The header holds -4 * A's
  coefficients, so that s * p = -4 atanh(s) (exact: a power-of-two scaling).

Running this file prints the coefficients; tests/test_fit_box_muller.py
checks that the constants in the header equal them.
"""
import numpy as np

NODES = 2000


def _nodes(half_width):
    return np.cos(np.pi * (np.arange(NODES) + 0.5) / NODES) * half_width


def _lstsq(u, target, degree):
    vander = np.vstack([u ** k for k in range(degree + 1)]).T
    c, *_ = np.linalg.lstsq(vander, target, rcond=None)
    return c.astype(np.float32)


def _fit_odd(f, half_width, degree):
    """f(t) = t * P(t^2): P's coefficients."""
    t = _nodes(half_width)
    return _lstsq(t * t, f(t) / t, degree)


def _fit_even(f, half_width, degree):
    """f(t) = Q(t^2): Q's coefficients."""
    t = _nodes(half_width)
    return _lstsq(t * t, f(t), degree)


def fit():
    """(sin_coeffs, cos_coeffs) as float32 arrays, lowest power of t^2 first."""
    a = np.pi / 4
    return _fit_odd(lambda t: np.sin(a * t), 1.0, 3), _fit_even(lambda t: np.cos(a * t), 1.0, 3)


ATANH_HALF_WIDTH = 0.18


def fit_atanh():
    """A's coefficients (float32, lowest power of s^2 first)."""
    return _fit_odd(np.arctanh, ATANH_HALF_WIDTH, 2)


def max_errors():
    """Largest |fit - exact| of the sine, cosine and atanh fits over fine
    grids of their intervals, in double precision with the float32
    coefficients."""
    s, c = fit()
    t = np.linspace(-1.0, 1.0, 200001)
    u = t * t
    a = np.pi / 4
    es = np.max(np.abs(np.polyval(s.astype(np.float64)[::-1], u) * t - np.sin(a * t)))
    ec = np.max(np.abs(np.polyval(c.astype(np.float64)[::-1], u) - np.cos(a * t)))
    h = fit_atanh()
    x = np.linspace(-ATANH_HALF_WIDTH, ATANH_HALF_WIDTH, 200001)
    eh = np.max(np.abs(np.polyval(h.astype(np.float64)[::-1], x * x) * x - np.arctanh(x)))
    return float(es), float(ec), float(eh)


if __name__ == "__main__":
    s, c = fit()
    h = fit_atanh()
    print("sin:", " ".join(f"{x:.8e}f" for x in s))
    print("cos:", " ".join(f"{x:.8e}f" for x in c))
    print("-4 atanh:", " ".join(f"{x:.8e}f" for x in (-4 * h)))
    print("max errors (sin, cos, atanh):", max_errors())
