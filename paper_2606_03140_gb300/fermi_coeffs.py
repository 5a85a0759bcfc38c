"""Polynomial coefficients of the finite-temperature Fermi-operator recursion (GPU path).

The recursion writes the Fermi operator as F = (I + U_n) / 2 with U_n = tanh(beta (mu - h~) / 2)
and builds U_n from a low-temperature start by the doubling identity of tanh,
tanh(2a) = 2 tanh(a) / (1 + tanh(a)^2):

* start: U_0 = tanh(z), z = beta_0 (mu I - h~) / 2, beta_0 = beta / 2^n, with every
  eigenvalue of z in [-1, 1]; tanh is taken as the odd polynomial z q(z^2) below;
* n doublings: U <- 2 U (I + U^2)^-1, with (I + V)^-1, V = U^2 in [0, 1], taken as the
  polynomial r(V) below.

Both polynomials are near-minimax fits (Lawson-weighted least squares on Chebyshev nodes) in
the monomial basis, whose coefficients stay below 1 in magnitude on these intervals.  Running
this file prints the C arrays held in ``csrc/fermi_coeffs.h``; the degrees are one pair for
the FP32-class forms and one for the FP64 form.  Nothing here is used at run time.
"""
import numpy as np


def lawson_fit(fun, a, b, powers, npts=6000, iters=80):
    x = np.cos(np.pi * (np.arange(npts) + 0.5) / npts) * (b - a) / 2 + (a + b) / 2
    y = fun(x)
    A = np.stack([x ** p for p in powers], axis=1)
    w = np.full(npts, 1.0 / npts)
    c = None
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * sw[:, None], y * sw, rcond=None)
        e = np.abs(A @ c - y)
        w = w * (e + 1e-300)
        w /= w.sum()
    xx = np.linspace(a, b, 400001)
    err = float(np.max(np.abs(np.stack([xx ** p for p in powers], axis=1) @ c - fun(xx))))
    return c, err


def tanh_coeffs(deg):
    """a_k of tanh(z) ~ sum_k a_k z^(2k+1) on [-1, 1] (deg odd)."""
    return lawson_fit(np.tanh, -1.0, 1.0, [2 * k + 1 for k in range((deg - 1) // 2 + 1)])


def inv_coeffs(deg):
    """c_k of 1 / (1 + v) ~ sum_k c_k v^k on [0, 1]."""
    return lawson_fit(lambda v: 1.0 / (1.0 + v), 0.0, 1.0, list(range(deg + 1)))


def c_array(name, c):
    body = ", ".join(f"{v:.17e}" for v in c)
    return f"constexpr double {name}[{len(c)}] = {{{body}}};"


if __name__ == "__main__":
    for tag, dt, di in (("Mixed", 15, 9), ("F64", 23, 15)):
        ct, et = tanh_coeffs(dt)
        ci, ei = inv_coeffs(di)
        print(f"// {tag}: tanh degree {dt} (max error {et:.1e} on [-1, 1]); "
              f"(1 + v)^-1 degree {di} (max error {ei:.1e} on [0, 1])")
        print(c_array(f"kTanh{tag}", ct))
        print(c_array(f"kInv{tag}", ci))
