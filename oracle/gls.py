"""Least-squares Farrow fractional-delay design for the FP64 oracle.

TEST INFRASTRUCTURE ONLY (see oracle/api.py). Independent of the CUDA library,
which designs its own table by another route.

Sec. II-B, Eq. 3-4: the tap weights of an L-tap fractional-delay filter are
polynomials of order M in the fractional delay, h(k; alpha) = sum_q c_q(k)
alpha^q, with coefficients chosen by a least-squares fit of the frequency
response in the complex domain (the design the text names). Convention of this
repository: taps k = -L/2 .. L/2-1 act as y = sum_k h(k; alpha) x[m0 - k] for
the read position m0 + alpha, so the ideal response is
    sum_k h(k; alpha) e^{-j w k} = e^{j w alpha}     (|w| < pi, alpha in [0, 1)),
whose exact solution is h(k; alpha) = sinc(alpha + k). The design minimises
    integral over alpha in [0, 1] and w in [0, pi] of
    V(w) | sum_k h(k; alpha) e^{-j w k} - e^{j w alpha} |^2,
    V = 1 on the passband [0, passband pi] and STOP_WEIGHT above it,
over the real coefficients c_q(k). The paper fits the passband; the small
weight above it (a reading: the passband-only problem is rank deficient, its
Gram matrix has eigenvalues near zero) makes the optimum unique. Here the
integrals are Gauss-Legendre rules on [0, passband pi], [passband pi, pi] and
[0, 1], and the problem is solved as one real linear least-squares system
(real and imaginary parts stacked).
"""
from __future__ import annotations

import numpy as np

STOP_WEIGHT = 1e-3


def design(taps: int, order: int, passband: float, stop_weight: float = STOP_WEIGHT,
           n_w: int = 0, n_a: int = 32) -> np.ndarray:
    """Coefficients c[k + L/2][q] (taps x (order + 1)) of the least-squares
    Farrow design for `taps` taps, polynomial order `order`, passband edge
    `passband` * pi and weight `stop_weight` above the passband."""
    L, M = int(taps), int(order)
    if L < 2 or L % 2 or not 1 <= M <= 8 or not 0.0 < passband < 1.0:
        raise ValueError("taps even >= 2, order 1..8, passband in (0, 1)")
    n_w = n_w or 4 * L + 32
    xw, ww = np.polynomial.legendre.leggauss(n_w)
    xa, wa = np.polynomial.legendre.leggauss(n_a)
    wp = passband * np.pi
    w = np.concatenate([0.5 * wp * (xw + 1.0), wp + 0.5 * (np.pi - wp) * (xw + 1.0)])
    w_w = np.concatenate([0.5 * wp * ww, stop_weight * 0.5 * (np.pi - wp) * ww])
    n_w = w.size
    a = 0.5 * (xa + 1.0)                 # delay nodes on [0, 1]
    w_a = 0.5 * wa
    k = np.arange(-L // 2, L // 2)
    q = np.arange(M + 1)
    W, A = np.meshgrid(w, a, indexing="ij")                      # (n_w, n_a)
    sq = np.sqrt(np.outer(w_w, w_a))                             # quadrature weights
    # columns (k, q): alpha^q e^{-j w k}
    cols = (A[..., None, None] ** q[None, None, None, :]) * np.exp(-1j * W[..., None, None] * k[None, None, :, None])
    cols = cols * sq[..., None, None]
    target = np.exp(1j * W * A) * sq
    Phi = cols.reshape(n_w * n_a, L * (M + 1))
    rhs = target.reshape(-1)
    Ar = np.concatenate([Phi.real, Phi.imag])
    br = np.concatenate([rhs.real, rhs.imag])
    sol, *_ = np.linalg.lstsq(Ar, br, rcond=None)
    return sol.reshape(L, M + 1)


def taps_at(c: np.ndarray, alpha) -> np.ndarray:
    """h(k; alpha) for every tap (rows) at the given alpha values (columns)."""
    a = np.atleast_1d(np.asarray(alpha, dtype=np.float64))
    return np.stack([np.polynomial.polynomial.polyval(a, c[i]) for i in range(c.shape[0])])


def response(c: np.ndarray, alpha: float, w) -> np.ndarray:
    """sum_k h(k; alpha) e^{-j w k} of the design."""
    L = c.shape[0]
    k = np.arange(-L // 2, L // 2)
    h = taps_at(c, alpha)[:, 0]
    return np.exp(-1j * np.outer(np.atleast_1d(w), k)) @ h
