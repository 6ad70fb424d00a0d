"""Pins of the oracle's least-squares Farrow design (Sec. II-B, Eq. 3-4) and of
the oracle's synthesis with a given Farrow table (no GPU).

- limits with known optima: a vanishing passband without weight above it gives
  the maximally flat (Lagrange) interpolator; a uniform weight over the whole
  band decouples the taps, so each tap is the L2 projection of the ideal
  sinc(alpha + k) onto polynomials of the order;
- the time-reversal symmetry h(k; alpha) = h(-1 - k; 1 - alpha) of the problem;
- a motionless source with a Farrow table equals the static image-source RIR
  (built here from brute-force mirrored images and numpy polynomials)
  convolved with the signal.
"""
import numpy as np
import pytest

from oracle import api as oracle
from oracle import brute
from oracle import gls
from tests.scenes import rel_l2


def _lagrange(nodes, i, x):
    r = 1.0
    for j, nj in enumerate(nodes):
        if j != i:
            r *= (x - nj) / (nodes[i] - nj)
    return r


@pytest.mark.parametrize("L,M", [(2, 1), (4, 3)])
def test_small_passband_is_lagrange(L, M):
    # taps k = -L/2 .. L/2-1 read x[m0 - k], i.e. the samples at offsets -k
    c = gls.design(L, M, 0.02, stop_weight=0.0)
    alpha = np.array([0.0, 0.25, 0.6, 0.95])
    h = gls.taps_at(c, alpha)
    nodes = [-k for k in range(-L // 2, L // 2)]
    ref = np.array([[_lagrange(nodes, i, a) for a in alpha] for i in range(L)])
    assert np.max(np.abs(h - ref)) < 1e-3


@pytest.mark.parametrize("L,M", [(8, 2), (16, 4)])
def test_uniform_full_band_is_per_tap_projection(L, M):
    c = gls.design(L, M, 0.5, stop_weight=1.0)
    xa, wa = np.polynomial.legendre.leggauss(48)
    a, wa = 0.5 * (xa + 1.0), 0.5 * wa
    V = np.vander(a, M + 1, increasing=True)
    G = V.T @ (wa[:, None] * V)
    ref = np.stack([np.linalg.solve(G, V.T @ (wa * np.sinc(a + k))) for k in range(-L // 2, L // 2)])
    assert np.max(np.abs(c - ref)) < 1e-9


@pytest.mark.parametrize("L,M,p", [(8, 1, 0.5), (32, 4, 0.9), (64, 3, 0.8)])
def test_time_reversal_symmetry(L, M, p):
    c = gls.design(L, M, p)
    a = np.linspace(0.0, 1.0, 11)
    assert np.max(np.abs(gls.taps_at(c, a) - gls.taps_at(c, 1.0 - a)[::-1])) < 1e-11


def test_response_improves_with_order():
    w = np.linspace(0.0, 0.85 * np.pi, 64)
    errs = []
    for M in (1, 2, 3, 4):
        c = gls.design(32, M, 0.85)
        errs.append(max(np.max(np.abs(gls.response(c, a, w) - np.exp(1j * w * a)))
                        for a in np.linspace(0.0, 1.0, 9)))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])) and errs[-1] < 0.05


def test_static_source_with_farrow_table():
    L, M, fs, c0 = 16, 3, 16000.0, 343.0
    coef = gls.design(L, M, 0.8)
    src = np.array([1.3, 1.1, 1.4])
    sc = oracle.Scene(dims=(5.0, 4.0, 3.0), beta=(0.7, 0.8, 0.6, 0.9, 0.75, 0.65), mic=(2.5, 2.0, 1.2),
                      K=2, fs=fs, tiers=((1, 1), (10**9, 16)), taps=L, window=2, farrow=coef,
                      traj_kind=0, traj=list(src) + [1.0, 0.5, 0.2, 0.0], duration=1.0)
    x = np.random.default_rng(9).standard_normal(2000)
    y = oracle.synthesize(sc, x)
    h = np.zeros(1500)
    mic = np.array(sc.mic)
    for sign, off, hits in brute.mirror_images(sc.dims, 2 * sc.K + 3):
        n_lat, _ = brute.lattice_of(sign, off, sc.dims)
        if sum(abs(v) for v in n_lat) > sc.K:
            continue
        d = np.linalg.norm(np.array(sign) * src + np.array(off) - mic)
        tau = d * fs / c0
        gain = np.prod([sc.beta[w] ** hits[w] for w in range(6)]) / (4 * np.pi * d)
        ct = int(np.ceil(tau))
        alpha = ct - tau                     # read position n - tau = (n - ceil(tau)) + alpha
        for i, k in enumerate(range(-L // 2, L // 2)):
            h[ct + k] += gain * np.polynomial.polynomial.polyval(alpha, coef[i])
    ref = np.convolve(x, h)[: x.size]
    assert rel_l2(y, ref) < 1e-12
