"""Pins of the oracle's precision envelope (no GPU).

Where a read position n - tau lies within delta samples of an integer, the side
of the integer it falls on is decided by the precision of the delay, and both
sides are evaluations of the method (Eq. 5 and 8). The envelope holds, per
output (or per input sample for the adjoint), the difference between the two
sides. Pinned here:
- delta = 0: no envelope, and the output is the plain synthesis;
- the windowed sinc (Hann, Kaiser) is continuous across the wrap, h(k; 1) =
  h(k + 1; 0): its envelope is negligible;
- a first-order least-squares Farrow design jumps at the wrap: for a motionless
  source in free field whose delay lies 1e-9 samples below an integer, the
  envelope equals the change between two plain oracle runs with the delay just
  below and just above that integer (forward, and the adjoint for a single
  upstream sample).
"""
import numpy as np

from oracle import api as oracle
from oracle import gls

EPS = 1e-9


def _still_free_field(D_minus_eps: float, window=2, taps=8, order=1, passband=0.5):
    # direct path only (all walls absorbing), source at rest 0.86 m from the
    # microphone; c set so that the delay is exactly the requested value
    fs = 16000.0
    src, mic = np.array([2.3, 2.0, 1.4]), np.array([1.6, 2.5, 1.2])
    d = float(np.linalg.norm(src - mic))
    c = d * fs / D_minus_eps
    farrow = gls.design(taps, order, passband) if window == 2 else None
    return oracle.Scene(dims=(5.0, 4.0, 3.0), beta=(0.0,) * 6, mic=tuple(mic), K=0, fs=fs, c=c,
                        tiers=((10**9, 16),), taps=taps, window=window, traj_kind=0,
                        traj=list(src) + [1.0, 0.0, 0.0, 0.0], duration=1.0, farrow=farrow)


def test_zero_delta_is_the_plain_synthesis():
    sc = _still_free_field(40.0 - 0.3)
    x = np.random.default_rng(1).standard_normal(600)
    y, env = oracle.synthesize_envelope(sc, x, delta=0.0)
    assert np.array_equal(y, oracle.synthesize(sc, x))
    assert not env.any()


def test_windowed_sinc_is_continuous_across_the_wrap():
    x = np.random.default_rng(2).standard_normal(600)
    for window in (0, 1):
        sc = _still_free_field(40.0 - EPS, window=window, taps=32)
        y, env = oracle.synthesize_envelope(sc, x, delta=1e-4)
        assert np.linalg.norm(env) < 1e-6 * np.linalg.norm(y)


def test_envelope_is_the_jump_between_the_two_sides():
    x = np.random.default_rng(3).standard_normal(600)
    below = _still_free_field(40.0 - EPS)      # read position just above an integer (alpha = EPS)
    above = _still_free_field(40.0 + EPS)      # just below it (alpha = 1 - EPS, one sample earlier)
    y0, env = oracle.synthesize_envelope(below, x, delta=1e-4)
    y1 = oracle.synthesize(above, x)
    jump = np.abs(y1 - y0)
    assert np.max(jump) > 1e-3 * np.max(np.abs(y0))        # the design does jump
    assert np.max(np.abs(env - jump)) < 1e-7 * np.max(np.abs(y0))
    # a delta below the offset sees no wrap
    _, env_small = oracle.synthesize_envelope(below, x, delta=EPS / 2)
    assert not env_small.any()


def test_adjoint_envelope_is_the_jump_between_the_two_sides():
    below, above = _still_free_field(40.0 - EPS), _still_free_field(40.0 + EPS)
    n_in = 600
    dy = np.zeros(n_in)
    dy[300] = 1.7                                  # one upstream sample: no sums of signs
    dx0, env = oracle.adjoint_x_envelope(below, dy, n_in, delta=1e-4)
    dx1 = oracle.adjoint_x(above, dy, n_in)
    assert np.array_equal(dx0, oracle.adjoint_x(below, dy, n_in))
    jump = np.abs(dx1 - dx0)
    assert np.max(jump) > 1e-3 * np.max(np.abs(dx0))
    assert np.max(np.abs(env - jump)) < 1e-7 * np.max(np.abs(dx0))
