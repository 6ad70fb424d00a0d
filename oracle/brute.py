"""Pure-Python brute force: a third, independent reading of the method for tiny
rooms (a few hundred images, a few hundred samples).

TEST INFRASTRUCTURE ONLY. It does not use oracle.cpp nor the CUDA library.
Images come from repeated mirroring of the source across the six walls
(breadth first), not from the lattice formula; the spline is evaluated with
de Boor's algorithm, not with the basis recursion; the Kaiser window uses its
own series. Everything is plain Python floats.
"""
from __future__ import annotations

import math


def mirror_images(dims, max_depth):
    """Breadth-first mirroring across walls x=0, x=Lx, y=0, y=Ly, z=0, z=Lz.

    Each image is an affine map of the source position, coordinate-wise
    q_d -> sign_d * q_d + offset_d, reached first at depth rho (its reflection
    count); hits[w] counts reflections off wall w on that shortest path.
    Returns a list of (sign[3], offset[3], hits[6]).
    """
    start = ((1, 1, 1), (0.0, 0.0, 0.0), (0, 0, 0, 0, 0, 0))
    seen = {(start[0], start[1])}
    out = [start]
    frontier = [start]
    for _ in range(max_depth):
        nxt = []
        for sign, off, hits in frontier:
            for w in range(6):
                a, side = divmod(w, 2)
                s, o = list(sign), list(off)
                # reflect q -> -q (plane 0) or q -> 2L - q (plane L) applied to s*q + o
                s[a] = -s[a]
                o[a] = -o[a] if side == 0 else 2.0 * dims[a] - o[a]
                key = (tuple(s), tuple(round(v, 9) for v in o))
                if key in seen:
                    continue
                seen.add(key)
                h = list(hits)
                h[w] += 1
                item = (tuple(s), tuple(o), tuple(h))
                out.append(item)
                nxt.append(item)
        frontier = nxt
    return out


def lattice_of(sign, off, dims):
    """(n, p) of a mirrored image: sign = 1 - 2p, offset = 2 n L."""
    p = [(1 - s) // 2 for s in sign]
    n = [int(round(o / (2.0 * L))) for o, L in zip(off, dims)]
    return n, p


def _deboor(ctrl, u):
    """Clamped uniform cubic B-spline at u in [0, 1] by de Boor's algorithm."""
    m = len(ctrl)
    segs = m - 3
    knots = [0.0] * 4 + [i / segs for i in range(1, segs)] + [1.0] * 4
    k = min(3 + int(u * segs), m - 1)  # knot span index with knots[k] <= u < knots[k+1]
    d = [list(ctrl[j + k - 3]) for j in range(4)]
    for r in range(1, 4):
        for j in range(3, r - 1, -1):
            i = j + k - 3
            den = knots[i + 4 - r] - knots[i]
            a = 0.0 if den == 0 else (u - knots[i]) / den
            d[j] = [(1 - a) * d[j - 1][c] + a * d[j][c] for c in range(3)]
    return d[3]


def _path(kind, tr, n_ctrl, duration, t):
    if kind == 0:
        nrm = math.sqrt(tr[3] ** 2 + tr[4] ** 2 + tr[5] ** 2)
        return [tr[i] + tr[6] * t * tr[3 + i] / nrm for i in range(3)]
    if kind == 1:
        ang = tr[5] + tr[4] * t / tr[3]
        return [tr[0] + tr[3] * math.cos(ang), tr[1] + tr[3] * math.sin(ang), tr[2]]
    ctrl = [tr[3 * i: 3 * i + 3] for i in range(n_ctrl)]
    return _deboor(ctrl, min(1.0, max(0.0, t / duration)))


def source(scene, t):
    return _path(scene.traj_kind, scene.traj, scene.n_ctrl, scene.duration, t)


def mic_at(scene, mic, t):
    """Microphone position at time t: static, or moved with the array by
    a(t) - a(0) when the scene has an array trajectory."""
    kind = getattr(scene, "arr_kind", -1)
    if kind < 0:
        return list(mic)
    a0 = _path(kind, scene.arr_traj, scene.arr_n_ctrl, scene.arr_duration, 0.0)
    at = _path(kind, scene.arr_traj, scene.arr_n_ctrl, scene.arr_duration, t)
    return [mic[d] + at[d] - a0[d] for d in range(3)]


def _bessel_i0(v):
    s, term, j = 1.0, 1.0, 1
    while term > 1e-18 * s:
        term *= (v / 2.0) ** 2 / (j * j)
        s += term
        j += 1
    return s


def _window(scene, u):
    L = scene.taps
    if scene.window == 0:
        return 0.5 + 0.5 * math.cos(2.0 * math.pi * u / L)
    z = max(0.0, 1.0 - (2.0 * u / L) ** 2)
    return _bessel_i0(scene.kaiser_beta * math.sqrt(z)) / _bessel_i0(scene.kaiser_beta)


def _kernel(scene, u):
    s = 1.0 if u == 0 else math.sin(math.pi * u) / (math.pi * u)
    return _window(scene, u) * s


def synthesize(scene, x, n_out, mic_index=0):
    """y[n] = sum over images with |n|_1 <= K of beta/(4 pi d) * windowed-sinc
    interpolation of x at n - d fs / c, d linearly interpolated between knots.
    `scene` is a workload scene description (tiers given as knot rates in Hz)."""
    dims = scene.dims
    mic = [float(v) for v in scene.mics[mic_index]]
    tiers = [(t[0], int(round(scene.fs / t[1])), int(t[2]) if len(t) > 2 else 1) for t in scene.tiers]
    Q = getattr(scene, "up_halfwidth", 4)
    imgs = []
    for sign, off, hits in mirror_images(dims, 2 * scene.K + 3):
        n, _ = lattice_of(sign, off, dims)
        if sum(abs(v) for v in n) > scene.K:
            continue
        beta = 1.0
        for w in range(6):
            beta *= scene.beta[w] ** hits[w]
        rho = sum(hits)
        step, up = tiers[-1][1], tiers[-1][2]
        for max_rho, st, u in tiers:
            if rho <= max_rho:
                step, up = st, u
                break
        imgs.append((sign, off, beta, step, up))

    def dist_at(sign, off, te, m):
        q = source(scene, te)
        return math.sqrt(sum((sign[d] * q[d] + off[d] - m[d]) ** 2 for d in range(3)))

    def dist(sign, off, t):
        m = mic_at(scene, mic, t)
        if getattr(scene, "delay_model", 0) != 1:
            return dist_at(sign, off, t, m)
        # emission-time path length: c tau = |r(t - tau) - m(t)|, by bisection
        # (c tau - |r(t - tau) - m| increases with tau below the speed of sound)
        lo, hi = 0.0, 1.0
        while scene.c * hi - dist_at(sign, off, t - hi, m) < 0.0:
            hi *= 2.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if scene.c * mid - dist_at(sign, off, t - mid, m) < 0.0:
                lo = mid
            else:
                hi = mid
            if hi - lo <= 1e-17:
                break
        return scene.c * 0.5 * (lo + hi)

    def kaiser8(u):
        z = max(0.0, 1.0 - (u / Q) ** 2)
        return _bessel_i0(8.0 * math.sqrt(z)) / _bessel_i0(8.0)

    memo = {}

    def point(sign, off, step, up, k):
        # distance at interpolation point k (sample k * step / up), memoised
        key = (sign, off, step, up, k)
        if key not in memo:
            memo[key] = point_eval(sign, off, step, up, k)
        return memo[key]

    def point_eval(sign, off, step, up, k):
        if up == 1:
            return dist(sign, off, k * step / scene.fs)
        j0 = math.floor(k / up)
        x = k / up
        ws, acc = 0.0, 0.0
        for j in range(j0 - Q + 1, j0 + Q + 1):
            u = x - j
            h = (1.0 if u == 0 else math.sin(math.pi * u) / (math.pi * u)) * kaiser8(u)
            ws += h
            acc += h * dist(sign, off, j * step / scene.fs)
        return acc / ws

    half = scene.taps // 2
    y = []
    for n in range(n_out):
        acc = 0.0
        for sign, off, beta, step, up in imgs:
            sp = step // up
            k0 = n // sp
            frac = (n - k0 * sp) / sp
            d0 = point(sign, off, step, up, k0)
            d1 = point(sign, off, step, up, k0 + 1)
            d = d0 + frac * (d1 - d0)
            t = n - d * scene.fs / scene.c
            m0 = math.floor(t)
            e = 0.0
            for k in range(-half, half):
                m = m0 - k
                if 0 <= m < len(x):
                    e += _kernel(scene, t - m) * x[m]
            acc += beta / (4.0 * math.pi * d) * e
        y.append(acc)
    return y
