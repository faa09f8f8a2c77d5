"""Seeded synthetic workloads (problem parameters only, no solver arithmetic).

The paper's convergence studies use a Gaussian beam in the unit cube (Sec. 4,
"Problem Setup") and its application a layered high-contrast seismic model
driven by a tight Gaussian point source (Sec. 5).  Neither the beam data nor
the seismic model is available, so these generators produce inputs of the
same shape: unit-cube Gaussian sources, and a box with horizontally layered
piecewise-constant wavespeed and a point-like Gaussian source.

Random draws use SplitMix64 in counter form, u_k = (out_k >> 11) 2^-53,
out_k = mix(seed + (k+1) 0x9E3779B97F4A7C15).
"""
import math

_G = 0x9E3779B97F4A7C15
_M = (1 << 64) - 1


def _u(seed, k):
    z = (seed + (k + 1) * _G) & _M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M
    z ^= z >> 31
    return (z >> 11) * (1.0 / 9007199254740992.0)


def rademacher_rows(seed, j0, j1, n):
    """Rows j0 .. j1-1 of a seeded n-column sign matrix (entries +-1.0): entry
    (j, i) is the sign bit of SplitMix64 output k = j n + i (counter form, as
    _u; vectorised with wrapping uint64 arithmetic).  Used to sketch long
    vectors (random projections) in tests."""
    import numpy as np
    k = (np.arange(j0 * n, j1 * n, dtype=np.uint64) + np.uint64(1))
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + k * np.uint64(_G)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return np.where((z >> np.uint64(63)) == 1, -1.0, 1.0).reshape(j1 - j0, n)


def config1():
    """4^3 hexes, p = 2, omega = 4, c = 1, Gaussian at the cube centre, 2-level p-MG, FP64."""
    return dict(problem=dict(n=(4, 4, 4), p=2, omega=4.0, src_center=(0.5, 0.5, 0.5), src_width=0.1),
                opts=dict(n_levels=2, p_min=1, precision="fp64", tol=1e-8),
                name="unit cube 4^3 p=2 omega=4, 2-level p-MG, complex128")


def config2(precision="mixed"):
    """16^3 hexes, p = 3, omega = 16 pi, c = 1, seeded source in [0.3, 0.7]^3, 3 levels."""
    x0 = tuple(0.3 + 0.4 * _u(2, k) for k in range(3))
    return dict(problem=dict(n=(16, 16, 16), p=3, omega=16 * math.pi, src_center=x0, src_width=0.1),
                opts=dict(n_levels=3, p_min=2, precision=precision, tol=1e-8),
                name="unit cube 16^3 p=3 omega=16pi, 3-level h/p V(1,1), %s V-cycle" % precision)


def config3(precision="mixed"):
    """[0,2]x[0,2]x[0,1], 32x32x16 hexes, p = 3, omega = 20 pi, 6 seeded layers, 4 levels."""
    n = (32, 32, 16)
    cuts = []
    k = 0
    while len(cuts) < 5:
        v = 1 + int(15 * _u(3, k))
        k += 1
        if v not in cuts:
            cuts.append(v)
    cuts.sort()
    speeds = []
    for _ in range(6):
        speeds.append(0.1 + 0.9 * _u(3, k))
        k += 1
    x0 = (0.5 + _u(3, k), 0.5 + _u(3, k + 1), 0.25 + 0.5 * _u(3, k + 2))
    bounds = [0] + cuts + [n[2]]
    c = []
    for kz in range(n[2]):
        layer = max(i for i in range(6) if bounds[i] <= kz)
        c.extend([speeds[layer]] * (n[0] * n[1]))
    return dict(problem=dict(n=n, p=3, omega=20 * math.pi, x0=(0, 0, 0), x1=(2, 2, 1), wavespeed=c,
                             src_center=x0, src_width=0.02),
                opts=dict(n_levels=4, p_min=2, precision=precision, tol=1e-8),
                name="layered box 32x32x16 p=3 omega=20pi, 4-level, %s V-cycle" % precision,
                layers=dict(cuts=cuts, speeds=speeds))


def config3_small(precision="fp64"):
    """The layered-medium hierarchy shape at test size: [0,2]x[0,2]x[0,1],
    8x8x4 hexes, p = 3, omega = 8 pi, one seeded wavespeed per horizontal
    element layer (4 layers, U[0.1, 1], seed 33), source centre drawn in
    [0.5,1.5]^2 x [0.25,0.75] (seed 33), width 0.08; 4 levels
    p3 -> p2 -> 4x4x2 -> 2x2x1 (two stacked h-transitions)."""
    n = (8, 8, 4)
    speeds = [0.1 + 0.9 * _u(33, k) for k in range(4)]
    x0 = (0.5 + _u(33, 4), 0.5 + _u(33, 5), 0.25 + 0.5 * _u(33, 6))
    c = [speeds[kz] for kz in range(n[2]) for _ in range(n[0] * n[1])]
    return dict(problem=dict(n=n, p=3, omega=8 * math.pi, x0=(0, 0, 0), x1=(2, 2, 1), wavespeed=c,
                             src_center=x0, src_width=0.08),
                opts=dict(n_levels=4, p_min=2, precision=precision, tol=1e-8),
                name="layered box 8x8x4 p=3 omega=8pi, 4-level, %s V-cycle" % precision)


def _stream_opts(n, precision):
    return dict(n_levels=4, p_min=2 if n % 2 == 0 else 1, precision=precision, tol=1e-8, coarsest="auto")


def config4(count=64, precision="mixed"):
    """64 independent problems (seed 4): n^3 with n ~ U{8..24}, p ~ U{2,3,4},
    omega ~ U[4, 12 pi], c = 1, Gaussian source x0 ~ U[0.3, 0.7]^3, sigma 0.1.
    Hierarchy: p-coarsening to 2, then halving n while it is even, at most 4
    levels.  Odd n stops h-coarsening; there p is coarsened down to 1 instead,
    so that no such problem is left with a single level.  The options ask for
    the dense coarsest solve only where level 0 is small ("auto")."""
    out = []
    k = 0
    for _ in range(count):
        n = 8 + int(17 * _u(4, k))
        p = 2 + int(3 * _u(4, k + 1))
        om = 4.0 + (12 * math.pi - 4.0) * _u(4, k + 2)
        x0 = tuple(0.3 + 0.4 * _u(4, k + 3 + d) for d in range(3))
        k += 6
        out.append(dict(problem=dict(n=(n, n, n), p=p, omega=om, src_center=x0, src_width=0.1),
                        opts=_stream_opts(n, precision)))
    return out


def config5(count=2000, precision="mixed"):
    """Serving stream (seed 5): n^3 with n ~ U{8..48}, p ~ U{2..5},
    omega ~ U[4, 32 pi], wavespeed constant (prob. 0.5) or 4 seeded layers in
    U[0.1, 1], Gaussian source; inter-arrival times are drawn separately
    (unit-rate exponentials, scaled by the caller's rate).  Hierarchy options
    as in config4."""
    out = []
    k = 0
    for _ in range(count):
        n = 8 + int(41 * _u(5, k))
        p = 2 + int(4 * _u(5, k + 1))
        om = 4.0 + (32 * math.pi - 4.0) * _u(5, k + 2)
        x0 = tuple(0.3 + 0.4 * _u(5, k + 3 + d) for d in range(3))
        layered = _u(5, k + 6) >= 0.5
        speeds = [0.1 + 0.9 * _u(5, k + 7 + i) for i in range(4)]
        gap = -math.log(1.0 - _u(5, k + 11))
        k += 12
        pk = dict(n=(n, n, n), p=p, omega=om, src_center=x0, src_width=0.1)
        if layered:
            pk["wavespeed"] = [speeds[min(3, (4 * kz) // n)] for kz in range(n) for _ in range(n * n)]
        out.append(dict(problem=pk, opts=_stream_opts(n, precision), gap=gap))
    return out
