"""Seeded test inputs shared by the oracle pins and the GPU parity tests (no MPDATA arithmetic)."""
import numpy as np

from paper_1407_1309_gb300 import workloads as wl


def nondivergent(shape, rng, cmax):
    """Random discretely nondivergent periodic advector (constant in 1D, corner
    streamfunction differences in 2D, discrete curl of an edge potential in 3D)."""
    nd = len(shape)
    if nd == 1:
        return [np.full(shape, rng.uniform(-cmax, cmax))]
    if nd == 2:
        return wl.streamfunction_advector(rng.normal(size=shape), cmax)
    # Ax[i, b, c] is the x-edge from corner (i, b, c) to (i+1, b, c), likewise Ay[a, j, c], Az[a, b, k]
    Ax, Ay, Az = (rng.normal(size=shape) for _ in range(3))
    up = lambda a, d: np.roll(a, -1, axis=d)
    fx = (up(up(Az, 0), 1) - up(Az, 0)) - (up(up(Ay, 0), 2) - up(Ay, 0))
    fy = (up(up(Ax, 1), 2) - up(Ax, 1)) - (up(up(Az, 0), 1) - up(Az, 1))
    fz = (up(up(Ay, 0), 2) - up(Ay, 2)) - (up(up(Ax, 1), 2) - up(Ax, 2))
    s = cmax / max(np.abs(fx).max(), np.abs(fy).max(), np.abs(fz).max())
    return [fx * s, fy * s, fz * s]


def divergence(gc):
    return sum(v - np.roll(v, 1, d) for d, v in enumerate(gc))


def smooth_positive(shape, rng, n_modes=6):
    """2 + 0.5 * (normalised seeded low modes): strictly positive, no flat regions."""
    f = wl.low_modes(rng, shape, n_modes)
    return 2.0 + 0.5 * f / np.abs(f).max()


def boxes(shape, rng, lo=1.0, hi=4.0, frac=0.3):
    return np.where(rng.uniform(size=shape) < frac, hi, lo)
