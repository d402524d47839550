"""Seeded synthetic inputs shaped like the paper's advection tests.

This module only generates fields (initial conditions, discretely
nondivergent advectors, G factors); it contains none of MPDATA's arithmetic,
imports nothing else from this package, and serves the CUDA path, the oracle
tests and the benchmark alike.  All arrays are float64 numpy arrays in the
library's layout: row-major, last dimension fastest, advector component d at
index i on the face between cell i and cell i + e_d (periodic).

Discrete nondivergence: 2D advectors are differences of a streamfunction held
at cell corners, 3D advectors are discrete curls of a vector potential held on
cell edges, so every cell's net flux telescopes to zero.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "hello_1d", "rotation_2d", "rotation_steps", "deformational_3d", "deformational_scale",
    "ensemble_2d", "adjoint_2d", "gaussian_1d_cell_means", "low_modes", "streamfunction_advector",
    "agnesi_1d", "oscillator_1d",
]


def hello_1d(n=500, courant=0.5):
    """1D periodic test: box of height 1 on cells 50..100 (inclusive) over 0, plus a
    Gaussian of peak 1 and sigma 15 cells centred on cell 300; constant Courant number."""
    x = np.arange(n, dtype=np.float64)
    psi = np.zeros(n)
    psi[50:101] = 1.0
    psi += np.exp(-0.5 * ((x - 300.0) / 15.0) ** 2)
    return psi, [np.full(n, float(courant))]


def agnesi_1d(n=101, dx=0.1, a=0.5, courant=0.5):
    """The "hello world" of Sect. 3.3: n data points dx apart (the outermost ones on the domain
    edges, which are open), a variable-sign Witch of Agnesi 8 a^3 / (x^2 + 4 a^2) centred in the
    domain and shifted down by 0.5, constant Courant number.  Returns psi, [gc]; with open
    edges the last advector entry is not an interior face and is not read."""
    x = np.arange(n, dtype=np.float64) * dx
    xc = 0.5 * (n - 1) * dx
    psi = 8.0 * a ** 3 / ((x - xc) ** 2 + 4.0 * a ** 2) - 0.5
    return psi, [np.full(n, float(courant))]


def oscillator_1d(n=1000, courant=0.5, dt=1.0, period=1400.0):
    """Translating harmonic oscillator of Sect. 4.2: psi_t + (u psi)_x = omega phi,
    phi_t + (u phi)_x = -omega psi, on n cells of 1 m (periodic), u = courant m/s, time step
    dt s.  psi(x) = 0.5 (1 + cos(2 pi x / 100)) for 50 < x < 150 (cell centres), else 0; phi = 0.
    The paper gives the initial condition and the 1400 s of simulated time, not omega, the grid or
    the step; here omega = 2 pi / period.  Returns psi, phi, [gc], omega."""
    x = np.arange(n, dtype=np.float64) + 0.5
    psi = np.where((x > 50.0) & (x < 150.0), 0.5 * (1.0 + np.cos(2.0 * math.pi * x / 100.0)), 0.0)
    return psi, np.zeros(n), [np.full(n, float(courant))], 2.0 * math.pi / period


def rotation_steps(n):
    """Steps per revolution so that |C| = 0.5 at distance n/2 from the centre."""
    return int(math.ceil(2.0 * math.pi * (n / 2.0) / 0.5))


def rotation_2d(n=1024, steps_per_rev=None):
    """Solid-body rotation of a cone (rotating-cone example, Sect. 3.6, scaled to n^2).

    Streamfunction phi = omega*dt*r^2/2 on cell corners around the domain centre,
    face fluxes are its differences.  Cone radius 0.15 n, height 4 on background 1,
    centred at (n/2, n/2 + n/4) in cell-centre coordinates, profile
    h (1 - d^2/R^2)^2 as in the paper's rotating-cone listing.
    Returns psi, [gc0, gc1], steps per revolution."""
    if steps_per_rev is None:
        steps_per_rev = rotation_steps(n)
    w = 2.0 * math.pi / steps_per_rev  # omega * dt
    c = n / 2.0
    i = np.arange(n, dtype=np.float64)
    # face of dim 0 at (i, j): x = i + 1, spanning y in [j, j+1]
    gc0 = np.broadcast_to((w * (i + 0.5 - c))[None, :], (n, n)).copy()
    gc1 = np.broadcast_to((-w * (i + 0.5 - c))[:, None], (n, n)).copy()
    xc, yc = (i + 0.5)[:, None], (i + 0.5)[None, :]
    R = 0.15 * n
    d2 = (xc - c) ** 2 + (yc - (c + 0.25 * n)) ** 2
    psi = 1.0 + np.where(d2 <= R * R, 4.0 * (1.0 - d2 / (R * R)) ** 2, 0.0)
    return psi, [gc0, gc1], steps_per_rev


def low_modes(rng, shape, n_modes, kmax=3, amplitude=1.0):
    """Sum of n_modes seeded periodic Fourier modes cos(2 pi k.x + phase), 1 <= |k|_inf <= kmax,
    sampled at cell centres of a unit periodic box."""
    nd = len(shape)
    grids = np.meshgrid(*[(np.arange(s) + 0.5) / s for s in shape], indexing="ij")
    f = np.zeros(shape)
    for _ in range(n_modes):
        while True:
            k = rng.integers(-kmax, kmax + 1, size=nd)
            if np.any(k != 0):
                break
        ph = rng.uniform(0, 2 * math.pi)
        a = rng.normal()
        f += amplitude * a * np.cos(2 * math.pi * sum(k[d] * grids[d] for d in range(nd)) + ph)
    return f


def streamfunction_advector(phi, max_courant):
    """Discretely nondivergent periodic 2D advector from a corner streamfunction.

    phi[a, b] is the streamfunction at the corner (a, b) shared by cells (a-1..a, b-1..b);
    gc0[i, j] = phi[i+1, j+1] - phi[i+1, j],  gc1[i, j] = -(phi[i+1, j+1] - phi[i, j+1]),
    then both are scaled so that max |C| = max_courant."""
    p = np.roll(np.roll(phi, -1, 0), -1, 1)           # phi[i+1, j+1]
    gc0 = p - np.roll(phi, -1, 0)                      # - phi[i+1, j]
    gc1 = -(p - np.roll(phi, -1, 1))                   # - phi[i, j+1]
    s = max_courant / max(np.abs(gc0).max(), np.abs(gc1).max())
    return [gc0 * s, gc1 * s]


def ensemble_2d(n_fields=512, seed=0, sizes=tuple(range(64, 513, 32)), max_courant=0.5):
    """Batched ensemble: n_fields independent periodic 2D fields with side lengths drawn
    uniformly from `sizes`, each with its own streamfunction advector (6 low modes,
    max |C| = max_courant) and psi = 1 + Gaussian (sigma ~ U[0.05, 0.15] * n).
    Returns a list of (psi, [gc0, gc1])."""
    rng = np.random.default_rng(seed)
    out = []
    ns = rng.choice(np.asarray(sizes), size=n_fields)
    for n in ns:
        n = int(n)
        phi = low_modes(rng, (n, n), 6)
        gc = streamfunction_advector(phi, max_courant)
        sig = rng.uniform(0.05, 0.15) * n
        cx, cy = rng.uniform(0, n, size=2)
        x = np.arange(n) + 0.5
        dx = np.minimum(np.abs(x - cx), n - np.abs(x - cx))[:, None]
        dy = np.minimum(np.abs(x - cy), n - np.abs(x - cy))[None, :]
        psi = 1.0 + np.exp(-0.5 * (dx ** 2 + dy ** 2) / sig ** 2)
        out.append((psi, gc))
    return out


def adjoint_2d(n=512, seed=0, max_courant=0.5):
    """Adjoint test inputs: psi0 = 2 + 6 low modes (amplitude 0.5, strictly positive, no
    flat regions), a streamfunction advector (max |C| = max_courant) and a smooth seeded
    perturbation used to build the target state.  Returns psi0, [gc0, gc1], perturbation."""
    rng = np.random.default_rng(seed)
    f = low_modes(rng, (n, n), 6)
    psi0 = 2.0 + 0.5 * f / np.abs(f).max()
    gc = streamfunction_advector(low_modes(rng, (n, n), 6), max_courant)
    pert = low_modes(rng, (n, n), 6)
    pert /= np.sqrt(np.mean(pert ** 2))
    return psi0, gc, pert


# ---------------------------------------------------------------- 3D deformational flow

def _edge_integrals(n):
    """Exact edge integrals of the vector potential A = (0, -s2, s1) on a unit periodic cube,
    s1 = sin^2(pi x) sin^2(pi y) sin(2 pi z) / pi, s2 = sin^2(pi x) sin(2 pi y) sin^2(pi z) / pi.

    Ez[a, b, k] = int over z in [k h, (k+1) h] of A_z at corner line (a h, b h)
    Ey[a, j, c] = int over y in [j h, (j+1) h] of A_y at corner line (a h, c h)"""
    h = 1.0 / n
    t = np.arange(n) * h                  # corner coordinates
    s2x = np.sin(math.pi * t) ** 2
    # int sin(2 pi z) dz over [kh, (k+1)h] = (cos(2 pi kh) - cos(2 pi (k+1)h)) / (2 pi)
    i_sin2 = (np.cos(2 * math.pi * t) - np.cos(2 * math.pi * (t + h))) / (2 * math.pi)
    s2y = s2x
    s2z = s2x
    Ez = (s2x[:, None, None] * s2y[None, :, None] * i_sin2[None, None, :]) / math.pi
    Ey = -(s2x[:, None, None] * i_sin2[None, :, None] * s2z[None, None, :]) / math.pi
    return Ez, Ey


def deformational_3d(n=256, seed=0, max_courant=0.4, iga=False):
    """3D deformational flow on a unit periodic cube (n^3 cells).

    Advector: discrete curl of the edge-integrated vector potential above
    (u = 2 sin^2(pi x) sin(2 pi y) sin(2 pi z), v = -sin(2 pi x) sin^2(pi y) sin(2 pi z),
    w = -sin(2 pi x) sin(2 pi y) sin^2(pi z)), scaled to max |C| = max_courant.
    G = 1 + 0.2 f / max|f| with f 8 seeded low modes; the advector is the mass flux
    G*C itself, so it stays discretely nondivergent.  psi: two seeded overlapping
    Gaussians (sigma ~ 0.08, peak 1, background 0), or +1 and -1 blobs with iga=True.
    The advector is multiplied by cos(pi t / T) at t = (step + 1/2) dt
    (deformational_scale).  Returns psi, [gc0, gc1, gc2], G."""
    rng = np.random.default_rng(seed)
    amp = rng.uniform(0.5, 1.5)
    Ez, Ey = _edge_integrals(n)
    roll = np.roll
    # flux_x(i,j,k) at x=(i+1)h: Ez(i+1, j+1, k) - Ez(i+1, j, k) - (Ey(i+1, j, k+1) - Ey(i+1, j, k))
    Ez1 = roll(Ez, -1, 0)
    Ey1 = roll(Ey, -1, 0)
    fx = (roll(Ez1, -1, 1) - Ez1) - (roll(Ey1, -1, 2) - Ey1)
    # flux_y(i,j,k) at y=(j+1)h: -(Ez(i+1, j+1, k) - Ez(i, j+1, k))
    Ezj = roll(Ez, -1, 1)
    fy = -(roll(Ezj, -1, 0) - Ezj)
    # flux_z(i,j,k) at z=(k+1)h: Ey(i+1, j, k+1) - Ey(i, j, k+1)
    Eyk = roll(Ey, -1, 2)
    fz = roll(Eyk, -1, 0) - Eyk
    s = amp * max_courant / (amp * max(np.abs(fx).max(), np.abs(fy).max(), np.abs(fz).max()))
    gc = [fx * s, fy * s, fz * s]
    f = low_modes(rng, (n, n, n), 8)
    G = 1.0 + 0.2 * f / np.abs(f).max()
    x = (np.arange(n) + 0.5) / n
    psi = np.zeros((n, n, n))
    signs = (1.0, -1.0) if iga else (1.0, 1.0)
    for sgn in signs:
        c = rng.uniform(0.35, 0.65, size=3)
        sig = 0.08 * rng.uniform(0.9, 1.1)
        d = [np.minimum(np.abs(x - c[a]), 1 - np.abs(x - c[a])) for a in range(3)]
        r2 = d[0][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[2][None, None, :] ** 2
        psi += sgn * np.exp(-0.5 * r2 / sig ** 2)
    return psi, gc, G


def deformational_scale(step, period_steps=1280):
    """Time factor cos(pi t / T) of the deformational advector at t = (step + 1/2) dt."""
    return math.cos(math.pi * (step + 0.5) / period_steps)


def gaussian_1d_cell_means(n_cells, dx, x0, sigma):
    """Cell means of the normalised Gaussian of Eq. 7 on cells [i dx, (i+1) dx],
    obtained by integrating the Gaussian analytically over each cell."""
    edges = np.arange(n_cells + 1) * dx
    cdf = 0.5 * (1.0 + np.vectorize(math.erf)((edges - x0) / (sigma * math.sqrt(2.0))))
    return np.diff(cdf) / dx
