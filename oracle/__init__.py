"""MPDATA oracle -- test infrastructure only.

A plain FP64 CPU implementation of one MPDATA time step (libmpdata++ 0.1 paper,
Sect. 3.1 and 4.1), with its tangent-linear and adjoint, written in C++
(``mpdata_oracle.cpp``) and loaded through ctypes.  Only the tests, the
package smoke check and the benchmark's CPU-baseline leg use this module; the
CUDA library never imports, links or calls it.

Parity status per function (details in the header of ``mpdata_oracle.cpp``):
every sub-step is pinned by the tests in ``tests/test_oracle_pins.py`` (open edges
in ``tests/test_oracle_open.py``), except
the multi-dimensional cross terms of the third-order option, which are pinned
only by the convergence order on a diagonal flow.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mpdata_oracle.cpp")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "libmpdata_oracle.so")

# option bits, same values as the library interface (the oracle defines its own)
FCT, TOT, IGA, NUG, KAHAN, RHS_EULER_A, RHS_EULER_B = 1, 2, 4, 8, 16, 32, 64
ABS = 256  # |psi| in the psi-fractions of the pseudo-velocity (variable-sign fields)
DFL = 512  # divergent-flow term of the pseudo-velocity
OPEN0, OPEN1, OPEN2 = 1024, 2048, 4096  # open edges along dimension 0, 1, 2 (else periodic)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (host C++ only, no CUDA)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-shared", "-fPIC", SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i64, i32, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint
            dbl = ctypes.c_double
            lib.mpo_step_ex.argtypes = [i32, d, d, d, d, d, d, d, dbl, i32, u32, i64, d, d]
            lib.mpo_step_ex.restype = i32
            lib.mpo_tl_step.argtypes = [i32, d, d, d, d, d, d, d, dbl, i32, u32, d, d, d, d, d]
            lib.mpo_tl_step.restype = i32
            lib.mpo_adj_step.argtypes = [i32, d, d, d, d, d, d, d, dbl, i32, u32, d, d, d, d]
            lib.mpo_adj_step.restype = i32
            lib.mpo_mass.argtypes = [i32, d, d, d]
            lib.mpo_mass.restype = dbl
            lib.mpo_set_threads.argtypes = [i32]
            lib.mpo_set_threads.restype = i32
            _lib = lib
    return _lib


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prep(psi, gc, g, r):
    psi = _f64(psi)
    nd = psi.ndim
    if len(gc) != nd:
        raise ValueError("need one advector component per dimension")
    gc = [_f64(v) for v in gc]
    for v in gc:
        if v.shape != psi.shape:
            raise ValueError("advector components must have the field's shape")
    g, r = _f64(g), _f64(r)
    shape = np.array(psi.shape, dtype=np.int64)
    gcp = [_ptr(v) for v in gc] + [None] * (3 - nd)
    return psi, nd, shape, gc, gcp, g, r


def _opts(opts, g, r, rhs):
    o = int(opts)
    if g is not None:
        o |= NUG
    if r is not None:
        o |= RHS_EULER_B if rhs == "euler_b" else RHS_EULER_A
    return o


def step(psi, gc, g=None, r=None, dt=0.0, n_iters=2, opts=0, n_steps=1,
         rhs="euler_a", return_bounds=False):
    """Advance psi by n_steps MPDATA steps; returns the new field (a copy).

    gc: sequence of advector components (G times Courant number), one per
    dimension, each with psi's shape; component d at index i sits on the face
    between cell i and cell i + e_d (periodic).  g: G field or None (G = 1).
    r: source term or None; rhs selects 'euler_a' or 'euler_b' (Sect. 4.1).
    """
    psi, nd, shape, gc, gcp, g, r = _prep(psi, gc, g, r)
    out = psi.copy()
    mx = np.zeros_like(out) if return_bounds else None
    mn = np.zeros_like(out) if return_bounds else None
    rc = _load().mpo_step_ex(nd, _ptr(shape), _ptr(out), *gcp, _ptr(g), _ptr(r), float(dt),
                             int(n_iters), _opts(opts, g, r, rhs), int(n_steps), _ptr(mx), _ptr(mn))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return (out, mx, mn) if return_bounds else out


def tl_step(psi, gc, dpsi, dgc, g=None, r=None, dt=0.0, n_iters=2, opts=0, rhs="euler_a"):
    """Tangent-linear of one step at (psi, gc) applied to (dpsi, dgc)."""
    psi, nd, shape, gc, gcp, g, r = _prep(psi, gc, g, r)
    dpsi = _f64(dpsi)
    dgc = [None if v is None else _f64(v) for v in dgc] + [None] * (3 - nd)
    out = np.zeros_like(psi)
    rc = _load().mpo_tl_step(nd, _ptr(shape), _ptr(psi), *gcp, _ptr(g), _ptr(r), float(dt),
                             int(n_iters), _opts(opts, g, r, rhs), _ptr(dpsi),
                             *[_ptr(v) for v in dgc], _ptr(out))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return out


def adj_step(psi, gc, psi_bar, g=None, r=None, dt=0.0, n_iters=2, opts=0, rhs="euler_a"):
    """Adjoint of one step at (psi, gc): returns (dL/dpsi^n, [dL/dgc_d])."""
    psi, nd, shape, gc, gcp, g, r = _prep(psi, gc, g, r)
    pb = _f64(psi_bar).copy()
    gcb = [np.zeros_like(psi) for _ in range(nd)]
    ptrs = [_ptr(v) for v in gcb] + [None] * (3 - nd)
    rc = _load().mpo_adj_step(nd, _ptr(shape), _ptr(psi), *gcp, _ptr(g), _ptr(r), float(dt),
                              int(n_iters), _opts(opts, g, r, rhs), _ptr(pb), *ptrs)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return pb, gcb


def mass(psi, g=None):
    """Sum of G * psi in FP64 (G = 1 when g is None)."""
    psi = _f64(psi)
    g = _f64(g)
    shape = np.array(psi.shape, dtype=np.int64)
    return float(_load().mpo_mass(psi.ndim, _ptr(shape), _ptr(psi), _ptr(g)))


def set_threads(n: int) -> int:
    """Set the OpenMP thread count of the forward sweeps; returns the count in use."""
    return int(_load().mpo_set_threads(int(n)))


def step_trapez(psis, gcs, A, b=None, dt=1.0, n_iters=2, opts=0, n_steps=1, g=None):
    """Trapezoidal source scheme (Sect. 4.1, Eq. trapez) for a system of E equations on one grid
    whose sources are affine in the state, R_e = sum_f A[e, f] psi_f + b_e:

        psi^{n+1} = ADV(psi^n + dt/2 R^n) + dt/2 R^{n+1}.

    R^{n+1} = A psi^{n+1} + b makes the second half implicit: per cell the E x E system
    (I - dt/2 A) psi^{n+1} = psi* + dt/2 b is solved (numpy.linalg.solve), psi* = ADV(...)
    being one step of the advection of each equation (step(), no source bits).  For the
    translating oscillator of Sect. 4.2 this is the closed form given there.
    psis: E arrays of one shape; gcs: the advector components (one list for all equations, or
    one list per equation); b: None or E arrays.  Returns the E new arrays."""
    state = [np.array(p, dtype=np.float64) for p in psis]
    E = len(state)
    A = np.asarray(A, dtype=np.float64).reshape(E, E)
    per_eq = isinstance(gcs[0], (list, tuple))
    bb = [np.zeros_like(state[0]) if b is None else np.asarray(b[e], dtype=np.float64) for e in range(E)]
    M = np.eye(E) - 0.5 * dt * A
    for _ in range(int(n_steps)):
        R = [sum(A[e, f] * state[f] for f in range(E)) + bb[e] for e in range(E)]
        pre = [state[e] + 0.5 * dt * R[e] for e in range(E)]
        star = [step(pre[e], gcs[e] if per_eq else gcs, g=g, n_iters=n_iters, opts=opts) for e in range(E)]
        rhs = np.stack([(star[e] + 0.5 * dt * bb[e]).ravel() for e in range(E)])
        new = np.linalg.solve(M, rhs)
        state = [new[e].reshape(state[0].shape) for e in range(E)]
    return state


def vip_advector(h, qs, u_prev, dt, dx, eps=1e-8, opened=()):
    """Prognosed-velocity advector (Sect. 5.1-5.2): velocities u_d = q_d / h where h > eps (else 0)
    at the cell centres, extrapolated linearly in time to n + 1/2 (1.5 u^n - 0.5 u^{n-1}; u^{n-1} =
    u^n at the first step, u_prev None), interpolated linearly to the cell walls and turned into
    Courant numbers (times dt / dx).  Face i+1/2 along d sits at index i (between cells i and
    i+e_d); along an open dimension the last entry is not an interior face (copied there from the
    last interior face, never read by the step).  Returns (advector components, u^n)."""
    u = [np.where(h > eps, q / np.where(h > eps, h, 1.0), 0.0) for q in qs]
    prev = u if u_prev is None else u_prev
    gc = []
    for d, (un, up) in enumerate(zip(u, prev)):
        ue = 1.5 * un - 0.5 * up
        right = np.roll(ue, -1, axis=d)
        c = 0.5 * (ue + right) * (dt / dx)
        if d in opened:
            idx = [slice(None)] * ue.ndim
            idx[d] = -1
            src = [slice(None)] * ue.ndim
            src[d] = -2
            c[tuple(idx)] = c[tuple(src)]
        gc.append(c)
    return gc, u


def sw_forcing(h, dx, opened=()):
    """Shallow-water momentum sources of Sect. 5.3-5.4, R_d = -h dh/dx_d (g = 1), the gradient a
    centred difference (h_{i+e_d} - h_{i-e_d}) / (2 dx); beyond an open edge h is the edge value."""
    out = []
    for d in range(h.ndim):
        hp, hm = np.roll(h, -1, axis=d), np.roll(h, 1, axis=d)
        if d in opened:
            first = [slice(None)] * h.ndim
            first[d] = 0
            last = [slice(None)] * h.ndim
            last[d] = -1
            hm[tuple(first)] = h[tuple(first)]
            hp[tuple(last)] = h[tuple(last)]
        out.append(-h * (hp - hm) / (2.0 * dx))
    return out


def step_shallow_water(h, qs, dt, dx, n_iters=2, opts=0, n_steps=1, eps=1e-8, u_prev=None):
    """Shallow-water system with prognosed velocity (Sect. 5): h_t + div(u h) = 0,
    (q_d)_t + div(u q_d) = -h dh/dx_d with q_d = u_d h, advanced by the trapezoidal scheme of
    Sect. 4.1 (Eq. trapez), whose second half is explicit here because h has no source (the
    footnote of Sect. 5.3): per step the advector at n + 1/2 comes from vip_advector, the momenta
    get dt/2 R^n, h and the momenta are advected by one MPDATA step each (step(), the given
    options, G = 1), and the momenta get dt/2 R^{n+1} from the new h.  Open edges as the OPEN
    bits of opts say.  Returns (h, [q_d], u^n of the last step) for continuing a run."""
    h = np.array(h, dtype=np.float64)
    qs = [np.array(q, dtype=np.float64) for q in qs]
    opened = tuple(d for d in range(h.ndim) if int(opts) & (OPEN0 << d))
    for _ in range(int(n_steps)):
        gc, u_prev = vip_advector(h, qs, u_prev, dt, dx, eps, opened)
        R = sw_forcing(h, dx, opened)
        qs = [q + 0.5 * dt * r for q, r in zip(qs, R)]
        h = step(h, gc, n_iters=n_iters, opts=opts)
        qs = [step(q, gc, n_iters=n_iters, opts=opts) for q in qs]
        R = sw_forcing(h, dx, opened)
        qs = [q + 0.5 * dt * r for q, r in zip(qs, R)]
    return h, qs, u_prev
