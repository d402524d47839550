"""Handle wrapper over the C ABI for torch tensors.

PyTorch provides the device memory and the stream; every step runs in the
CUDA library through ``capi``.
"""
from __future__ import annotations

import torch

from . import capi

_DT = {torch.float32: capi.F32, torch.float64: capi.F64}


class Mpdata:
    """One handle of the library: n_fields fields of one dimensionality.

    shapes: a shape tuple (one field) or a list of shape tuples (a batch of
    fields held concatenated, field after field).  The handle's stream is the
    current torch stream of `device` at construction unless one is given.
    """

    def __init__(self, shapes, dtype=torch.float32, n_iters=2, opts=0, device=None, stream=None):
        if isinstance(shapes, (tuple, torch.Size)) and all(isinstance(s, int) for s in shapes):
            shapes = [tuple(shapes)]
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        self.ndims = len(self.shapes[0])
        if any(len(s) != self.ndims for s in self.shapes):
            raise ValueError("all fields of a handle have the same number of dimensions")
        if dtype not in _DT:
            raise ValueError("dtype must be torch.float32 or torch.float64")
        self.dtype = dtype
        self.n_iters = int(n_iters)
        self.opts = int(opts)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.h = capi.mpdata_create(self.ndims, self.shapes, _DT[dtype], self.n_iters, self.opts, self.stream)
        self.sizes = [int(torch.Size(s).numel()) for s in self.shapes]
        self.total = sum(self.sizes)

    # -- stepping -----------------------------------------------------------------
    def step(self, psi, gc, g=None, r=None, dt=0.0, n_steps=1):
        """Advance psi in place by n_steps steps."""
        capi.mpdata_step(self.h, psi, gc, g, r, dt, n_steps)
        return psi

    def advance(self, psi_in, psi_out, gc, g=None, r=None, dt=0.0, n_steps=1, gc_scale=None):
        capi.mpdata_advance(self.h, psi_in, psi_out, gc, g, r, dt, n_steps, gc_scale)
        return psi_out

    def advance_compensated(self, psi_in, lo_in, psi_out, lo_out, gc, g=None, r=None, dt=0.0, n_steps=1,
                            gc_scale=None):
        """advance() on the compensated FP32 state psi = hi + lo (FP32 handles, one 2D field,
        n_iters = 2): hi in psi_*, lo in lo_*; returns (psi_out, lo_out)."""
        capi.mpdata_advance_compensated(self.h, psi_in, lo_in, psi_out, lo_out, gc, g, r, dt, n_steps, gc_scale)
        return psi_out, lo_out

    def adjoint_step(self, psi_n, gc, psi_bar, g=None, gc_bar=None, r=None, dt=0.0, r_bar=None):
        """psi_bar (in place): dL/dpsi^{n+1} -> dL/dpsi^n; gc_bar[d] += dL/dgc_d.  Handles with an
        Euler source pass the step's source r and dt (and r_bar += dL/dR if given)."""
        if r is not None:
            capi.mpdata_adjoint_step_rhs(self.h, psi_n, gc, g, r, dt, psi_bar, gc_bar, r_bar)
        else:
            capi.mpdata_adjoint_step(self.h, psi_n, gc, g, psi_bar, gc_bar)
        return psi_bar

    def tape_numel(self):
        """Elements of this handle's dtype in one step's adjoint tape."""
        esize = 4 if self.dtype == torch.float32 else 8
        return capi.mpdata_adjoint_tape_bytes(self.h) // esize

    def adjoint_record(self, psi_n, gc, tape, psi_next=None, g=None):
        """Forward step psi_n -> psi_next (if given) keeping its tape for adjoint_replay."""
        capi.mpdata_adjoint_record(self.h, psi_n, gc, g, tape, psi_next)

    def adjoint_replay(self, psi_n, gc, tape, psi_bar, g=None, gc_bar=None):
        """adjoint_step from a recorded tape (psi_n and gc as at recording)."""
        capi.mpdata_adjoint_replay(self.h, psi_n, gc, g, tape, psi_bar, gc_bar)
        return psi_bar

    def set_rhs_linear(self, A, b=None):
        """Sources R = A psi + b of the trapezoidal scheme (handles created with RHS_TRAPEZ): the
        handle's fields are the system's equations; b (a tensor of the handle's total size, or
        None) is read at every step and must stay alive."""
        self._rhs_b = b
        capi.mpdata_set_rhs_linear(self.h, A, b)

    def sw_advance(self, state, dt, dx, eps=1e-8, n_steps=1):
        """Shallow-water system (handles created with SW): state = [h, q_0, ..] concatenated,
        advanced in place; the handle keeps the previous step's velocities for the next call."""
        capi.mpdata_sw_advance(self.h, state, dt, dx, eps, n_steps)
        return state

    def sw_reset(self):
        """The next sw_advance step starts a new run (no previous velocities)."""
        capi.mpdata_sw_reset(self.h)

    def set_stream(self, stream):
        """Send later work of the handle to `stream` (a torch.cuda.Stream)."""
        capi.mpdata_set_stream(self.h, stream)
        self.stream = stream

    def capture(self, psi_in, psi_out, gc, n_steps, g=None, r=None, dt=0.0, gc_scale=None):
        """Capture `n_steps` steps (psi_in -> psi_out) into a torch.cuda.CUDAGraph; replaying
        the graph re-runs them with whatever the captured buffers hold at that time.  One
        un-captured step is run first so that every one-time set-up happens outside the capture."""
        prev = self.stream
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        self.set_stream(side)
        try:
            scratch = torch.empty_like(psi_out)
            with torch.cuda.stream(side):
                self.advance(psi_in, scratch, gc, g, r, dt, 1)
            side.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=side):
                self.advance(psi_in, psi_out, gc, g, r, dt, n_steps, gc_scale)
        finally:
            self.set_stream(prev)
        return graph

    # -- FP64 reductions --------------------------------------------------------------
    def mass(self, psi, g=None):
        m = capi.mpdata_reduce(self.h, psi, g, len(self.shapes))
        return m if len(m) > 1 else m[0]

    def diff_norms(self, a, b):
        l2, li = capi.mpdata_diff_norms(self.h, a, b, len(self.shapes))
        return (l2, li) if len(l2) > 1 else (l2[0], li[0])

    def check_courant(self, gc, g=None):
        return capi.mpdata_check_courant(self.h, gc, g)

    def tune(self, knob, value):
        capi.mpdata_tune(self.h, knob, value)

    def request_stop(self):
        capi.mpdata_request_stop(self.h)

    def clear_stop(self):
        capi.mpdata_clear_stop(self.h)

    def sync(self):
        capi.mpdata_sync(self.h)

    def close(self):
        if getattr(self, "h", None):
            capi.mpdata_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
