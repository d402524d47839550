"""Differentiable MPDATA rollouts: gradients of a final-state loss with respect to
the initial field psi0 and the advector components GC.

Forward: n_steps steps through the C ABI (fused kernels where they apply),
keeping psi every `checkpoint_every` steps on the device.  Backward: for each
segment, last first, the states inside the segment are recomputed from its
checkpoint (except for the last two segments when the backward runs on graphs with
tapes: the forward records their states and tapes itself, in the backward's own buffers,
since the backward would recompute exactly those first), then the hand-written adjoint
kernels walk the segment backwards,
accumulating dL/dGC over all steps.  When one segment's tapes fit in device
memory (`tape_budget`), the recomputation records every step's tape
(mpdata_adjoint_record: states and intermediates in one forward sweep) and the
walk back runs only the reverse sweeps (mpdata_adjoint_replay); otherwise each
step's tape is recomputed inside mpdata_adjoint_step.  Where the tape has a fused
form (2D, two passes, FCT or none, no other option) the recording runs the forward's
own fused kernel with tape stores, so the recomputed states equal the forward's bit
for bit; in the other cases they come from the staged kernels, which round
differently from the fused forward, and the gradient is that of the staged
trajectory from each checkpoint.  Memory is
one field per checkpoint plus one segment of states (and tapes).  With
use_graphs (default) the work of one segment is captured once as a CUDA graph
on static buffers and replayed per segment, so the host issues one replay per
segment instead of tens of launches per step; with tapes, the recording of the
next segment (earlier in time) runs on a second stream while the current
segment's reverse sweeps run, on two alternating buffer sets.
"""
from __future__ import annotations

import torch

from .solver import Mpdata


class MPDATAFunction(torch.autograd.Function):
    """psi_T = MPDATA^n_steps(psi0; GC).  Use as
    ``MPDATAFunction.apply(solver, n_steps, checkpoint_every, use_graphs, psi0, *gc)``."""

    @staticmethod
    def forward(ctx, solver: Mpdata, n_steps: int, checkpoint_every: int, use_graphs: bool, psi0, *gc):
        if n_steps < 1 or checkpoint_every < 1:
            raise ValueError("n_steps and checkpoint_every must be >= 1")
        cur = psi0.detach().contiguous().clone()
        nxt = torch.empty_like(cur)
        gcd = [g.detach().contiguous() for g in gc]
        ckpts = [cur.clone()]
        # the segments whose tapes this forward records for the backward (last first: buffer set
        # 0 for the last segment, 1 for the one before), when the backward will be the pipelined
        # one on graphs with tapes
        n_ck = (n_steps + checkpoint_every - 1) // checkpoint_every
        pre = {}
        if (use_graphs and any(ctx.needs_input_grad[4:]) and _fused_record(solver) and
                _tapes_fit(solver, 2 * min(checkpoint_every, n_steps), cur)):
            token = object()
            for idx, seg in enumerate(range(n_ck - 1, max(n_ck - 3, -1), -1)):
                start, end = seg * checkpoint_every, min(seg * checkpoint_every + checkpoint_every, n_steps)
                sg = _segment_graph(solver, end - start, cur, gcd, True, idx % 2)
                sg.owner = token
                pre[seg] = sg
            ctx.pre_token = token
        s = 0
        while s < n_steps:
            seg = s // checkpoint_every
            if seg in pre:  # this segment's steps by the backward's own recording graph
                sg = pre[seg]
                sg.load(gcd)
                sg.states[0].copy_(cur)
                sg.rec_graph.replay()
                nxt.copy_(sg.spare)
                cur, nxt = nxt, cur
                s = min(s + checkpoint_every, n_steps)
            else:
                solver.advance(cur, nxt, gcd)
                cur, nxt = nxt, cur
                s += 1
            if s % checkpoint_every == 0 and s < n_steps:
                ckpts.append(cur.clone())
        ctx.pre = set(pre)
        ctx.solver = solver
        ctx.n_steps = n_steps
        ctx.every = checkpoint_every
        ctx.n_gc = len(gc)
        ctx.use_graphs = use_graphs
        ctx.save_for_backward(*ckpts, *gcd)
        return cur

    @staticmethod
    def backward(ctx, grad_out):
        saved = ctx.saved_tensors
        n_ck = len(saved) - ctx.n_gc
        ckpts, gc = list(saved[:n_ck]), list(saved[n_ck:])
        solver, n, every = ctx.solver, ctx.n_steps, ctx.every
        pb = grad_out.detach().contiguous().clone()
        gcb = [torch.zeros_like(g) for g in gc]
        taped = _tapes_fit(solver, 2 * min(every, n), pb)  # two buffer sets when pipelined
        if ctx.use_graphs and taped:
            pre = {seg for seg in getattr(ctx, "pre", set())}
            return (None, None, None, None,
                    *_pipelined_backward(solver, ckpts, gc, pb, n, every, pre, getattr(ctx, "pre_token", None)))
        taped = taped or _tapes_fit(solver, min(every, n), pb)
        if ctx.use_graphs:
            used = []
            for seg in range(n_ck - 1, -1, -1):
                start, end = seg * every, min(seg * every + every, n)
                sg = _segment_graph(solver, end - start, pb, gc, taped)
                if sg not in used:
                    sg.load(gc)
                    used.append(sg)
                sg.run(ckpts[seg], pb)
            for sg in used:
                for acc, b in zip(gcb, sg.gcb):
                    acc += b
            return (None, None, None, None, pb, *gcb)
        for seg in range(n_ck - 1, -1, -1):
            start, end = seg * every, min(seg * every + every, n)
            states = [ckpts[seg]]
            if taped:
                # every step recorded with its result (the segment's last result is not needed,
                # but with it the recording is the forward's own fused step where that applies)
                tapes = torch.empty((end - start, solver.tape_numel()), dtype=pb.dtype, device=pb.device)
                for s in range(end - start):
                    nxt = torch.empty_like(states[-1])
                    solver.adjoint_record(states[-1], gc, tapes[s], psi_next=nxt)
                    if s + 1 < end - start:
                        states.append(nxt)
                for s in range(end - start - 1, -1, -1):
                    solver.adjoint_replay(states[s], gc, tapes[s], pb, gc_bar=gcb)
                continue
            for _ in range(start, end - 1):
                nxt = torch.empty_like(states[-1])
                solver.advance(states[-1], nxt, gc)
                states.append(nxt)
            for s in range(end - 1, start - 1, -1):
                solver.adjoint_step(states[s - start], gc, pb, gc_bar=gcb)
        return (None, None, None, None, pb, *gcb)


# Device memory one segment's tapes may take (bytes); None: a quarter of the free memory.
tape_budget = None


def _fused_record(solver: Mpdata) -> bool:
    """Whether mpdata_adjoint_record runs the forward's own fused kernel (one 2D field, two
    passes, FCT or none and no other option), so that a recorded step's result is the
    forward step's bit for bit."""
    from . import capi
    return (len(solver.shapes) == 1 and len(solver.shapes[0]) == 2 and solver.n_iters == 2 and
            (solver.opts & ~capi.FCT) == 0)


def _tapes_fit(solver: Mpdata, length: int, like) -> bool:
    need = length * solver.tape_numel() * like.element_size()
    if tape_budget is not None:
        return need <= tape_budget
    free, _total = torch.cuda.mem_get_info(like.device)
    return need <= free // 4


def _pipelined_backward(solver: Mpdata, ckpts, gc, pb, n: int, every: int, pre=frozenset(), token=None):
    """The taped backward with graphs, two segments in flight: while one segment's reverse
    sweeps run on one stream, the next segment (earlier in time; it needs only its checkpoint)
    records its states and tapes on another.  Two buffer sets alternate between segments.
    Segments in `pre` were recorded by the forward into their buffer set, which still holds
    them if no other rollout has recorded into it since (`token`)."""
    dev = pb.device
    cur = torch.cuda.current_stream(dev)
    gcb = [torch.zeros_like(g) for g in gc]
    s_rec, s_rev = _pipeline_streams(solver, dev)
    s_rec.wait_stream(cur)
    s_rev.wait_stream(cur)
    segs = []  # (segment, its buffer set), last segment first
    for idx, seg in enumerate(range(len(ckpts) - 1, -1, -1)):
        start, end = seg * every, min(seg * every + every, n)
        segs.append((seg, _segment_graph(solver, end - start, pb, gc, True, idx % 2)))
    used = []
    for _, sg in segs:
        if sg not in used:
            used.append(sg)
    with torch.cuda.stream(s_rev):
        for sg in used:
            sg.load(gc)
    s_rec.wait_stream(s_rev)
    last_rev = {}  # buffer set -> event after its last reverse sweep
    for seg, sg in segs:
        if sg in last_rev:
            s_rec.wait_event(last_rev[sg])
        with torch.cuda.stream(s_rec):
            if seg not in pre or token is None or getattr(sg, "owner", None) is not token:
                sg.states[0].copy_(ckpts[seg])
                sg.rec_graph.replay()
            recorded = torch.cuda.Event()
            recorded.record(s_rec)
        s_rev.wait_event(recorded)
        with torch.cuda.stream(s_rev):
            sg.pb.copy_(pb)
            sg.rev_graph.replay()
            pb.copy_(sg.pb)
            done = torch.cuda.Event()
            done.record(s_rev)
        last_rev[sg] = done
    for sg in used:
        sg.owner = None  # a second backward of the same forward recomputes its segments
    with torch.cuda.stream(s_rev):
        for sg in used:
            for acc, b in zip(gcb, sg.gcb):
                acc += b
    cur.wait_stream(s_rev)
    cur.wait_stream(s_rec)
    for t in [pb, *gcb, *ckpts]:
        t.record_stream(s_rev)
    for t in ckpts:
        t.record_stream(s_rec)
    return (pb, *gcb)


def _pipeline_streams(solver: Mpdata, dev):
    streams = solver.__dict__.get("_pipeline_streams")
    if streams is None:
        streams = (torch.cuda.Stream(dev), torch.cuda.Stream(dev))
        solver.__dict__["_pipeline_streams"] = streams
    return streams


class _SegmentGraph:
    """The backward work of one checkpoint segment (recompute its states, then the adjoint
    steps last to first) captured as a CUDA graph on static buffers: the states, psi_bar,
    the advector and its accumulated adjoint (and, when taped, every step's tape) all belong
    to the graph."""

    def __init__(self, solver: Mpdata, length: int, like, gc_like, taped: bool):
        self.states = [torch.zeros_like(like) for _ in range(length)]
        self.pb = torch.empty_like(like)
        self.gc = [torch.zeros_like(g) for g in gc_like]
        self.gcb = [torch.zeros_like(g) for g in gc_like]
        self.spare = torch.empty_like(like)  # the result of a segment's last recorded step
        self.tapes = torch.zeros((length, solver.tape_numel()), dtype=like.dtype, device=like.device) \
            if taped else None
        gc, gcb, tapes = self.gc, self.gcb, self.tapes
        dev = like.device
        prev = solver.stream
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        solver.set_stream(side)
        try:
            with torch.cuda.stream(side):  # first use allocates the handle's adjoint scratch
                tmp = torch.zeros_like(like)
                scratch = [torch.zeros_like(g) for g in gc]
                solver.advance(self.states[0], tmp, gc)
                solver.adjoint_step(self.states[0], gc, tmp, gc_bar=scratch)
                if taped:
                    solver.adjoint_record(self.states[0], gc, tapes[0], psi_next=tmp)
                    solver.adjoint_replay(self.states[0], gc, tapes[0], tmp, gc_bar=scratch)
            side.synchronize()
            if taped:  # the recording and the reverse sweeps as separate graphs, so that they
                # can run on two streams (_pipelined_backward), or back to back (run)
                self.rec_graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self.rec_graph, stream=side):
                    for s in range(length):
                        nxt = self.states[s + 1] if s + 1 < length else self.spare
                        solver.adjoint_record(self.states[s], gc, tapes[s], psi_next=nxt)
                self.rev_graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self.rev_graph, stream=side):
                    for s in range(length - 1, -1, -1):
                        solver.adjoint_replay(self.states[s], gc, tapes[s], self.pb, gc_bar=gcb)
                self.graph = None
            else:
                self.graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self.graph, stream=side):
                    for s in range(length - 1):
                        solver.advance(self.states[s], self.states[s + 1], gc)
                    for s in range(length - 1, -1, -1):
                        solver.adjoint_step(self.states[s], gc, self.pb, gc_bar=gcb)
        finally:
            solver.set_stream(prev)

    def load(self, gc):
        """Start a backward pass: take the advector and clear the accumulated adjoint."""
        for dst, src in zip(self.gc, gc):
            dst.copy_(src)
        for b in self.gcb:
            b.zero_()

    def run(self, checkpoint, pb):
        self.states[0].copy_(checkpoint)
        self.pb.copy_(pb)
        if self.graph is None:
            self.rec_graph.replay()
            self.rev_graph.replay()
        else:
            self.graph.replay()
        pb.copy_(self.pb)


def _segment_graph(solver: Mpdata, length: int, like, gc, taped: bool, slot: int = 0) -> _SegmentGraph:
    """The captured segment of this length, kept on the handle (a rollout has at most two
    segment lengths: checkpoint_every and the remainder; the pipelined backward uses two
    buffer sets, `slot` 0 and 1, of each)."""
    cache = solver.__dict__.setdefault("_segment_graphs", {})
    key = (length, like.dtype, tuple(like.shape), taped, slot)
    if key not in cache:
        cache[key] = _SegmentGraph(solver, length, like, gc, taped)
    return cache[key]


def rollout(solver: Mpdata, psi0, gc, n_steps: int, checkpoint_every: int = 20, use_graphs: bool = True):
    """Differentiable n-step rollout (see MPDATAFunction)."""
    return MPDATAFunction.apply(solver, n_steps, checkpoint_every, use_graphs, psi0, *gc)
