"""Handles used from several host threads at once.

The library's one-time launch set-up (opt-in shared-memory sizes, persistent grid sizes) is
kept per device and made under a lock, so two threads that launch the same kernels for the
first time on two streams of one device both get it before their first launch.  Each thread
here owns a handle on its own stream; the results must equal a serial run bit for bit.
"""
import threading

import numpy as np
import pytest
import torch

from helpers import nondivergent, smooth_positive
from paper_1407_1309_gb300 import capi
from paper_1407_1309_gb300.solver import Mpdata

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")

JOBS = [
    ((18, 21, 40), torch.float64, 3, capi.TOT | capi.FCT),   # 3D FP64 corrective march: > 48 KB shared
    ((18, 21, 40), torch.float32, 3, capi.TOT | capi.FCT),
    ((300, 260), torch.float32, 2, capi.FCT),
    ((300, 260), torch.float64, 2, capi.FCT),
    ((1500,), torch.float64, 2, capi.FCT),
]


def inputs(shape, dtype, seed):
    rng = np.random.default_rng(seed)
    t = lambda a: torch.tensor(a, dtype=dtype, device=DEV)
    return t(smooth_positive(shape, rng)), [t(v) for v in nondivergent(shape, rng, 0.35)]


def run(job, seed, stream):
    shape, dtype, n_iters, opts = job
    with torch.cuda.stream(stream):
        psi, gc = inputs(shape, dtype, seed)
        with Mpdata(shape, dtype=dtype, n_iters=n_iters, opts=opts, stream=stream) as m:
            out = torch.empty_like(psi)
            m.advance(psi, out, gc, n_steps=6)
            stream.synchronize()
            return out.cpu()


def test_two_threads_two_streams_equal_serial_runs():
    serial = [run(job, i, torch.cuda.current_stream()) for i, job in enumerate(JOBS)]
    results = [[None] * len(JOBS) for _ in range(2)]
    errors = []

    def worker(w):
        try:
            s = torch.cuda.Stream(DEV)
            order = range(len(JOBS)) if w == 0 else reversed(range(len(JOBS)))
            for i in order:
                results[w][i] = run(JOBS[i], i, s)
        except Exception as ex:  # reported by the main thread
            errors.append(ex)

    threads = [threading.Thread(target=worker, args=(w,)) for w in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for w in range(2):
        for i in range(len(JOBS)):
            assert torch.equal(results[w][i], serial[i]), (w, JOBS[i])
