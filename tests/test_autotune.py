"""Autotuner: cache round trip (host only) and a GPU run that keeps results unchanged."""
import json

import numpy as np
import pytest
import torch

from paper_1407_1309_gb300 import autotune, capi, workloads


class FakeSolver:
    def __init__(self):
        self.device = torch.device("cpu")
        self.shapes = [(8, 8)]
        self.total = 64
        self.dtype = torch.float32
        self.n_iters = 2
        self.opts = 1
        self.tuned = []

    def tune(self, knob, value):
        self.tuned.append((knob, value))


def test_cache_hit_applies_stored_tile(tmp_path, monkeypatch):
    monkeypatch.setenv("MPDATA_GB300_TUNE_CACHE", str(tmp_path / "c.json"))
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda d=None: "fake")
    s = FakeSolver()
    key = autotune.key_of(s)
    (tmp_path / "c.json").write_text(json.dumps({key: {"kernel": 2, "tile_rows": 24, "seconds_per_step": 1e-5}}))
    best, sec, timings = autotune.autotune(s, None, None)
    assert best == (2, 24, 1) and sec == 1e-5 and timings == {}
    assert s.tuned == [(capi.TUNE_KERNEL, 2), (capi.TUNE_TILE_ROWS, 24), (capi.TUNE_STEPS_PER_LAUNCH, 1)]


def test_cache_hit_applies_stored_fusion_depth(tmp_path, monkeypatch):
    monkeypatch.setenv("MPDATA_GB300_TUNE_CACHE", str(tmp_path / "c.json"))
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda d=None: "fake")
    s = FakeSolver()
    entry = {"kernel": 0, "tile_rows": 0, "steps_per_launch": 3, "seconds_per_step": 1e-5}
    (tmp_path / "c.json").write_text(json.dumps({autotune.key_of(s): entry}))
    best, _, _ = autotune.autotune(s, None, None)
    assert best == (0, 0, 3) and (capi.TUNE_STEPS_PER_LAUNCH, 3) in s.tuned


def test_cache_entry_without_kernel_means_automatic(tmp_path, monkeypatch):
    monkeypatch.setenv("MPDATA_GB300_TUNE_CACHE", str(tmp_path / "c.json"))
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda d=None: "fake")
    s = FakeSolver()
    (tmp_path / "c.json").write_text(json.dumps({autotune.key_of(s): {"tile_rows": 8, "seconds_per_step": 2e-5}}))
    best, _, _ = autotune.autotune(s, None, None)
    assert best == (0, 8, 1)
    assert s.tuned == [(capi.TUNE_KERNEL, 0), (capi.TUNE_TILE_ROWS, 8), (capi.TUNE_STEPS_PER_LAUNCH, 1)]


def test_candidates_cover_every_kernel_family_and_fusion_depth():
    fams = {k for k, _, d in autotune.CANDIDATES if d == 1}
    assert fams == {1, 2, 3} and all(r == 0 or 4 <= r <= 65536 for _, r, _ in autotune.CANDIDATES)
    assert {d for _, _, d in autotune.CANDIDATES} == {1, 2, 3, 4}


def test_batched_handles_search_lane_widths_and_tile_heights():
    fams = {k for k, _, _ in autotune.BATCH_CANDIDATES}
    assert fams == {1, 3} and all(d == 1 and 4 <= r <= 65536 for _, r, d in autotune.BATCH_CANDIDATES)


def test_fusion_depth_only_where_the_temporal_blocking_kernel_covers_the_handle():
    s = FakeSolver()
    assert autotune.tblock_applies(s)
    for opt in (capi.TOT, capi.NUG, capi.ABS, capi.DFL, capi.KAHAN, capi.OPEN0, capi.STAGED):
        s.opts = capi.FCT | opt
        assert not autotune.tblock_applies(s), opt
    s.opts, s.n_iters = capi.FCT, 3
    assert not autotune.tblock_applies(s)
    s.n_iters, s.shapes = 2, [(8, 8, 8)]
    assert not autotune.tblock_applies(s)
    s.shapes = [(8, 8), (8, 8)]
    assert not autotune.tblock_applies(s)


@pytest.mark.gpu
def test_autotune_picks_a_candidate_and_results_do_not_change(tmp_path, monkeypatch):
    monkeypatch.setenv("MPDATA_GB300_TUNE_CACHE", str(tmp_path / "c.json"))
    from paper_1407_1309_gb300.solver import Mpdata
    psi_np, gc_np, _ = workloads.rotation_2d(256)
    dev = torch.device("cuda")
    psi = torch.tensor(psi_np, dtype=torch.float32, device=dev)
    gc = [torch.tensor(v, dtype=torch.float32, device=dev) for v in gc_np]
    with Mpdata((256, 256), dtype=torch.float32, n_iters=2, opts=capi.FCT) as m:
        ref = torch.empty_like(psi)
        m.advance(psi, ref, gc, n_steps=5)
        best, sec, timings = autotune.autotune(m, psi, gc, steps=3, flush_bytes=0)
        assert best in autotune.CANDIDATES and sec > 0 and len(timings) == len(autotune.CANDIDATES)
        out = torch.empty_like(psi)
        m.advance(psi, out, gc, n_steps=5)
        torch.cuda.synchronize()
        # the tile height changes the schedule, not the arithmetic; the two kernel families
        # agree to rounding (the compiler fuses multiply-adds differently in each)
        assert torch.linalg.norm(out - ref) <= 1e-6 * torch.linalg.norm(ref)
        stored = json.loads((tmp_path / "c.json").read_text())[autotune.key_of(m)]
        assert (stored["kernel"], stored["tile_rows"], stored["steps_per_launch"]) == best
