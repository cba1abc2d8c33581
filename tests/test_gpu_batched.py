"""Uneven batches (segments of different lengths and rates): the batched C
entry points and their CUDA-graph capture give the per-group results, and
those match the FP64 oracle."""
import numpy as np
import pytest

from oracle import qtam_oracle as O
from paper_2603_29785_gb300 import batch, qtam

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

QS, FMIN, FMAX, K = (8.0, 16.0, 32.0), 20.0, 2048.0, 128


@pytest.fixture(scope="module")
def uneven():
    segs, rates = batch.uneven_workload(n_segments=14, durations=(1, 2, 4), seed=3)
    cache = batch.PlanCache(QS, FMIN, FMAX, K, device=0)
    ub = batch.UnevenBatch(segs, rates, cache, tune=True)
    return segs, rates, cache, ub


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_groups_cover_every_segment(uneven):
    segs, rates, cache, ub = uneven
    seen = sorted(i for g in ub.groups for i in g.index)
    assert seen == list(range(len(segs)))
    assert len(cache) == len(ub.groups) >= 4
    for g in ub.groups:
        assert all(len(segs[i]) == g.N and rates[i] == g.fs for i in g.index)


def test_batched_equals_per_group_calls(uneven):
    segs, rates, cache, ub = uneven
    ub.roundtrip()
    torch.cuda.synchronize()
    for g in ub.groups:
        y = g.plan.forward(g.x)
        torch.cuda.synchronize()
        assert torch.equal(torch.view_as_real(y), torch.view_as_real(g.y))     # same kernels, same bits
        xh = g.plan.inverse(y)
        torch.cuda.synchronize()
        assert float((xh - g.xh).norm() / xh.norm()) < 1e-6                   # atomics: order may differ


def test_batched_matches_oracle(uneven):
    segs, rates, cache, ub = uneven
    ub.roundtrip()
    torch.cuda.synchronize()
    for i in (0, 1, 5, len(segs) - 1):
        fs, x = rates[i], segs[i].astype(np.float64)
        g = O.geometry(fs, len(x), QS, FMIN, FMAX, K)
        Y = ub.envelopes(i).cpu().numpy().astype(np.complex128)
        assert rel(Y, O.forward(g, x)) < 1e-6
        tau = cache.get(fs, len(x)).info["p_floor_rel"]
        xh = ub.reconstruction(i).cpu().numpy().astype(np.float64)
        assert rel(xh, O.projection(g, x, tau=tau)) < 1e-5


def test_graph_replay_equals_eager(uneven):
    segs, rates, cache, ub = uneven
    ub.roundtrip()
    torch.cuda.synchronize()
    y_eager = [g.y.clone() for g in ub.groups]
    x_eager = [g.xh.clone() for g in ub.groups]
    for g in ub.groups:
        g.y.zero_()
        g.xh.zero_()
    for n_streams in (1, 3):
        for g in ub.groups:
            g.y.zero_()
            g.xh.zero_()
        ub.capture(n_streams=n_streams)
        ub.replay()
        torch.cuda.synchronize()
        for g, ye, xe in zip(ub.groups, y_eager, x_eager):
            assert torch.equal(torch.view_as_real(g.y), torch.view_as_real(ye))
            assert float((g.xh - xe).norm() / xe.norm()) < 1e-6
