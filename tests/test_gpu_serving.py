"""Continuous batching on the GPU: requests that arrive while others run are
admitted into free slots, their steps overlap on the device (one stream per
request), and each request's activation map is the same alone and in the
mix (bitwise: every kernel is deterministic and per-request)."""
import numpy as np
import pytest

from paper_2510_27447_gb300 import binding
from paper_2510_27447_gb300 import serving as S
from paper_2510_27447_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _jobs(t_end=1.2):
    reqs = W.request_stream(6, 400.0, seed=11, sides=(33, 65), t_end=t_end)
    return [S.Job(r.rid, r.arrival_s, r.side ** 2, int(round(t_end / r.dt)), W.request_workload(r))
            for r in reqs]


@pytest.mark.parametrize("precision", [binding.FP64, binding.MIXED])
def test_results_are_identical_alone_and_in_the_mix(precision):
    opts = lambda: binding.default_options(precision=precision)       # noqa: E731
    jobs = _jobs()
    assert {j.payload.model for j in jobs} == {W.LR91, W.TP06_EPI}
    alone = {}
    for j in jobs:
        ex = S.GpuExecutor(opts, dt=0.02)
        d = S.Server(ex, max_slots=1, chunk_steps=20).run([S.Job(j.rid, 0.0, j.n_nodes, j.n_steps, j.payload)])
        alone[j.rid] = d[0].result
    ex = S.GpuExecutor(opts, dt=0.02)
    mixed = S.Server(ex, max_slots=6, chunk_steps=7).run(jobs)
    assert len(mixed) == len(jobs)
    for c in mixed:
        a = alone[c.rid]
        assert np.sum(~np.isnan(a)) > 0                # the S1 strip activated
        np.testing.assert_array_equal(np.isnan(c.result), np.isnan(a))
        np.testing.assert_array_equal(c.result[~np.isnan(a)], a[~np.isnan(a)])
    s = S.summarize(mixed)
    assert s["p99_ms"] >= s["p50_ms"] > 0


@pytest.mark.parametrize("precision", [binding.FP64, binding.MIXED])
def test_batched_serving_gives_each_request_the_same_map_alone_and_in_the_mix(precision):
    """The batched form: resident requests advance together through
    bd_batch_step (one batch per membrane model), requests join at chunk
    boundaries; a request's activation map is the same as when it is served
    alone through the same batched kernels."""
    opts = lambda: binding.default_options(precision=precision)       # noqa: E731
    jobs = _jobs()
    alone = {}
    for j in jobs:
        ex = S.GpuExecutor(opts, dt=0.02)
        d = S.Server(ex, max_slots=1, chunk_steps=20, batched=True).run(
            [S.Job(j.rid, 0.0, j.n_nodes, j.n_steps, j.payload)])
        alone[j.rid] = d[0].result
        ex.close()
    ex = S.GpuExecutor(opts, dt=0.02)
    mixed = S.Server(ex, max_slots=6, chunk_steps=7, batched=True).run(jobs)
    ex.close()
    assert len(mixed) == len(jobs)
    for c in mixed:
        a = alone[c.rid]
        assert np.sum(~np.isnan(a)) > 0
        np.testing.assert_array_equal(np.isnan(c.result), np.isnan(a))
        np.testing.assert_array_equal(c.result[~np.isnan(a)], a[~np.isnan(a)])


@pytest.mark.parametrize("precision", [binding.FP64, binding.MIXED])
def test_hybrid_serving_gives_each_request_the_same_map_alone_and_in_the_mix(precision):
    """Batched form with a size threshold: 33 x 33 requests advance in
    batches, 65 x 65 ones alone on their own streams, in one server; every
    request's map is the same as when it is served alone in the same form."""
    opts = lambda: binding.default_options(precision=precision)       # noqa: E731
    jobs = _jobs()
    assert {j.n_nodes for j in jobs} == {33 ** 2, 65 ** 2}
    alone = {}
    for j in jobs:
        ex = S.GpuExecutor(opts, dt=0.02, solo_nodes=2000)
        d = S.Server(ex, max_slots=1, chunk_steps=20, batched=True).run(
            [S.Job(j.rid, 0.0, j.n_nodes, j.n_steps, j.payload)])
        alone[j.rid] = d[0].result
        ex.close()
    ex = S.GpuExecutor(opts, dt=0.02, solo_nodes=2000)
    mixed = S.Server(ex, max_slots=6, chunk_steps=7, batched=True).run(jobs)
    ex.close()
    assert len(mixed) == len(jobs)
    for c in mixed:
        a = alone[c.rid]
        assert np.sum(~np.isnan(a)) > 0
        np.testing.assert_array_equal(np.isnan(c.result), np.isnan(a))
        np.testing.assert_array_equal(c.result[~np.isnan(a)], a[~np.isnan(a)])
