"""Scheduler logic of the continuous-batching server (no GPU): admission by
free slot and HBM footprint, FIFO order, overlap of admitted requests,
completion accounting and latency statistics."""
import numpy as np
import pytest

from paper_2510_27447_gb300 import serving as S
from paper_2510_27447_gb300 import workloads as W


def _jobs(n, rate, seed, sizes=(1089, 4225, 16641)):
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(n):
        t += rng.exponential(1.0 / rate)
        out.append(S.Job(r, t, int(sizes[rng.integers(0, len(sizes))]), 200))
    return out


def test_every_request_completes_once_with_positive_latency():
    ex = S.VirtualExecutor(rate=2e8)
    done = S.Server(ex, max_slots=4, hbm_budget=10**9, chunk_steps=25).run(_jobs(40, 50.0, 1))
    assert sorted(c.rid for c in done) == list(range(40))
    for c in done:
        assert c.finished >= c.admitted >= c.arrival
    s = S.summarize(done)
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_slots_and_memory_bound_the_resident_set():
    ex = S.VirtualExecutor(rate=1e8, bytes_per_node=1000)
    jobs = [S.Job(r, 0.0, 16641, 100) for r in range(10)]
    # budget fits two 16641-node requests at a time although 6 slots are free
    done = S.Server(ex, max_slots=6, hbm_budget=2 * 16641 * 1000, chunk_steps=20).run(jobs)
    assert len(done) == 10
    assert ex.max_live == 2


def test_fifo_admission_and_overlap():
    ex = S.VirtualExecutor(rate=1e8)
    jobs = [S.Job(r, 0.001 * r, 4225, 100) for r in range(8)]
    done = S.Server(ex, max_slots=3, hbm_budget=10**12, chunk_steps=10).run(jobs)
    assert ex.started == list(range(8))          # admitted in arrival order
    assert ex.max_live == 3                      # requests overlap up to the slot count
    # with processor sharing, three resident requests finish later than one alone
    first = min(done, key=lambda c: c.rid)
    assert first.latency > 4225 * 100 / 1e8


def test_request_larger_than_budget_is_refused():
    ex = S.VirtualExecutor(bytes_per_node=1000)
    with pytest.raises(ValueError):
        S.Server(ex, max_slots=2, hbm_budget=1000).run([S.Job(0, 0.0, 5000, 10)])


def test_idle_gaps_advance_the_clock_to_the_next_arrival():
    ex = S.VirtualExecutor(rate=1e9)
    jobs = [S.Job(0, 0.0, 1089, 10), S.Job(1, 5.0, 1089, 10)]
    done = S.Server(ex, max_slots=2, hbm_budget=10**9).run(jobs)
    late = [c for c in done if c.rid == 1][0]
    assert late.admitted >= 5.0 and late.latency < 0.1


def test_request_stream_workloads_are_well_formed():
    reqs = W.request_stream(16, 40.0, seed=4, t_end=2.0)
    assert all(r.side in (33, 65, 129, 257, 513) for r in reqs)
    assert all(250 <= r.s2_time <= 350 for r in reqs)
    times = [r.arrival_s for r in reqs]
    assert times == sorted(times)
    w = W.request_workload(reqs[0])
    assert w.n_nodes == reqs[0].side ** 2 and w.n_steps == 100
    assert w.stimuli[0].mask.sum() > 0


def test_batched_form_completes_every_request_and_joins_at_chunk_boundaries():
    ex = S.VirtualExecutor(rate=1e8)
    jobs = [S.Job(r, 0.002 * r, 1089 * (1 + r % 3), 60 + 20 * (r % 2)) for r in range(12)]
    done = S.Server(ex, max_slots=6, hbm_budget=10**12, chunk_steps=20, batched=True).run(jobs)
    assert sorted(c.rid for c in done) == list(range(12))
    assert 2 < ex.max_live <= 6                 # several requests share each chunk, within the slots
    for c in done:
        assert c.finished >= c.admitted >= c.arrival


def test_handle_construction_does_not_stall_resident_requests():
    """A slow build (a worker's time) delays only its own request: the
    resident one keeps advancing and finishes as if alone."""
    ex = S.VirtualExecutor(rate=1e8, setup=1.0)
    jobs = [S.Job(0, 0.0, 1000, 100), S.Job(1, 1.5, 1000, 100)]
    done = {c.rid: c for c in S.Server(ex, max_slots=2, hbm_budget=10**9, chunk_steps=10).run(jobs)}
    # job 0: built in 1 s, then 1e5 node-steps at 1e8/s alone; job 1 arrives at 1.5 s
    assert done[0].finished == pytest.approx(1.001, abs=0.01)
    assert done[1].admitted == pytest.approx(1.5, abs=0.01)
    assert done[1].finished >= 2.5


def test_closed_loop_keeps_the_client_count_outstanding():
    ex = S.VirtualExecutor(rate=1e8)
    jobs = [S.Job(r, 99.0, 4225, 50) for r in range(10)]
    done = S.Server(ex, max_slots=8, hbm_budget=10**12, chunk_steps=10).run_closed(jobs, clients=3)
    assert len(done) == 10 and ex.max_live == 3
    assert min(c.arrival for c in done) == 0.0            # arrival times are the submission times


def test_fifo_schedule_and_offered_load():
    jobs = [S.Job(0, 0.0, 100, 10), S.Job(1, 0.5, 100, 10), S.Job(2, 5.0, 100, 10)]
    done = S.fifo_schedule(jobs, [1.0, 1.0, 1.0])
    fin = {c.rid: c.finished for c in done}
    assert fin == {0: 1.0, 1: 2.0, 2: 6.0}
    sm = S.summarize(done)
    assert sm["offered_node_steps_per_s"] == pytest.approx(3000 / 5.0)
    assert sm["node_steps_per_s"] == pytest.approx(3000 / 6.0)
    assert sm["served_over_offered"] == pytest.approx(5.0 / 6.0)


def test_batched_form_serves_large_requests_alone():
    """With a size threshold the batched server groups only the small
    requests (by mesh size); requests at or above it advance alone, and every
    request completes, including ones of zero steps."""
    ex = S.VirtualExecutor(rate=1e8, solo_nodes=10000)
    jobs = [S.Job(r, 0.001 * r, (1089, 4225, 16641)[r % 3], 0 if r == 7 else 40 + 10 * (r % 2)) for r in range(15)]
    done = S.Server(ex, max_slots=8, hbm_budget=10**12, chunk_steps=20, batched=True).run(jobs)
    assert sorted(c.rid for c in done) == list(range(15))
    size = {j.rid: j.n_nodes for j in jobs}
    grouped = {r for g in ex.grouped for r in g}
    assert grouped == {j.rid for j in jobs if j.n_nodes < 10000}
    for g in ex.grouped:
        assert len({size[r] for r in g}) == 1                 # one mesh size per group
    assert any(len(g) > 1 for g in ex.grouped)                # small requests share chunks


@pytest.mark.parametrize("max_solo", [1, 2])
def test_solo_limit_bounds_the_large_requests_advancing_at_once(max_solo):
    """Batched form with max_solo: requests served alone advance at most
    max_solo at a time (the others wait, admitted and built), the small
    ones keep batching meanwhile, and every request completes."""
    ex = S.VirtualExecutor(rate=1e8, solo_nodes=10000)
    jobs = [S.Job(r, 0.0005 * r, (1089, 16641, 4225, 16641)[r % 4], 40) for r in range(16)]
    done = S.Server(ex, max_slots=10, hbm_budget=10**12, chunk_steps=10, batched=True,
                    max_solo=max_solo).run(jobs)
    assert sorted(c.rid for c in done) == list(range(16))
    assert ex.max_busy_solo == max_solo
    assert any(len(g) > 1 for g in ex.grouped)
