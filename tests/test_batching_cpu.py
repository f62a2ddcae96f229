"""Host logic of the batch packing (no GPU): the candidate splits of a set of
handles into batches never mix membrane models or precisions, cover every
handle exactly once, and the tuner keys its choice by the shape class."""
from types import SimpleNamespace

from paper_2510_27447_gb300 import batching as B


def _sim(model, prec, n):
    return SimpleNamespace(model=model, opts=SimpleNamespace(precision=prec), N=n)


def _mix():
    sims = []
    for k in range(20):
        sims.append(_sim(k % 2, 1, (33, 65, 129)[k % 3] ** 2))
    sims.append(_sim(0, 0, 33 ** 2))            # an FP64 handle among the mixed ones
    return sims


def test_every_packing_covers_each_handle_once_and_keeps_batches_compatible():
    sims = _mix()
    cands = B.candidate_packings(sims)
    assert {"model", "size"} <= set(cands)
    for name, packing in cands.items():
        flat = sorted(i for b in packing for i in b)
        assert flat == list(range(len(sims))), name
        for b in packing:
            assert len({(sims[i].model, sims[i].opts.precision) for i in b}) == 1, name
    # one batch per (model, precision); per size: one per (model, precision, N)
    assert len(cands["model"]) == 3
    assert len(cands["size"]) == len({(s.model, s.opts.precision, s.N) for s in sims})


def test_capped_packings_hold_at_most_k_handles_sorted_by_size():
    sims = _mix()
    for name, packing in B.candidate_packings(sims).items():
        if not name.startswith("cap"):
            continue
        k = int(name[3:])
        for b in packing:
            assert 1 <= len(b) <= k
            sizes = [sims[i].N for i in b]
            assert sizes == sorted(sizes)


def test_capped_packings_that_repeat_a_batch_count_are_dropped():
    # four handles of one model: cap4/8/16 would each give one batch, the same
    # count as "model" -- none is offered
    sims = [_sim(0, 1, 33 ** 2) for _ in range(4)]
    cands = B.candidate_packings(sims)
    assert set(cands) == {"model", "size"}


def test_shape_class_ignores_order():
    sims = _mix()
    assert B.shape_class(sims) == B.shape_class(list(reversed(sims)))
    assert B.shape_class(sims) != B.shape_class(sims[:-1])


def test_option_candidates_cover_the_layout_and_thread_choices():
    from paper_2510_27447_gb300 import binding
    s_mixed = B.option_candidates(True, binding.MIXED)
    s_fp64 = B.option_candidates(False, binding.FP64)
    assert s_mixed["auto"] == {} and s_fp64["auto"] == {}
    assert {"wide_sell": -1, "csr_lanes": 16} in s_mixed.values()
    assert {"vec4": -1} in s_mixed.values()
    assert "sell32" not in B.option_candidates(True, binding.FP64)     # no vector-load copy in FP64
    assert {c.get("cg_block") for c in s_fp64.values()} == {None, 256, 1024}
    for c in list(s_mixed.values()) + list(s_fp64.values()):
        o = binding.default_options(**c)                                   # every key is an option
        for k, v in c.items():
            assert getattr(o, k) == v
