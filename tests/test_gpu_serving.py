"""Serving on the GPU: results through the continuous-batching loop (lanes overlapping on
the device) are bitwise equal to the same requests served one at a time."""
import numpy as np
import pytest

from paper_2310_16829_gb300 import lma, serving as S, workloads as WL

pytestmark = pytest.mark.gpu


def _resident():
    return WL.perovskite_workload(cells=5, nx=256, n_slices=12, n_phonons=1, seed_base=3100,
                                  probes=64)


def _fresh(seed):
    return WL.perovskite_workload(cells=5, nx=256, n_slices=8, n_phonons=1, seed_base=seed,
                                  probes=32)


def _requests():
    reqs = []
    for k in range(4):
        cx, cy, op, spc = WL.edit_request(5, k, 3200)
        reqs.append(S.EditRequest(cx, cy, op, spc, region_probes=16))
        reqs.append(S.ImageRequest("full_256", seed=500 + k))
    return reqs


def _serve(budget, max_inst, concurrent):
    lanes = [S.edit_lane(_resident()), S.image_lane("full_256", _fresh, max_instances=max_inst)]
    srv = S.Server(lanes, budget_bytes=budget)
    reqs = _requests()
    if concurrent:
        tickets = [srv.submit(r) for r in reqs]
        res = [t.wait(600) for t in tickets]
    else:
        res = [srv.submit(r).wait(600) for r in reqs]
    srv.close()
    return res, srv


def test_results_are_the_same_alone_and_in_the_mix():
    import torch
    assert torch.cuda.is_available()
    mix, srv_mix = _serve(budget=64 << 30, max_inst=3, concurrent=True)
    alone, _ = _serve(budget=64 << 30, max_inst=1, concurrent=False)
    for a, b in zip(mix, alone):
        assert a.error is None and b.error is None, (a.error, b.error)
        assert np.array_equal(a.image, b.image)
    # the mix really overlapped: several image instances were admitted
    assert len(srv_mix.lanes["full_256"].instances) > 1
    # edits re-propagate only part of the resident exit waves (a column already removed
    # by an earlier edit changes nothing)
    edits = [r for r in mix if isinstance(r.request, S.EditRequest)]
    assert any(r.n_stale > 0 for r in edits)


def test_image_requests_match_a_direct_call():
    res, _ = _serve(budget=64 << 30, max_inst=2, concurrent=True)
    w = _fresh(500)
    ctx = lma.Context(0)
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    direct = basis.image(w.detectors, w.region, recompute=True)
    assert np.array_equal(res[1].image, direct)
