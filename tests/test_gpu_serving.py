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


def test_warm_edits_make_no_device_allocation():
    """Once an edit lane is warm, an edit and its region image allocate nothing: device
    allocation can wait for the whole device, which would hold an edit behind other
    lanes' full images."""
    import torch
    assert torch.cuda.is_available()
    w = _resident()
    ctx = lma.Context(0)
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    st = torch.cuda.Stream()
    basis.propagate(0, stream=st)
    dx = w.grid.lx / w.grid.nx

    def edit(k):
        cx, cy, op, spc = WL.edit_request(5, k, 3300)
        px, py = int(round(cx / dx)) // 4 * 4, int(round(cy / dx)) // 4 * 4
        region = WL.Region(px - 32, py - 32, 16, 16, (4, 4))
        spec.edit_column(basis, cx, cy, 0.5, op, spc)
        return basis.image(w.detectors, region, stream=st)

    edit(0)                       # warm: region tables, item-list slab, staging buffer
    ctx.profile_enable(True)
    for k in range(1, 6):
        assert np.all(np.isfinite(edit(k)))
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    assert prof["allocations"] == 0, prof
    assert prof["slice"]["launches"] >= 1
    basis.close()
    spec.close()
    ctx.close()


def test_bounded_lane_serves_the_unbounded_images():
    """A lane whose store holds 1024 of the 4096 exit waves computes its images part by
    part (Sec. 4.2.4) and returns the unbounded lane's images bit for bit."""
    lanes = [S.image_lane("full_256", _fresh, max_instances=1),
             S.image_lane("bounded_256", _fresh, max_instances=1, max_resident=1024)]
    srv = S.Server(lanes, budget_bytes=1 << 40)
    full = [srv.submit(S.ImageRequest("full_256", seed=700 + k)) for k in range(2)]
    bounded = [srv.submit(S.ImageRequest("bounded_256", seed=700 + k)) for k in range(2)]
    res_f = [t.wait(600) for t in full]
    res_b = [t.wait(600) for t in bounded]
    srv.close()
    for a, b in zip(res_f, res_b):
        assert a.error is None and b.error is None
        assert np.array_equal(a.image, b.image)
    assert lanes[1].reserve_bytes < lanes[0].reserve_bytes
