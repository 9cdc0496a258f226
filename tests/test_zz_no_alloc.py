"""The readout entry point that allocates no device memory (collected last on purpose).

Some callers cannot call cudaMalloc: their device memory is held by another
allocator, or their process must not grow its device footprint. For them
lma_readout_noalloc reads out caller-held exit waves into a caller-held output
with all scratch in a fixed device array. This test checks it against
lma_image on the same specimen, twice in a row (the scratch array keeps the
previous call's contents, so the second call checks that the accumulator is
cleared).
"""
import numpy as np
import pytest

from paper_2310_16829_gb300 import lma, workloads as WL

pytestmark = pytest.mark.gpu

PIXEL_TOL = 1e-4


def _noalloc_case(w, dets, region):
    """lma_image (the allocating entry point) and two no-allocation readouts of the same
    exit waves; the library's allocation counter must stay at zero across the readouts."""
    import torch
    assert torch.cuda.is_available(), "GPU test"
    ctx = lma.Context(0)
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    basis.propagate(0)                                  # every exit wave current
    ref = basis.image(dets, region)                     # the allocating entry point
    n = int(basis.info().n_translates)
    U = torch.empty((n, 128, 128), dtype=torch.complex64, device="cuda")
    for i in range(n):
        basis.exit_wave(i, out=U[i])
    out = torch.empty((len(dets), region.npy, region.npx), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    ctx.profile_enable(False)                           # resets the counters, no event timing
    for call in range(2):
        out.fill_(float("nan"))
        basis.readout_noalloc(U, dets, region, out)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        rel = np.max(np.abs(got - ref) / np.abs(ref))
        assert rel <= PIXEL_TOL, (call, rel)
        assert np.array_equal(got, ref), call             # same kernel, same inputs: same bits
    assert ctx.profile_read()["allocations"] == 0


def test_readout_without_allocation_matches_lma_image():
    """Windows equal to the whole 128^2 cell: placements are cyclic."""
    w = WL.simple_cubic_workload()
    dets = [WL.Detector(0.0, 0.02), WL.Detector(0.02, 0.06), WL.Detector(0.06, 0.2)]
    _noalloc_case(w, dets, WL.Region(3, 5, 13, 7, (3, 5)))


def test_readout_without_allocation_non_periodic_windows():
    """A 256^2 cell: each 128^2 window is a part of the cell, placements are truncated, and
    the region wraps around the cell edge."""
    w = WL.perovskite_workload(cells=5, nx=256, n_slices=6, n_phonons=1, seed_base=2900)
    dets = [WL.Detector(0.0, 0.025), WL.Detector(0.07, 0.2)]
    _noalloc_case(w, dets, WL.Region(250, 60, 6, 5, (4, 4)))


def test_readout_without_allocation_rejects_oversized_regions():
    import torch
    w = WL.perovskite_workload(n_phonons=1, n_slices=2)
    ctx = lma.Context(0)
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    U = torch.zeros((1, 128, 128), dtype=torch.complex64, device="cuda")
    out = torch.empty((1, 128, 128), dtype=torch.float64, device="cuda")
    with pytest.raises(lma.LmaError) as e:
        basis.readout_noalloc(U, w.detectors, WL.Region(0, 0, 128, 128, (4, 4)), out)
    assert e.value.status == lma.LMA_ERR_INVALID and "scratch" in str(e.value)
