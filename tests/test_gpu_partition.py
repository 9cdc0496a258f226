"""Memory-bounded images (Sec. 4.2.4) on the GPU: every strategy gives the unbounded image
bit for bit (the same exit waves and readings, held in a bounded store), and the number of
exit waves propagated per configuration is the plan's T_{P_1..P_l}."""
import numpy as np
import pytest

from paper_2310_16829_gb300 import lma, workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lma.Context(0)


@pytest.mark.parametrize("precision", [WL.PREC_C64, WL.PREC_FP16_STORE])
def test_partitioned_image_equals_unbounded_image(ctx, precision):
    w = WL.perovskite_workload(cells=5, nx=256, n_slices=6, n_phonons=2, seed_base=2400)
    w.basis.precision = precision
    region = WL.Region(36, 180, 21, 15, (4, 4))      # wraps around the cell edge
    dets = [WL.Detector(0.0, 0.02), WL.Detector(0.07, 0.2)]
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    ref = basis.image(dets, region, recompute=True)
    for strategy in (lma.LMA_PART_ROWS, lma.LMA_PART_RECTANGLES, lma.LMA_PART_RECTANGLES_COLUMN_MAJOR,
                     lma.LMA_PART_GREEDY):
        for M in (200, 420):
            _, n_parts, runs, peak = basis.partition(region, strategy, M, start=100)
            ctx.profile_enable(True)
            got = basis.image_partitioned(dets, region, strategy, M, start=100)
            prof = ctx.profile_read()
            ctx.profile_enable(False)
            assert np.array_equal(got, ref), (strategy, M)
            # translate-slices propagated = T per configuration x slices x configurations
            assert prof["slice"]["units"] == runs * w.grid.n_slices * len(w.phonons), (strategy, M)
            assert prof["synth"]["units"] == region.npx * region.npy * len(w.phonons)
            assert n_parts > 1 and peak <= M


def test_partitioned_store_is_bounded_and_reused(ctx):
    w = WL.perovskite_workload(cells=5, nx=256, n_slices=4, n_phonons=1, seed_base=2500)
    region = WL.Region(0, 0, 32, 32, (4, 4))
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    ref = basis.image(w.detectors, region, recompute=True)
    basis.image_partitioned(w.detectors, region, lma.LMA_PART_RECTANGLES, 300)
    ctx.profile_enable(True)
    got = basis.image_partitioned(w.detectors, region, lma.LMA_PART_RECTANGLES, 300)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    assert np.array_equal(got, ref)
    assert prof["allocations"] == 0      # plan tables and the bounded store are kept
