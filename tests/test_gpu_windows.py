"""Propagation windows other than 128 x 128 (Sec. 4.2.1 option (ii), windows of X' x Y'
pixels): W = 64 (the whole wave in shared memory) and W = 256 (the wave in a global scratch,
columns staged through shared memory with bulk copies), with the detection window D = 128.
Each exit wave is the multislice of its translate on its own W x W window; the synthesis
places it into the probe's 128 x 128 window, truncated where it overhangs (W = 256) or
surrounded by zeros (W = 64). Against the FP64 oracle with the same W and D.

Tolerances as in the parity tests: exit waves to 5e-5 of their peak, readings to 1e-4
relative or three times the complex64 floor of the same image (``parity_floor``).
"""
import dataclasses

import numpy as np
import pytest

from oracle import lma_oracle as O
from paper_2310_16829_gb300 import lma, workloads as WL
from parity_floor import assert_floor, oracles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lma.Context(0)


def _with_window(w, W):
    return dataclasses.replace(w, basis=dataclasses.replace(w.basis, window=W))


@pytest.mark.parametrize("W,case", [(64, "simple_cubic"), (64, "perovskite_256"), (256, "perovskite_256"),
                                    (256, "perovskite_512_wide_band")])
def test_window_exit_waves_and_images_match_oracle(ctx, W, case):
    if case == "simple_cubic":
        w = WL.simple_cubic_workload()
        region = WL.Region(0, 0, 3, 2, (8, 8))
        idx = (0, 33, 1023)
    elif case == "perovskite_256":
        w = WL.perovskite_workload(cells=5, nx=256, n_slices=6, n_phonons=2, seed_base=2900)
        region = WL.Region(250, 60, 4, 3, (4, 4))   # wraps around the cell edge
        idx = (0, 63, 64 * 32 + 17, 4095)
    else:
        w = WL.perovskite_workload(n_phonons=1, n_slices=8)
        w = dataclasses.replace(w, grid=dataclasses.replace(w.grid, bandlimit_frac=1.0))
        region = WL.Region(508, 4, 3, 3, (4, 4))
        idx = (0, 127 * 128 + 1)
    w = _with_window(w, W)
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    assert basis.info().window == W
    basis.propagate(0)
    orc, emu = oracles(w)
    for i in idx:
        got = basis.exit_wave(i)
        assert got.shape == (W, W)
        ref = orc.exit_wave(0, i)
        assert np.max(np.abs(got - ref)) < 5e-5 * np.max(np.abs(ref)), (W, case, i)
    dets = [WL.Detector(0.0, 0.02), WL.Detector(0.06, 0.2)]
    img = basis.image(dets, region, recompute=True).reshape(2, -1)
    probes = O.region_probes(region.px0, region.py0, region.npx, region.npy, region.spacing_px,
                             w.grid.nx, w.grid.ny)
    assert_floor(img, orc.image(dets, probes), emu.image(dets, probes), label=f"W={W} {case}")


def test_window_256_edit_and_partition_equal_full_recompute(ctx):
    """The other callers of the slice step with W = 256: a column edit gives the bits of a full
    recompute, and a memory-bounded partitioned image the bits of the plain image."""
    w = _with_window(WL.perovskite_workload(cells=10, nx=512, n_slices=4, n_phonons=1, seed_base=3100), 256)
    region = WL.Region(200, 200, 6, 5, (4, 4))
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    plain = basis.image(w.detectors, region, recompute=True)
    part = basis.image_partitioned(w.detectors, region, lma.LMA_PART_ROWS, 128)
    assert np.array_equal(plain, part)
    cx, cy = 5.5 * WL.ABO3_A, 5.5 * WL.ABO3_A
    spec.edit_column(basis, cx, cy, 0.5, lma.LMA_EDIT_SET_SPECIES, 2)
    after = basis.image(w.detectors, region)
    ph = []
    for at in w.phonons:
        x, y, s, sp, _ = O.edit_column(at.x, at.y, at.slice, at.species, w.grid.lx, w.grid.ly, cx, cy, 0.5, 1, 2)
        ph.append(WL.Atoms(x, y, s, sp))
    spec2 = lma.Specimen(ctx, w.grid, w.potential, ph)
    full = lma.Basis(ctx, spec2, w.probe, w.basis).image(w.detectors, region, recompute=True)
    assert np.array_equal(after, full)


def test_window_forms_that_need_w128_are_rejected(ctx):
    w = _with_window(WL.perovskite_workload(cells=5, nx=256, n_slices=2, n_phonons=1), 64)
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    for prec in (WL.PREC_FP16_STORE, WL.PREC_MIXED):
        b = lma.Basis(ctx, spec, w.probe, dataclasses.replace(w.basis, precision=prec))
        with pytest.raises(lma.LmaError) as e:
            b.propagate(0)
        assert e.value.status == lma.LMA_ERR_UNSUPPORTED
    b = lma.Basis(ctx, spec, w.probe, w.basis)
    with pytest.raises(lma.LmaError) as e:
        b.image_realspace(3, 3, w.detectors, WL.Region(0, 0, 2, 2, (4, 4)))
    assert e.value.status == lma.LMA_ERR_UNSUPPORTED


def test_window_256_specimens_of_different_grids_in_one_launch(ctx):
    """Two W = 256 specimens with different grids, slice counts and propagators share one slice
    launch in lma_image_many (one job each: the kernel switches the propagator table between
    them); each image is bit for bit the image of its own call."""
    ws = [_with_window(WL.perovskite_workload(cells=5, nx=256, n_slices=6, n_phonons=1, seed_base=3300), 256),
          _with_window(WL.perovskite_workload(cells=10, nx=512, n_slices=3, n_phonons=1, seed_base=3400), 256)]
    regions = [WL.Region(250, 60, 4, 3, (4, 4)), WL.Region(100, 400, 5, 4, (4, 4))]
    objs = []
    single = []
    for w, r in zip(ws, regions):
        spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
        basis = lma.Basis(ctx, spec, w.probe, w.basis)
        objs.append((spec, basis))
        single.append(basis.image(w.detectors, r, recompute=True))
    outs = [np.empty_like(s) for s in single]
    lma.image_many(ctx, [b for _, b in objs], ws[0].detectors, regions, outs)
    for o, s in zip(outs, single):
        assert np.array_equal(o, s)
