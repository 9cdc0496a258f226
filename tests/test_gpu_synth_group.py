"""Grouped synthesis (step a4, Sec. 4.2.2): Psi_p = sum_j alpha_j U_{i_j} for groups of up to
4 neighbouring probes, each exit-wave element loaded once for all the group's probes that use
it, then a detection pass over the probe waves. Both forms sum every probe's terms in ascending
translate index, so the grouped form gives the readings of the per-probe gather bit for bit:
annuli (2D), rings (3D), patterns (4D), the FP16 store, windows W = 64 and 256, ragged groups at
the region's edges, several chunks of group rows, and a region that wraps around the cell.
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


def _both(ctx, fn):
    """fn() under the gather and under the grouped form (the context's form restored after)."""
    try:
        ctx.set_synth_mode(lma.LMA_SYNTH_GATHER)
        g = fn()
        ctx.set_synth_mode(lma.LMA_SYNTH_GROUPED)
        q = fn()
    finally:
        ctx.set_synth_mode(lma.LMA_SYNTH_AUTO)
    return g, q


def _objects(ctx, w):
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    return spec, lma.Basis(ctx, spec, w.probe, w.basis)


@pytest.mark.parametrize("case", ["w128_ragged", "w128_spacing8_wrap", "spacing_3_5", "case2_spacing2", "w64", "w256",
                                  "fp16_store", "L12", "L64"])
def test_grouped_equals_gather_bitwise(ctx, case):
    w = WL.perovskite_workload(cells=5, nx=256, n_slices=6, n_phonons=2, seed_base=5100)
    region = WL.Region(3, 5, 37, 23, (4, 4))            # 37 x 23 probes: ragged groups on two sides
    if case == "w128_spacing8_wrap":
        region = WL.Region(230, 200, 9, 7, (8, 8))      # wraps around the cell edge
    elif case == "w64":
        w = dataclasses.replace(w, basis=dataclasses.replace(w.basis, window=64))
    elif case == "w256":
        w = dataclasses.replace(w, basis=dataclasses.replace(w.basis, window=256))
        region = WL.Region(40, 60, 13, 10, (4, 4))
    elif case == "fp16_store":
        w = dataclasses.replace(w, basis=dataclasses.replace(w.basis, precision=WL.PREC_FP16_STORE))
    elif case == "spacing_3_5":
        region = WL.Region(7, 2, 11, 9, (3, 5))         # many coefficient sets, odd placements
    elif case == "case2_spacing2":
        region = WL.Region(0, 0, 18, 14, (2, 2))        # P = c R (Case 2): four coefficient sets
    elif case == "L12":
        w = dataclasses.replace(w, basis=dataclasses.replace(w.basis, L=12))
    elif case == "L64":
        w = dataclasses.replace(w, basis=dataclasses.replace(w.basis, L=64))   # groups of 4 x 64 entries
    spec, basis = _objects(ctx, w)
    dets = [WL.Detector(0.0, 0.02), WL.Detector(0.03, 0.06), WL.Detector(0.07, 0.2)]
    g, q = _both(ctx, lambda: basis.image(dets, region, recompute=True))
    assert np.all(np.isfinite(g)) and np.max(g) > 0
    assert np.array_equal(g, q), case


def test_grouped_rings_and_patterns_equal_gather(ctx):
    w = WL.perovskite_workload(cells=5, nx=256, n_slices=4, n_phonons=2, seed_base=5200)
    region = WL.Region(10, 20, 14, 9, (4, 4))
    spec, basis = _objects(ctx, w)
    g, q = _both(ctx, lambda: basis.image_rings(0.01, 12, region, recompute=True))
    assert np.array_equal(g, q)
    g, q = _both(ctx, lambda: basis.image_4d(6, 5, region, recompute=True))
    assert np.array_equal(g, q)


def test_grouped_chunks_of_group_rows_equal_one_launch(ctx):
    """A buffer limit of three group rows' waves splits the region into chunks; the readings
    are those of the unchunked grouped form and of the gather."""
    w = WL.perovskite_workload(cells=5, nx=256, n_slices=4, n_phonons=2, seed_base=5300)
    region = WL.Region(0, 0, 21, 29, (4, 4))
    spec, basis = _objects(ctx, w)
    g, one = _both(ctx, lambda: basis.image(w.detectors, region, recompute=True))
    ctx.set_synth_buffer_limit(3 * 4 * region.npx * 128 * 128 * 8)
    try:
        _, chunked = _both(ctx, lambda: basis.image(w.detectors, region, recompute=True))
    finally:
        ctx.set_synth_buffer_limit(0)
    assert np.array_equal(one, g)
    assert np.array_equal(chunked, g)
    with pytest.raises(lma.LmaError):
        ctx.set_synth_buffer_limit(-1)
    with pytest.raises(lma.LmaError):
        ctx.set_synth_mode(2)


def test_grouped_image_matches_oracle(ctx):
    """The grouped form against the FP64 oracle on a ragged region that wraps around the cell."""
    w = WL.perovskite_workload(cells=5, nx=256, n_slices=6, n_phonons=2, seed_base=5400)
    r = WL.Region(240, 230, 7, 6, (4, 4))
    spec, basis = _objects(ctx, w)
    ctx.set_synth_mode(lma.LMA_SYNTH_GROUPED)
    try:
        img = basis.image(w.detectors, r, recompute=True).reshape(len(w.detectors), -1)
    finally:
        ctx.set_synth_mode(lma.LMA_SYNTH_AUTO)
    orc, emu = oracles(w)
    probes = O.region_probes(r.px0, r.py0, r.npx, r.npy, r.spacing_px, w.grid.nx, w.grid.ny)
    assert_floor(img, orc.image(w.detectors, probes), emu.image(w.detectors, probes), label="grouped")
