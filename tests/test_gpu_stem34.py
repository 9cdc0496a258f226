"""GPU parity of the 3D STEM (rings) and 4D STEM (diffraction pattern) readouts of Sec. 3.1
against the FP64 oracle, and their consistency with the 2D image of the same exit waves.

Tolerance: 1e-4 relative per reading (ring reading or pattern pixel), or three times the
complex64 floor of the same readout (``parity_floor``: the oracle's readout restated in
complex64 on the same inputs); pixels outside the bandlimit are exactly zero on both sides.
"""
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


def _probes(region, w):
    return O.region_probes(region.px0, region.py0, region.npx, region.npy, region.spacing_px,
                           w.grid.nx, w.grid.ny)


def _perovskite():
    w = WL.perovskite_workload(cells=5, nx=256, n_slices=8, n_phonons=2, seed_base=2300)
    return w.with_region(WL.Region(250, 12, 5, 3, (4, 4)))   # wraps around the cell edge


def test_rings_match_oracle_simple_cubic(ctx):
    w = WL.simple_cubic_workload()
    region = WL.Region(0, 0, 3, 2, (8, 8))
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    got = basis.image_rings(0.01, 7, region, recompute=True).reshape(7, -1)
    orc, emu = oracles(w)
    assert_floor(got, orc.image_rings(0.01, 7, _probes(region, w)), emu.image_rings(0.01, 7, _probes(region, w)),
                 label="rings simple cubic")
    # the same rings twice: the fixed-order sums reproduce bit for bit
    again = basis.image_rings(0.01, 7, region).reshape(7, -1)
    assert np.array_equal(got, again)


def test_rings_match_oracle_perovskite_two_configurations(ctx):
    w = _perovskite()
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    got = basis.image_rings(0.012, 8, w.region, recompute=True).reshape(8, -1)
    orc, emu = oracles(w)
    assert_floor(got, orc.image_rings(0.012, 8, _probes(w.region, w)),
                 emu.image_rings(0.012, 8, _probes(w.region, w)), label="rings perovskite")


def test_rings_tile_the_2d_annulus(ctx):
    w = _perovskite()
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    rings = basis.image_rings(0.01, 9, w.region, recompute=True)
    two_d = basis.image([WL.Detector(0.02, 0.06), WL.Detector(0.0, 0.09)], w.region)
    assert np.max(np.abs(rings[2:6].sum(axis=0) / two_d[0] - 1)) < 1e-5
    assert np.max(np.abs(rings.sum(axis=0) / two_d[1] - 1)) < 1e-5


def test_pattern_matches_oracle(ctx):
    for w, region, A, B in ((WL.simple_cubic_workload(), WL.Region(0, 0, 2, 2, (8, 8)), 20, 12),
                            (_perovskite(), WL.Region(250, 12, 3, 2, (4, 4)), 45, 30)):
        spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
        basis = lma.Basis(ctx, spec, w.probe, w.basis)
        got = basis.image_4d(A, B, region, recompute=True)
        assert got.shape == (region.npy, region.npx, 2 * B + 1, 2 * A + 1)
        got = got.reshape(region.npy * region.npx, 2 * B + 1, 2 * A + 1).astype(np.float64)
        orc, emu = oracles(w)
        ref = orc.image_4d(A, B, _probes(region, w))
        e = emu.image_4d(A, B, _probes(region, w))
        ia, ib = np.arange(-A, A + 1), np.arange(-B, B + 1)
        band = 9 * (ia[None, :] ** 2 + ib[:, None] ** 2) <= w.basis.det_window ** 2
        for g, r, ee in zip(got, ref, e):
            # each probe's pattern is one row of the criterion
            assert_floor(g.reshape(1, -1), r.reshape(1, -1), ee.reshape(1, -1), label="pattern")
            # outside the bandlimit the pattern is exactly zero on both sides
            assert np.all(g[~band] == 0.0) and np.all(r[~band] == 0.0)


def test_pattern_summed_over_an_annulus_is_the_2d_reading(ctx):
    w = _perovskite()
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    A = w.basis.det_window // 2 - 1
    pat = basis.image_4d(A, A, w.region, recompute=True).astype(np.float64)
    r1, r2 = 0.02, 0.06
    two_d = basis.image([WL.Detector(r1, r2)], w.region)[0]
    dx = w.grid.lx / w.grid.nx
    ia = np.arange(-A, A + 1)
    ang = w.grid.lam * np.hypot(ia[None, :], ia[:, None]) / (w.basis.det_window * dx)
    sel = (ang >= r1) & (ang < r2)
    assert np.max(np.abs(pat[:, :, sel].sum(axis=-1) / two_d - 1)) < 1e-5


def test_invalid_3d_4d_arguments_are_rejected(ctx):
    w = WL.simple_cubic_workload()
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    region = WL.Region(0, 0, 2, 2, (8, 8))
    for args in ((0.01, 0), (0.0, 4), (-0.01, 4), (0.01, lma.LMA_MAX_RINGS + 1)):
        with pytest.raises(lma.LmaError) as e:
            basis.image_rings(*args, region, out=np.empty((max(1, args[1]), 2, 2)))
        assert e.value.status == lma.LMA_ERR_INVALID
    for hx, hy in ((64, 4), (4, 64), (-1, 0)):
        with pytest.raises(lma.LmaError) as e:
            basis.image_4d(hx, hy, region, out=np.empty((2, 2, 1, 1), np.float32))
        assert e.value.status == lma.LMA_ERR_INVALID
