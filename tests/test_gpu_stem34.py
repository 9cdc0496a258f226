"""GPU parity of the 3D STEM (rings) and 4D STEM (diffraction pattern) readouts of Sec. 3.1
against the FP64 oracle, and their consistency with the 2D image of the same exit waves.

Tolerances (the complex64 rounding floor of the 2D FFTs reaches every reading as an
absolute error of 1e-10 to a few 1e-9 of the incident intensity): every ring reading is
held to 1e-4 x max(reading, FLOOR) with FLOOR = 1e-4 of the beam, i.e. 1e-4 relative for
readings above 1e-4 of the beam and 1e-8 absolute below. Thin rings at the band edge
were measured at 4-5e-9 (84-86 mrad sliver) and 1.5e-10 on readings of 1e-7. Pattern
pixels are single |DFT|^2 values: each is held to 1e-4 of its pattern's maximum.
"""
import numpy as np
import pytest

from oracle import lma_oracle as O
from paper_2310_16829_gb300 import lma, workloads as WL

pytestmark = pytest.mark.gpu

TOL = 1e-4
FLOOR = 1e-4


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lma.Context(0)


def _oracle(w):
    orc = O.LmaOracle(O.params_from_workload(w))
    orc.set_specimen(w.phonons, w.potential.peak, w.potential.term_frac, w.potential.term_width,
                     w.potential.r_cut)
    return orc


def _probes(region, w):
    return O.region_probes(region.px0, region.py0, region.npx, region.npy, region.spacing_px,
                           w.grid.nx, w.grid.ny)


def _assert_readings(got, ref):
    got, ref = np.asarray(got), np.asarray(ref)
    err = np.abs(got - ref) / np.maximum(ref, FLOOR)
    assert err.max() < TOL, f"{err.max():.2e} of max(reading, {FLOOR})"


def _perovskite():
    w = WL.perovskite_workload(cells=5, nx=256, n_slices=8, n_phonons=2, seed_base=2300)
    return w.with_region(WL.Region(250, 12, 5, 3, (4, 4)))   # wraps around the cell edge


def test_rings_match_oracle_simple_cubic(ctx):
    w = WL.simple_cubic_workload()
    region = WL.Region(0, 0, 3, 2, (8, 8))
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    got = basis.image_rings(0.01, 7, region, recompute=True).reshape(7, -1)
    ref = _oracle(w).image_rings(0.01, 7, _probes(region, w))
    for a in range(7):
        _assert_readings(got[a], ref[a])
    # the same rings twice: the fixed-order sums reproduce bit for bit
    again = basis.image_rings(0.01, 7, region).reshape(7, -1)
    assert np.array_equal(got, again)


def test_rings_match_oracle_perovskite_two_configurations(ctx):
    w = _perovskite()
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    got = basis.image_rings(0.012, 8, w.region, recompute=True).reshape(8, -1)
    ref = _oracle(w).image_rings(0.012, 8, _probes(w.region, w))
    for a in range(8):
        _assert_readings(got[a], ref[a])


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
        ref = _oracle(w).image_4d(A, B, _probes(region, w))
        ia, ib = np.arange(-A, A + 1), np.arange(-B, B + 1)
        band = 9 * (ia[None, :] ** 2 + ib[:, None] ** 2) <= w.basis.det_window ** 2
        for g, r in zip(got, ref):
            assert np.abs(g - r).max() < TOL * r.max()
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
