"""Edge cases of the GPU path against the FP64 oracle: free space (no atoms), the extreme
numbers of input waves per probe (L = 1 and the maximum 64), a region of one probe, and a
non-square grid. Tolerances as in the parity tests: 1e-4 relative per reading, or three times the
complex64 floor of the same image (``parity_floor``); exit waves to 5e-5 of their peak."""
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


def _oracle(w):
    return oracles(w)[0]


def _image(ctx, w, dets, region):
    """GPU image, FP64 oracle image and the complex64 restatement's image of the region."""
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    got = basis.image(dets, region, recompute=True).reshape(len(dets), -1)
    probes = O.region_probes(region.px0, region.py0, region.npx, region.npy, region.spacing_px,
                             w.grid.nx, w.grid.ny)
    orc, emu = oracles(w)
    return got, (orc.image(dets, probes), emu.image(dets, probes)), basis


def _assert_readings(got, ref_emu):
    assert_floor(got, ref_emu[0], ref_emu[1])


def test_free_space_exit_waves_conserve_the_norm_and_match_the_oracle(ctx):
    """No atoms: t = 1, every exit wave is the input wave propagated through the specimen
    thickness; the Gaussian input wave lies inside the bandlimit, so its norm is conserved."""
    w = WL.simple_cubic_workload()
    w = dataclasses.replace(w, phonons=[WL.Atoms(np.zeros(0), np.zeros(0), np.zeros(0, np.int32),
                                                 np.zeros(0, np.int16))])
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    basis.propagate(0)
    orc = _oracle(w)
    for i in (0, 33, 1023):
        got = basis.exit_wave(i)
        ref = orc.exit_wave(0, i)
        assert np.max(np.abs(got - ref)) < 5e-5 * np.max(np.abs(ref)), i
    u0 = O.input_wave_window(0, 128, 128, 128, w.grid.dy, w.grid.dx, w.grid.lam, w.probe.alpha_max,
                             0.0, 0.0, 0.0)
    n0 = np.sum(np.abs(u0) ** 2)
    assert abs(np.sum(np.abs(basis.exit_wave(33).astype(np.complex128)) ** 2) / n0 - 1) < 1e-5
    dets = [WL.Detector(0.0, 0.02), WL.Detector(0.02, 0.06)]
    region = WL.Region(0, 0, 3, 2, (8, 8))
    got = basis.image(dets, region, recompute=True).reshape(2, -1)
    probes = O.region_probes(0, 0, 3, 2, (8, 8), 128, 128)
    _assert_readings(got, (orc.image(dets, probes), oracles(w)[1].image(dets, probes)))


@pytest.mark.parametrize("L", [1, 64])
def test_extreme_numbers_of_input_waves(ctx, L):
    w = WL.simple_cubic_workload()
    w.basis.L = L
    dets = [WL.Detector(0.0, 0.02), WL.Detector(0.02, 0.06)]
    got, ref, _ = _image(ctx, w, dets, WL.Region(3, 5, 3, 2, (8, 8)))
    _assert_readings(got, ref)


def test_region_of_one_probe(ctx):
    w = WL.perovskite_workload(cells=5, nx=256, n_slices=6, n_phonons=2, seed_base=2900)
    dets = [WL.Detector(0.0, 0.025), WL.Detector(0.07, 0.2)]
    got, ref, _ = _image(ctx, w, dets, WL.Region(255, 130, 1, 1, (4, 4)))
    _assert_readings(got, ref)


def test_non_square_grid(ctx):
    """256 x 128 pixels over 32 x 16 A: the window covers the whole period along y only."""
    w = WL.simple_cubic_workload()
    g = dataclasses.replace(w.grid, nx=256, lx=32.0)
    at = WL._layered_crystal(4.0, 8, 4, 10, [[(0.0, 0.0, 0)]], 0.0, None)
    w = dataclasses.replace(w, grid=g, phonons=[at])
    dets = [WL.Detector(0.0, 0.02), WL.Detector(0.02, 0.06)]
    got, ref, basis = _image(ctx, w, dets, WL.Region(250, 120, 4, 3, (4, 4)))
    _assert_readings(got, ref)
    assert basis.info().nax == 64 and basis.info().nay == 32


def test_odd_window_origins(ctx):
    """Input lattice offset (1, 3): every window origin is odd along x, so the slice kernel
    stages the transmission in 8-byte pieces (the other instantiation of its copy)."""
    w = WL.simple_cubic_workload()
    w.basis.in_offset_px = (1, 3)
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    basis.propagate(0)
    orc = _oracle(w)
    for i in (0, 31, 517, 1023):
        got = basis.exit_wave(i)
        ref = orc.exit_wave(0, i)
        assert np.max(np.abs(got - ref)) < 5e-5 * np.max(np.abs(ref)), i
    dets = [WL.Detector(0.0, 0.02), WL.Detector(0.02, 0.06)]
    got, ref, _ = _image(ctx, w, dets, WL.Region(5, 9, 3, 2, (8, 8)))
    _assert_readings(got, ref)


def test_fp16_store_readouts_are_consistent():
    """FP16 exit-wave store with the 3D (rings) and 4D (pattern) readouts: rings summed over an
    annulus and the pattern summed over it give the 2D reading of the same store (the FP16
    rounding is the same in all three), and a wide bandlimit (general slice kernel) keeps the
    bright field within 1e-3 of complex64."""
    import torch
    assert torch.cuda.is_available()
    ctx = lma.Context(0)
    w = WL.perovskite_workload(cells=5, nx=256, n_slices=8, n_phonons=2, seed_base=2300)
    w = w.with_region(WL.Region(250, 12, 5, 3, (4, 4)))
    w.basis.precision = WL.PREC_FP16_STORE
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    rings = basis.image_rings(0.01, 9, w.region, recompute=True)
    two_d = basis.image([WL.Detector(0.02, 0.06), WL.Detector(0.0, 0.09)], w.region)
    assert np.max(np.abs(rings[2:6].sum(axis=0) / two_d[0] - 1)) < 1e-5
    assert np.max(np.abs(rings.sum(axis=0) / two_d[1] - 1)) < 1e-5
    A = w.basis.det_window // 2 - 1
    pat = basis.image_4d(A, A, w.region, recompute=True).astype(np.float64)
    dx = w.grid.lx / w.grid.nx
    ia = np.arange(-A, A + 1)
    ang = w.grid.lam * np.hypot(ia[None, :], ia[:, None]) / (w.basis.det_window * dx)
    sel = (ang >= 0.02) & (ang < 0.06)
    assert np.max(np.abs(pat[:, :, sel].sum(axis=-1) / two_d[0] - 1)) < 1e-5
    # general (unpruned) slice kernel with the FP16 store: bandlimit radius 44.8 px
    wide = dataclasses.replace(w, grid=dataclasses.replace(w.grid, bandlimit_frac=0.7))
    spec_w = lma.Specimen(ctx, wide.grid, wide.potential, wide.phonons)
    bf = [WL.Detector(0.0, 0.02)]
    half = lma.Basis(ctx, spec_w, wide.probe, wide.basis).image(bf, wide.region, recompute=True)
    full = lma.Basis(ctx, spec_w, wide.probe, dataclasses.replace(wide.basis, precision=WL.PREC_C64)
                     ).image(bf, wide.region, recompute=True)
    assert np.max(np.abs(half / full - 1)) < 1e-3


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_gives_up_and_the_context_stays_usable(which):
    """The bounded mbarrier wait of the tensor-core and W = 256 slice kernels, run on a phase
    that nothing completes in one warp (0) and in the 16 warps of a CTA (1), gives up, and the
    call returns LMA_ERR_TIMEOUT. The status word is cleared: the next tensor-core image in the
    same context is bit for bit the image of a fresh context."""
    import time

    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c1 = lma.Context(0)
    t0 = time.perf_counter()
    st = c1.selftest_wait(which)
    dt = time.perf_counter() - t0
    assert st == lma.LMA_ERR_TIMEOUT, st
    assert "gave up a bounded wait" in c1.lib.lma_last_error(c1.h).decode()
    assert dt < 30.0, dt
    w = WL.simple_cubic_workload()
    w = dataclasses.replace(w, basis=dataclasses.replace(w.basis, precision=WL.PREC_MIXED))
    region = WL.Region(0, 0, 4, 4, (8, 8))

    def image(c):
        spec = lma.Specimen(c, w.grid, w.potential, w.phonons)
        basis = lma.Basis(c, spec, w.probe, w.basis)
        return basis.image(w.detectors, region, recompute=True)

    got = image(c1)
    ref = image(lma.Context(0))
    assert np.array_equal(got, ref)
