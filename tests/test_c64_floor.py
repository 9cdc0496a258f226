"""The complex64 restatement of the oracle (``oracle.lma_c64``) and the oracle's process pool
(``oracle.pool``), on the CPU.

The restatement is what the GPU parity tests measure the rounding floor of complex64 with,
so it is pinned to things other than itself: its DFT against numpy's FP64 DFT, its arrays
really being single precision (a nonzero error of the size single precision makes), and its
image against the FP64 oracle's to single-precision accuracy. The pool is pinned bit for bit
to ``LmaOracle.image``. The floor itself is reported on the simple-cubic toy crystal and on a
16 x 16-probe block of one ABO3 configuration.
"""
import numpy as np
import pytest

from oracle import lma_c64 as C
from oracle import lma_oracle as O
from oracle import pool as OP
from paper_2310_16829_gb300 import workloads as WL

EPS32 = 2.0 ** -24


def _oracles(w):
    out = []
    for cls in (O.LmaOracle, C.LmaOracleC64):
        orc = cls(O.params_from_workload(w))
        orc.set_specimen(w.phonons, w.potential.peak, w.potential.term_frac, w.potential.term_width,
                         w.potential.r_cut)
        out.append(orc)
    return out


def test_single_precision_dft_against_fp64():
    rng = np.random.default_rng(3)
    a = (rng.standard_normal((16, 12)) + 1j * rng.standard_normal((16, 12))).astype(np.complex64)
    got = C.dft2(a)
    assert got.dtype == np.complex64
    ref = np.fft.fft2(a.astype(np.complex128))
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    # a single-precision transform: an error of the order of the FP32 unit roundoff, not zero
    assert 1e-9 < err < 30 * EPS32
    back = C.idft2(got)
    assert back.dtype == np.complex64
    assert np.max(np.abs(back - a)) < 30 * EPS32 * np.max(np.abs(a))


def test_exit_waves_are_complex64_and_match_fp64_to_single_precision():
    w = WL.simple_cubic_workload()
    o64, o32 = _oracles(w)
    for i in (0, 517):
        u64, u32 = o64.exit_wave(0, i), o32.exit_wave(0, i)
        assert u32.dtype == np.complex64 and u64.dtype == np.complex128
        err = np.max(np.abs(u32 - u64)) / np.max(np.abs(u64))
        assert 1e-9 < err < 1e-5, err


def test_transposed_operand_in_the_restatement_would_show():
    """The restatement's image differs from the oracle's only by rounding: a wrong step
    (here a transposed transmission) moves it by far more than the floor."""
    w = WL.perovskite_workload(cells=5, nx=256, n_slices=4, n_phonons=1, seed_base=2800)
    o64, o32 = _oracles(w)
    dets = [WL.Detector(0.0, 0.02), WL.Detector(0.06, 0.2)]
    probes = O.region_probes(250, 60, 2, 2, (4, 4), 256, 256)
    ref, emu = o64.image(dets, probes), o32.image(dets, probes)
    assert np.max(np.abs(emu[0] - ref[0]) / ref[0]) < 1e-5
    o32._t32[0] = np.ascontiguousarray(np.swapaxes(o32.transmission_stack_c64(0), 1, 2))
    o32._U.clear()
    bad = o32.image(dets, probes)
    assert np.max(np.abs(bad[1] - ref[1]) / ref[1]) > 100 * np.max(np.abs(emu[1] - ref[1]) / ref[1])


def test_pool_readings_equal_the_oracle_bit_for_bit():
    w = WL.simple_cubic_workload()
    dets = [WL.Detector(0.0, 0.02), WL.Detector(0.06, 0.2)]
    probes = O.region_probes(3, 5, 4, 3, (3, 5), 128, 128)
    r = OP.readings(w, dets, probes, c64=True, workers=2)
    o64, o32 = _oracles(w)
    assert np.array_equal(r["ref"], o64.image(dets, probes))
    assert np.array_equal(r["emu"], o32.image(dets, probes))
    assert r["workers"] == 2 and r["translates"] > 0


def test_pool_phonon_average_equals_the_oracle_bit_for_bit():
    w = WL.perovskite_workload(cells=5, nx=256, n_slices=3, n_phonons=2, seed_base=2300)
    probes = O.region_probes(250, 12, 2, 2, (4, 4), 256, 256)
    r = OP.readings(w, w.detectors, probes, workers=3)
    assert np.array_equal(r["ref"], _oracles(w)[0].image(w.detectors, probes))
    one = OP.readings(w, w.detectors, probes, phis=[1], workers=2)
    o = _oracles(w)[0]
    masks = o.detector_masks(w.detectors)
    want = np.array([o.pixel(1, (int(p[0]), int(p[1])), masks) for p in probes]).T
    assert np.array_equal(one["ref"], want)


def test_complex64_floor_simple_cubic_haadf():
    """The floor on the toy crystal's clipped 60-67 mrad band (1e-7..1e-4 of the beam):
    complex64 arithmetic alone misses 1e-4 relative on its weakest readings, while its
    absolute error stays near 1e-9 of the beam and bright field stays far inside 1e-4."""
    w = WL.simple_cubic_workload()
    dets = [WL.Detector(0.0, 0.02), WL.Detector(0.06, 0.2)]
    probes = O.region_probes(0, 0, 16, 16, (8, 8), 128, 128)
    r = OP.readings(w, dets, probes, c64=True)
    ref, emu = r["ref"], r["emu"]
    rel = np.abs(emu - ref) / ref
    assert rel[0].max() < 1e-5
    assert rel[1].max() > 1e-4                  # the floor is real
    assert np.abs(emu[1] - ref[1]).max() < 3e-9
    kap = C.floor_scale(ref, emu)
    print(f"simple cubic: HAADF readings {ref[1].min():.2e}..{ref[1].max():.2e}, complex64 error "
          f"max {rel[1].max():.2e} relative, median {np.median(rel[1]):.2e}, kappa {kap[1]:.2e}")


@pytest.mark.slow
def test_complex64_floor_perovskite_one_configuration():
    """The floor on a 16 x 16-probe block of one ABO3 configuration (512^2, 50 slices; the
    benchmark workload's HAADF band, 7e-6..2e-4 of the beam): some readings miss 1e-4
    relative in complex64 arithmetic alone."""
    w = WL.perovskite_workload(n_phonons=1)
    dets = [WL.Detector(0.0, 0.025), WL.Detector(0.07, 0.2)]
    probes = OP.subregion_probes(w.region, 0, 0, 16, 512, 512)
    r = OP.readings(w, dets, probes, c64=True)
    ref, emu = r["ref"], r["emu"]
    rel = np.abs(emu - ref) / ref
    assert rel[0].max() < 3e-5
    assert 1e-5 < rel[1].max() < 1e-3
    kap = C.floor_scale(ref, emu)
    print(f"ABO3 one configuration: HAADF readings {ref[1].min():.2e}..{ref[1].max():.2e}, complex64 "
          f"error max {rel[1].max():.2e} relative, median {np.median(rel[1]):.2e}, kappa {kap[1]:.2e}")


def test_floor_bound_is_the_larger_of_the_two():
    ref = np.array([[1.0, 1e-6, 4e-8]])
    emu = np.array([[1.0 + 1e-6, 1e-6 + 2e-10, 4e-8 + 4e-11]])
    q = np.array([1e-6, 2e-10 / 1e-3, 4e-11 / 2e-4])
    kap = C.floor_scale(ref, emu)
    assert np.isclose(kap[0], max(q.max(), 3 * np.sqrt(np.mean(q * q))))
    b = C.floor_bound(ref, emu, 1e-4, 3.0)
    assert np.allclose(b[0], np.maximum(1e-4 * ref[0], 3 * kap[0] * np.sqrt(ref[0])))
    # a row of one reading: the envelope is three times its error
    assert np.isclose(C.floor_scale(np.array([[4e-6]]), np.array([[4e-6 + 2e-9]]))[0], 3 * 2e-9 / 2e-3)
