"""The tensor-core precision form (LMA_PREC_MIXED): the slice step's 32-point DFT stages as
split-FP16 (hi + lo) products on the tensor cores, accumulated in FP32, against the FP64
oracle and against the FP32 (complex64) path.

Tolerances. The split keeps about 22 significant bits per operand and the accumulation is
FP32, so the exit waves are held to the complex64 bound (5e-5 of their peak after up to 50
slices), against the oracle and against the FP32 path's exit waves (measured 1.4e-5 after 50
slices at 512^2); images to the mixed-
precision contract, 1e-3 relative per pixel, or three times the complex64 floor of the same pixels
(``parity_floor``), whichever is larger.
"""
import dataclasses

import numpy as np
import pytest

from oracle import lma_oracle as O
from oracle import pool as OP
from paper_2310_16829_gb300 import lma, workloads as WL
from parity_floor import assert_floor, oracles

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-3


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lma.Context(0)


def _mixed(w):
    return dataclasses.replace(w, basis=dataclasses.replace(w.basis, precision=WL.PREC_MIXED))


@pytest.mark.parametrize("case", ["simple_cubic", "perovskite_512", "odd_origins", "wide_band"])
def test_tensor_core_exit_waves_match_oracle_and_fp32(ctx, case):
    """Exit waves of the tensor-core slice kernel: pruned (2/3 bandlimit) and general (0.7)
    instantiations, even and odd window origins, windows that wrap around the cell edge."""
    if case == "perovskite_512":
        w = WL.perovskite_workload(n_phonons=1)
        idx = (0, 127, 128 * 64 + 70, 128 * 128 - 1)
    else:
        w = WL.simple_cubic_workload()
        idx = (0, 31, 517, 1023)
        if case == "odd_origins":
            w.basis.in_offset_px = (1, 3)
        if case == "wide_band":
            w = dataclasses.replace(w, grid=dataclasses.replace(w.grid, bandlimit_frac=0.7))
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    tc = lma.Basis(ctx, spec, w.probe, _mixed(w).basis)
    fp = lma.Basis(ctx, spec, w.probe, w.basis)
    tc.propagate(0)
    fp.propagate(0)
    orc = oracles(w)[0]
    for i in idx:
        got, f32, ref = tc.exit_wave(i), fp.exit_wave(i), orc.exit_wave(0, i)
        peak = np.max(np.abs(ref))
        assert np.max(np.abs(got - ref)) < 5e-5 * peak, (case, i, np.max(np.abs(got - ref)) / peak)
        assert np.max(np.abs(got - f32)) < 5e-5 * peak, (case, i, np.max(np.abs(got - f32)) / peak)


def test_tensor_core_image_simple_cubic(ctx):
    w = WL.simple_cubic_workload()
    dets = [WL.Detector(0.0, 0.02), WL.Detector(0.02, 0.06), WL.Detector(0.06, 0.2)]
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, _mixed(w).basis)
    img = basis.image(dets, w.region).reshape(3, -1)
    probes = O.region_probes(0, 0, 16, 16, (8, 8), 128, 128)
    orc, emu = oracles(w)
    ref = orc.image(dets, probes)
    assert_floor(img, ref, emu.image(dets, probes), tol=MIXED_TOL, label="tensor cores, simple cubic")
    assert np.max(np.abs(img[:2] - ref[:2]) / ref[:2]) < 1e-4


@pytest.mark.slow
def test_tensor_core_image_perovskite_512_two_configurations(ctx):
    """The benchmark workload's specimen with two configurations in the benchmark's launch
    configuration: two 16 x 16-probe subregions (one wrapping the cell edge) against the
    oracle, HAADF within the mixed-precision bound 1e-3 (or three times the complex64 floor)."""
    w = WL.perovskite_workload(n_phonons=2)
    dets = [WL.Detector(0.0, 0.025), WL.Detector(0.07, 0.2)]
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, _mixed(w).basis)
    img = basis.image(dets, w.region, recompute=True)
    subs = [(0, 0), (56, 24)]
    probes = np.concatenate([OP.subregion_probes(w.region, a0, b0, 16, 512, 512) for a0, b0 in subs])
    r = OP.readings(w, dets, probes, phis=[0, 1], c64=True)
    got = np.concatenate([img[:, b0:b0 + 16, a0:a0 + 16].reshape(2, -1) for a0, b0 in subs], axis=1)
    assert_floor(got, r["ref"], r["emu"], tol=MIXED_TOL, label="tensor cores, 512 two configurations")
    assert np.max(np.abs(got[0] - r["ref"][0]) / r["ref"][0]) < 1e-4


def test_tensor_core_batched_and_partitioned_images_equal_plain(ctx):
    """The tensor-core form through the other callers of the slice step: the memory-bounded
    partitioned image and a phonon batch of 1 give the same bits as the plain image."""
    w = WL.perovskite_workload(cells=5, nx=256, n_slices=6, n_phonons=2, seed_base=2900)
    w = _mixed(w)
    region = WL.Region(250, 60, 6, 5, (4, 4))
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    plain = lma.Basis(ctx, spec, w.probe, w.basis).image(w.detectors, region, recompute=True)
    one = lma.Basis(ctx, spec, w.probe, dataclasses.replace(w.basis, phonon_batch=1)).image(
        w.detectors, region, recompute=True)
    assert np.array_equal(plain, one)
    part = lma.Basis(ctx, spec, w.probe, w.basis).image_partitioned(w.detectors, region, lma.LMA_PART_ROWS, 64)
    assert np.array_equal(plain, part)
