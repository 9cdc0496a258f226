"""Trigonometric input waves (Sec. 4.2.3: the tensor product phi_n(x) phi_n(y) and the radial
phi_n(|v|)) through the GPU path against the FP64 oracle. Readings are held to 1e-4 relative
error, or to three times the complex64 floor of the same image (``parity_floor``)."""
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


@pytest.mark.parametrize("kind", [WL.BASIS_TRIG, WL.BASIS_TRIG_RADIAL])
def test_trig_input_waves_match_oracle(ctx, kind):
    for w, region in ((WL.simple_cubic_workload(), WL.Region(0, 0, 3, 2, (8, 8))),
                      (WL.perovskite_workload(cells=5, nx=256, n_slices=5, n_phonons=1, seed_base=2800),
                       WL.Region(252, 20, 3, 3, (4, 4)))):
        w.basis.kind = kind
        dets = [WL.Detector(0.0, 0.02), WL.Detector(0.06, 0.2)]
        spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
        basis = lma.Basis(ctx, spec, w.probe, w.basis)
        got = basis.image(dets, region, recompute=True).reshape(2, -1)
        orc, emu = oracles(w)
        probes = O.region_probes(region.px0, region.py0, region.npx, region.npy, region.spacing_px,
                                 w.grid.nx, w.grid.ny)
        assert_floor(got, orc.image(dets, probes), emu.image(dets, probes), label=f"{w.name} {kind}")


def test_closed_form_trig_coefficients_image_matches_oracle(ctx):
    """LMA_COEF_TRIG_CLOSED (Sec. 2, Sec. 4.2.3: coefficients from the probe's Fourier
    coefficients, no least squares) through synthesis and detection on the GPU against the
    oracle's image with the same closed form; and, with all the other inputs fixed, the image
    differs from the least-squares one (the coefficients are really the closed form)."""
    for w, region in ((WL.simple_cubic_workload(), WL.Region(0, 0, 3, 2, (8, 8))),
                      (WL.perovskite_workload(cells=5, nx=256, n_slices=5, n_phonons=1, seed_base=2800),
                       WL.Region(252, 20, 3, 3, (4, 4)))):
        w.basis.kind = WL.BASIS_TRIG
        w.basis.coef_mode = 1
        dets = [WL.Detector(0.0, 0.02), WL.Detector(0.06, 0.2)]
        spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
        basis = lma.Basis(ctx, spec, w.probe, w.basis)
        got = basis.image(dets, region, recompute=True).reshape(2, -1)
        orc, emu = oracles(w)
        probes = O.region_probes(region.px0, region.py0, region.npx, region.npy, region.spacing_px,
                                 w.grid.nx, w.grid.ny)
        ref = orc.image(dets, probes)
        assert_floor(got, ref, emu.image(dets, probes), label=f"{w.name} closed form")
        w.basis.coef_mode = 0
        ls = lma.Basis(ctx, spec, w.probe, w.basis).image(dets, region, recompute=True).reshape(2, -1)
        assert np.max(np.abs(ls - got) / np.maximum(ref, 1e-4)) > 1e-3, w.name
