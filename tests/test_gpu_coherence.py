"""Partial coherence on the GPU: one set of exit waves read out for several probe variants
(defocus, C_s) and averaged, against the FP64 oracle, against separate images computed with
one basis per variant, and against the plain image for a single base variant."""
import numpy as np
import pytest

from oracle import lma_oracle as O
from paper_2310_16829_gb300 import lma, workloads as WL
from parity_floor import assert_floor, oracles

pytestmark = pytest.mark.gpu

VARIANTS = [(-40.0, 0.0, 1.0), (0.0, 0.0, 2.0), (60.0, 0.0, 0.5)]


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lma.Context(0)


def _workload():
    w = WL.perovskite_workload(cells=5, nx=256, n_slices=6, n_phonons=2, seed_base=2600)
    return w.with_region(WL.Region(250, 100, 5, 3, (4, 4)))


def test_coherent_image_matches_oracle(ctx):
    w = _workload()
    dets = [WL.Detector(0.0, 0.02), WL.Detector(0.07, 0.2)]
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    got = basis.image_coherent(VARIANTS, dets, w.region, recompute=True).reshape(2, -1)
    orc, emu = oracles(w)
    probes = O.region_probes(250, 100, 5, 3, (4, 4), w.grid.nx, w.grid.ny)
    ref = orc.image_coherent(dets, probes, VARIANTS)
    # bright field: 1e-4 relative; the 6-slice slab's HAADF (1e-7..1e-6 of the beam) against
    # three times the complex64 floor of the same focal series
    assert np.max(np.abs(got[0] - ref[0]) / ref[0]) < 1e-4
    assert_floor(got, ref, emu.image_coherent(dets, probes, VARIANTS), label="coherent")


def test_coherent_image_equals_separate_variant_images(ctx):
    w = _workload()
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    got = basis.image_coherent(VARIANTS, w.detectors, w.region, recompute=True)
    wsum = sum(v[2] for v in VARIANTS)
    ref = np.zeros_like(got)
    for dz, cs, wt in VARIANTS:
        # Gaussian input waves depend on the aperture only: each variant's own basis has the
        # same exit waves and gives that variant's image
        pv = WL.Probe(w.probe.alpha_max, cs=cs, defocus=dz)
        bv = lma.Basis(ctx, spec, pv, w.basis)
        ref += wt / wsum * bv.image(w.detectors, w.region, recompute=True)
        bv.close()
    assert np.max(np.abs(got - ref) / ref) < 1e-12
    # one variant equal to the basis probe: the plain image, bit for bit
    one = basis.image_coherent([(w.probe.defocus, w.probe.cs, 1.0)], w.detectors, w.region)
    assert np.array_equal(one, basis.image(w.detectors, w.region))


def test_coherent_image_rejects_another_aperture(ctx):
    w = _workload()
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    basis.alpha_max = w.probe.alpha_max * 1.1      # variants built with another aperture
    with pytest.raises(lma.LmaError) as e:
        basis.image_coherent(VARIANTS, w.detectors, w.region)
    assert e.value.status == lma.LMA_ERR_INVALID
    basis.alpha_max = w.probe.alpha_max
    with pytest.raises(lma.LmaError):
        basis.image_coherent([(0.0, 0.0, 0.0)], w.detectors, w.region)
