"""Real-space propagation (Sec. 3.2: the propagation step as a convolution with q on K1 x K2
pixels) on the GPU against the FP64 oracle with the same kernel, and the Fourier path left
intact afterwards.

Tolerance: 1e-4 relative per reading, or three times the complex64 floor of the same image
(``parity_floor``), with the oracle's real-space pipeline restated in complex64.
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




@pytest.mark.parametrize("case", ["simple_cubic", "perovskite", "square_3", "square_5", "wide_15x3",
                                  "wide_25x11"])
def test_realspace_image_matches_oracle(ctx, case):
    """K1 != K2 in the perovskite and wide cases, so a transposed kernel fails; kernels wider
    than 13 columns take their row segment in two pieces (13 + 2 and 13 + 12 columns); the
    3 x 3 and 5 x 5 kernels run the instantiations with K2 fixed at compile time."""
    if case == "simple_cubic":
        w = WL.simple_cubic_workload()
        region, K = WL.Region(0, 0, 3, 2, (8, 8)), (7, 7)
    else:
        w = WL.perovskite_workload(cells=5, nx=256, n_slices=5, n_phonons=2, seed_base=2700)
        region, K = WL.Region(250, 60, 4, 3, (4, 4)), {"perovskite": (5, 9), "square_3": (3, 3), "square_5": (5, 5),
                                                       "wide_15x3": (15, 3), "wide_25x11": (25, 11)}[case]
    dets = [WL.Detector(0.0, 0.02), WL.Detector(0.06, 0.2)]
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    got = basis.image_realspace(K[0], K[1], dets, region).reshape(2, -1)
    probes = O.region_probes(region.px0, region.py0, region.npx, region.npy, region.spacing_px,
                             w.grid.nx, w.grid.ny)
    orc, emu = oracles(w, realspace=K)
    assert_floor(got, orc.image(dets, probes), emu.image(dets, probes), label=f"real space {case}")
    # the Fourier image afterwards: unchanged bits (the stored waves were marked stale)
    fourier = basis.image(dets, region)
    spec2 = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    fresh = lma.Basis(ctx, spec2, w.probe, w.basis).image(dets, region)
    assert np.array_equal(fourier, fresh)
    assert not np.array_equal(fourier, got.reshape(fourier.shape))


def test_realspace_arguments(ctx):
    w = WL.simple_cubic_workload()
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    region = WL.Region(0, 0, 2, 2, (8, 8))
    for K1, K2 in ((4, 5), (27, 5), (1, 5), (5, 27), (5, 4)):
        with pytest.raises(lma.LmaError) as e:
            basis.image_realspace(K1, K2, w.detectors, region)
        assert e.value.status == lma.LMA_ERR_INVALID
