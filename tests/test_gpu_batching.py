"""GPU batching: configurations per launch, several specimens per call, graph replay.

Batching changes only how the work is grouped into launches, never the arithmetic
of one exit wave or one probe reading, and the average over configurations is
summed in configuration order. So every batched form must be bitwise equal to the
one-configuration-at-a-time image, and that image is held to the oracle.
"""
import numpy as np
import pytest

from oracle import lma_oracle as O
from paper_2310_16829_gb300 import lma, workloads as WL
from parity_floor import assert_floor, oracles

pytestmark = pytest.mark.gpu

PIXEL_TOL = 1e-4


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lma.Context(0)


def _uneven(seed_shift=0):
    """Three small specimens of uneven size: 128^2 (window = grid, cyclic), 256^2, 512^2
    with a region that wraps around the cell edge."""
    a = WL.perovskite_workload(cells=3, nx=128, n_slices=6, n_phonons=3,
                               seed_base=2000 + seed_shift, probes=8)
    b = WL.perovskite_workload(cells=5, nx=256, n_slices=8, n_phonons=3, seed_base=2100 + seed_shift)
    c = WL.perovskite_workload(cells=10, nx=512, n_slices=6, n_phonons=2, seed_base=2200 + seed_shift)
    b = b.with_region(WL.Region(40, 24, 12, 10, (4, 4)))
    c = c.with_region(WL.Region(500, 8, 9, 7, (4, 4)))
    return [a, b, c]


def _objects(ctx, w, phonon_batch=0):
    desc = WL.BasisDesc(**{**w.basis.__dict__, "phonon_batch": phonon_batch})
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    return spec, lma.Basis(ctx, spec, w.probe, desc)


def _dev_out(w):
    import torch
    return torch.empty((len(w.detectors), w.region.npy, w.region.npx), dtype=torch.float64,
                       device="cuda:0")


def test_phonon_batch_is_bitwise_neutral(ctx):
    w = _uneven()[1]
    imgs = []
    for pb, expect in ((1, 1), (2, 2), (0, 3)):
        spec, basis = _objects(ctx, w, pb)
        imgs.append(basis.image(w.detectors, w.region, recompute=True))
        assert basis.info().phonon_batch == expect
    assert np.array_equal(imgs[0], imgs[1]) and np.array_equal(imgs[0], imgs[2])


def test_batched_image_matches_oracle_sampled(ctx):
    # 3 configurations in batches of 2 + 1 (a ragged last batch)
    w = _uneven()[1]
    spec, basis = _objects(ctx, w, 2)
    img = basis.image(w.detectors, w.region, recompute=True)[0]
    sample = WL.sample_probes(w.region, 3, seed=11)
    pix = np.stack([w.region.px0 + sample[:, 0] * 4, w.region.py0 + sample[:, 1] * 4], axis=1)
    orc, emu = oracles(w)
    got = img[sample[:, 1], sample[:, 0]]
    # 8-slice slab: weak HAADF readings, against three times the complex64 floor of the same pixels
    assert_floor(got.reshape(1, -1), orc.image(w.detectors, pix), emu.image(w.detectors, pix),
                 label="batched")


def test_image_many_equals_single_images_and_graph_replays(ctx):
    import torch
    ws = _uneven()
    single = []
    for w in ws:
        spec, basis = _objects(ctx, w)
        single.append(basis.image(w.detectors, w.region, recompute=True))
    objs = [_objects(ctx, w) for w in ws]
    bases = [b for _, b in objs]
    regions = [w.region for w in ws]
    st = torch.cuda.Stream()
    # plain batched call, host outputs
    outs = [np.empty_like(s) for s in single]
    lma.image_many(ctx, bases, ws[0].detectors, regions, outs, stream=st)
    for o, s in zip(outs, single):
        assert np.array_equal(o, s)
    # graph: the first call runs and captures, later calls replay
    douts = [_dev_out(w) for w in ws]
    for call in range(3):
        for d in douts:
            d.fill_(-1.0)
        ctx.profile_enable(True)
        lma.image_many(ctx, bases, ws[0].detectors, regions, douts, graph=True, stream=st)
        st.synchronize()
        prof = ctx.profile_read()
        ctx.profile_enable(False)
        for d, s in zip(douts, single):
            assert np.array_equal(d.cpu().numpy(), s), call
        if call > 0:
            # a replay issues no launch through the host path
            assert prof["slice"]["launches"] == 0 and prof["synth"]["launches"] == 0


def test_graph_replay_sees_new_atoms(ctx):
    import torch
    ws = _uneven()
    objs = [_objects(ctx, w) for w in ws]
    bases = [b for _, b in objs]
    regions = [w.region for w in ws]
    st = torch.cuda.Stream()
    douts = [_dev_out(w) for w in ws]
    lma.image_many(ctx, bases, ws[0].detectors, regions, douts, graph=True, stream=st)
    st.synchronize()
    first = [d.cpu().numpy() for d in douts]
    # new frozen-phonon draws of the same crystals (same atom counts): a replay
    new = _uneven(seed_shift=3000)
    for (spec, _), w2 in zip(objs, new):
        spec.set_atoms(w2.phonons)
    lma.image_many(ctx, bases, ws[0].detectors, regions, douts, graph=True, stream=st)
    st.synchronize()
    for k, w2 in enumerate(new):
        spec, basis = _objects(ctx, w2)
        ref = basis.image(w2.detectors, w2.region, recompute=True)
        got = douts[k].cpu().numpy()
        assert np.array_equal(got, ref), k
        assert not np.array_equal(got, first[k]), k


def test_image_many_graph_rejects_host_outputs(ctx):
    import torch
    ws = _uneven()[:1]
    spec, basis = _objects(ctx, ws[0])
    out = np.empty((1, ws[0].region.npy, ws[0].region.npx))
    with pytest.raises(lma.LmaError) as e:
        lma.image_many(ctx, [basis], ws[0].detectors, [ws[0].region], [out], graph=True,
                       stream=torch.cuda.Stream())
    assert e.value.status == lma.LMA_ERR_INVALID
    with pytest.raises(lma.LmaError) as e:
        lma.image_many(ctx, [basis], ws[0].detectors, [ws[0].region], [_dev_out(ws[0])],
                       recompute=False, graph=True, stream=torch.cuda.Stream())
    assert e.value.status == lma.LMA_ERR_INVALID


def test_slice_launch_modes_are_bitwise_equal(ctx):
    """One CTA per translate, persistent with a fixed stride, persistent with dynamic
    fetch: the same exit waves, so the same images (one specimen and three at once)."""
    ws = _uneven()
    objs = [_objects(ctx, w) for w in ws]
    bases = [b for _, b in objs]
    regions = [w.region for w in ws]
    results = {}
    try:
        for mode in (lma.LMA_SLICE_ONE_PER_ITEM, lma.LMA_SLICE_PERSISTENT, lma.LMA_SLICE_DYNAMIC):
            ctx.set_slice_mode(mode)
            one = bases[1].image(ws[1].detectors, ws[1].region, recompute=True)
            outs = [np.empty((1, w.region.npy, w.region.npx)) for w in ws]
            lma.image_many(ctx, bases, ws[0].detectors, regions, outs)
            results[mode] = (one, outs)
    finally:
        ctx.set_slice_mode(lma.LMA_SLICE_AUTO)
    ref_one, ref_outs = results[lma.LMA_SLICE_ONE_PER_ITEM]
    assert np.array_equal(ref_outs[1], ref_one)
    for mode, (one, outs) in results.items():
        assert np.array_equal(one, ref_one), mode
        for o, r in zip(outs, ref_outs):
            assert np.array_equal(o, r), mode
    with pytest.raises(lma.LmaError):
        ctx.set_slice_mode(7)


def test_autotune_times_every_mode_and_keeps_results():
    import torch
    assert torch.cuda.is_available()
    c = lma.Context(0)
    ws = _uneven()
    objs = [_objects(c, w) for w in ws]
    bases = [b for _, b in objs]
    regions = [w.region for w in ws]
    plain = [np.empty((1, w.region.npy, w.region.npx)) for w in ws]
    lma.image_many(c, bases, ws[0].detectors, regions, plain)
    assert c.tuning() == []
    tuned = [np.empty_like(p) for p in plain]
    lma.image_many(c, bases, ws[0].detectors, regions, tuned, autotune=True)
    for t, p in zip(tuned, plain):
        assert np.array_equal(t, p)
    recs = c.tuning()
    # one fused launch: three specimens, complex64 store, even window origins
    assert len(recs) == 1
    r = recs[0]
    assert r["n_jobs"] == 3 and not r["half"] and r["even"]
    assert r["n_items"] > 0 and r["translate_slices"] >= 6 * r["n_items"]
    assert all(v > 0 for v in r["ms"].values())
    assert r["mode"] == min(r["ms"], key=r["ms"].get)
    # the synthesis of each specimen is tuned as well: every strip width and grid timed once,
    # the fastest kept (the readings above are those of the untuned call, bit for bit)
    srecs = c.synth_tuning()
    assert len(srecs) == len(ws)
    for sr, w in zip(srecs, ws):
        assert sr["readout"] == "annuli" and not sr["half"] and sr["window"] == w.basis.window
        assert sr["n_items"] == w.region.npx * w.region.npy * len(w.phonons)
        # six gather variants, and two group shapes where the windows are not periodic
        periodic = w.grid.nx == w.basis.window == 128 and w.grid.ny == 128
        assert len(sr["ms"]) == (6 if periodic else 8) and all(v > 0 for v in sr["ms"].values())
        if sr["grouped"]:
            chosen = f"grouped_{sr['group'][0]}x{sr['group'][1]}"
        else:
            chosen = f"strip{sr['strip']}_{'persistent' if sr['persistent'] else 'per_probe'}"
        assert chosen == min(sr["ms"], key=sr["ms"].get)
    # a second tuned call reuses the choices, with the same bits
    again = [np.empty_like(p) for p in plain]
    lma.image_many(c, bases, ws[0].detectors, regions, again, autotune=True)
    assert len(c.tuning()) == 1 and len(c.synth_tuning()) == len(ws)
    for t, p in zip(again, plain):
        assert np.array_equal(t, p)
    c.close()
