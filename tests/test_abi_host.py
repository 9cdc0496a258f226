"""CPU checks of the C-ABI library: exports and the host-side logic (no device compute).

The host-only context (device = -1) runs the FP64 coefficient builder, the
lattice geometry and the edit bookkeeping; these are compared with the oracle.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import lma_oracle as O
from paper_2310_16829_gb300 import lma, workloads as WL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "lma.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lma_[A-Za-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    lib = lma.load()
    declared = _header_functions()
    assert declared == sorted(lma.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def _host_objects(w):
    ctx = lma.Context(-1)
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    return ctx, spec, basis


def _check_coefficients(w, probes, tol=1e-9):
    ctx, spec, basis = _host_objects(w)
    orc = O.LmaOracle(O.params_from_workload(w))
    for (px, py) in probes:
        al, off, tr, err = basis.coefficients(px, py)
        cs, idx = orc.coefficient_set((px, py))
        assert np.array_equal(off, cs.offsets), (px, py)
        assert np.array_equal(tr, idx), (px, py)
        assert np.max(np.abs(al - cs.alpha)) < tol * np.max(np.abs(cs.alpha))
        assert abs(err[0] - cs.err_l2) < 1e-9 and abs(err[1] - cs.err_sup) < 1e-9
    return basis


def test_coefficients_match_oracle_periodic_window():
    w = WL.simple_cubic_workload()
    b = _check_coefficients(w, [(0, 0), (8, 120), (127, 3)])
    assert b.info().n_sets == 2   # (0,0) and (8,120) share a class; (127,3) has its own


def test_coefficients_match_oracle_case1_single_set():
    w = WL.simple_cubic_workload()
    ctx, spec, basis = _host_objects(w)
    for p in [(0, 0), (8, 16), (120, 64), (40, 40)]:
        basis.coefficients(*p)
    assert basis.info().n_sets == 1      # Case 1: one coefficient set for the whole probe lattice


def test_coefficients_match_oracle_case2_and_probe_basis():
    w = WL.simple_cubic_workload()
    w.basis.kind = WL.BASIS_PROBE
    w.basis.L = 9
    _check_coefficients(w, [(0, 0), (1, 2), (2, 2), (3, 1)], tol=1e-8)


def test_coefficients_match_oracle_on_a_512_grid():
    w = WL.perovskite_workload(n_phonons=1)
    _check_coefficients(w, [(0, 0), (508, 4)])


@pytest.mark.parametrize("W", [64, 256])
def test_coefficients_match_oracle_other_windows(W):
    """Input waves sampled on W x W windows (Sec. 4.2.1 option (ii)): the least squares over the
    union of the L windows, against the oracle with the same W."""
    w = WL.perovskite_workload(n_phonons=1)
    w = w.__class__(**{**w.__dict__, "basis": WL.BasisDesc(**{**w.basis.__dict__, "window": W})})
    b = _check_coefficients(w, [(0, 0), (508, 4)])
    assert b.info().window == W and b.info().exit_wave_bytes == 128 * 128 * W * W * 8


def test_basis_info_and_lattice_count():
    w = WL.perovskite_workload(n_phonons=1)
    ctx, spec, basis = _host_objects(w)
    i = basis.info()
    assert i.n_translates == 128 * 128 and i.nax == 128 and i.nay == 128
    assert abs(i.gauss_sigma - O.gaussian_width(w.grid.lam, w.probe.alpha_max)) < 1e-15
    assert i.exit_wave_bytes == 128 * 128 * 128 * 128 * 8


def test_validation_errors():
    w = WL.simple_cubic_workload()
    ctx = lma.Context(-1)
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    bad = [
        dict(in_spacing_px=(3, 4)),        # does not divide the grid
        dict(in_offset_px=(4, 0)),         # offset >= spacing
        dict(f=3),                         # does not divide R
        dict(L=0),
        dict(L=65),
    ]
    for kw in bad:
        d = WL.BasisDesc(**{**w.basis.__dict__, **kw})
        with pytest.raises(lma.LmaError) as e:
            lma.Basis(ctx, spec, w.probe, d)
        assert e.value.status == lma.LMA_ERR_INVALID, kw
    for kw in (dict(window=32), dict(det_window=64), dict(window=256)):   # 256 > this 128^2 grid
        d = WL.BasisDesc(**{**w.basis.__dict__, **kw})
        with pytest.raises(lma.LmaError) as e:
            lma.Basis(ctx, spec, w.probe, d)
        assert e.value.status == lma.LMA_ERR_UNSUPPORTED, kw
    # atoms with a slice out of range
    at = w.phonons[0]
    bad_at = WL.Atoms(at.x, at.y, at.slice + 100, at.species)
    with pytest.raises(lma.LmaError) as e:
        lma.Specimen(ctx, w.grid, w.potential, [bad_at])
    assert e.value.status == lma.LMA_ERR_INVALID
    # device calls on a host-only context
    b = lma.Basis(ctx, spec, w.probe, w.basis)
    with pytest.raises(lma.LmaError) as e:
        b.propagate(0)
    assert e.value.status == lma.LMA_ERR_UNSUPPORTED


def test_edit_bookkeeping_matches_oracle_edit():
    w = WL.perovskite_workload(n_phonons=2, cells=10, nx=512, n_slices=4)
    ctx = lma.Context(-1)
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    cx, cy = 4.5 * WL.ABO3_A, 7.5 * WL.ABO3_A   # the O/B column at (1/2, 1/2) of cell (4, 7)
    n_changed, n_stale = spec.edit_column(None, cx, cy, 0.5, lma.LMA_EDIT_REMOVE)
    expect = 0
    for at in w.phonons:
        *_, nhit = O.edit_column(at.x, at.y, at.slice, at.species, w.grid.lx, w.grid.ly, cx, cy, 0.5, 0, 0)
        expect += nhit
    assert n_changed == expect and expect > 0 and n_stale == 0


# --------------------------------------------------------------------------- partitions (Sec. 4.2.4)

def _oracle_parts(w, region, strategy, M, start, period=(1, 1)):
    prm = O.params_from_workload(w)
    probes = O.region_probes(region.px0, region.py0, region.npx, region.npy, region.spacing_px,
                             w.grid.nx, w.grid.ny)
    sets = O.probe_translate_sets(prm, probes)
    if strategy == lma.LMA_PART_ROWS:
        parts = O.partition_rows(sets, region.npx, region.npy, M)
    elif strategy == lma.LMA_PART_GREEDY:
        parts = O.partition_greedy(sets, region.npx, region.npy, M, start)
    else:
        parts = O.partition_rectangles(sets, region.npx, region.npy, M,
                                       column_major=strategy == lma.LMA_PART_RECTANGLES_COLUMN_MAJOR,
                                       period=period)
    return parts, O.partition_cost(sets, parts), max(len(frozenset().union(*[sets[q] for q in p])) for p in parts)


@pytest.mark.parametrize("strategy", [lma.LMA_PART_ROWS, lma.LMA_PART_RECTANGLES,
                                      lma.LMA_PART_RECTANGLES_COLUMN_MAJOR, lma.LMA_PART_GREEDY])
def test_partition_equals_oracle(strategy):
    # ABO3 256^2 (Case 1: probes on the input lattice, period 1) and the simple-cubic crystal
    # with probes every 2 px (Case 2: input lattice every 4 px, period 2)
    cases = [(WL.perovskite_workload(cells=5, nx=256, n_slices=2, n_phonons=1),
              WL.Region(40, 200, 23, 17, (4, 4)), (1, 1), (60, 150, 400)),
             (WL.simple_cubic_workload(), WL.Region(6, 2, 19, 13, (2, 2)), (2, 2), (40, 90, 200))]
    for w, region, period, Ms in cases:
        ctx, spec, basis = _host_objects(w)
        for M in Ms:
            start = (region.npx * region.npy) // 3
            part, n, runs, peak = basis.partition(region, strategy, M, start)
            parts, T, pk = _oracle_parts(w, region, strategy, M, start, period)
            expect = np.empty(region.npx * region.npy, np.int32)
            for j, p in enumerate(parts):
                expect[p] = j
            assert n == len(parts) and runs == T and peak == pk, (strategy, M)
            assert np.array_equal(part.ravel(), expect), (strategy, M)
            assert peak <= M


def test_partition_validation():
    w = WL.simple_cubic_workload()
    ctx, spec, basis = _host_objects(w)
    region = WL.Region(0, 0, 4, 4, (8, 8))
    for strategy, M, start in ((7, 100, 0), (lma.LMA_PART_ROWS, w.basis.L - 1, 0),
                               (lma.LMA_PART_GREEDY, 100, 16), (lma.LMA_PART_GREEDY, 100, -1)):
        with pytest.raises(lma.LmaError) as e:
            basis.partition(region, strategy, M, start)
        assert e.value.status == lma.LMA_ERR_INVALID


def test_select_L_equals_oracle():
    import dataclasses
    for w, region in ((WL.simple_cubic_workload(), WL.Region(0, 0, 6, 5, (2, 2))),
                      (WL.perovskite_workload(cells=5, nx=256, n_slices=2, n_phonons=1), WL.Region(8, 4, 3, 3, (4, 4)))):
        ctx, spec, basis = _host_objects(w)
        prm = O.params_from_workload(w)
        probes = O.region_probes(region.px0, region.py0, region.npx, region.npy, region.spacing_px,
                                 w.grid.nx, w.grid.ny)
        for eps in (0.3, 0.15, 0.08):
            L, err = lma.select_L(ctx, spec, w.probe, w.basis, region, 40, eps)
            L_ref, err_ref = O.select_L(dataclasses.replace(prm, L=40), probes, eps, 40)
            assert L == L_ref and abs(err - err_ref) < 1e-9, (w.name, eps, L, L_ref, err, err_ref)
        assert lma.select_L(ctx, spec, w.probe, w.basis, region, 2, 1e-9)[0] == 0
        with pytest.raises(lma.LmaError):
            lma.select_L(ctx, spec, w.probe, w.basis, region, 65, 0.1)


@pytest.mark.parametrize("kind", [WL.BASIS_TRIG, WL.BASIS_TRIG_RADIAL])
def test_trig_input_waves_coefficients_match_oracle(kind):
    w = WL.simple_cubic_workload()
    w.basis.kind = kind
    _check_coefficients(w, [(0, 0), (8, 120), (127, 3)], tol=1e-8)
    w.basis.trig_degree = 9
    _check_coefficients(w, [(0, 0), (40, 40)], tol=1e-8)


def test_closed_form_trig_coefficients_match_oracle():
    """LMA_COEF_TRIG_CLOSED: the host's closed-form coefficients (Sec. 2, Sec. 4.2.3) and their
    approximation errors equal the oracle's, on the periodic 128^2 toy (n = 13, 32 input waves
    per axis) and on a 256^2 ABO3 slab (n = 25, 64 per axis); the L selection agrees too."""
    import dataclasses
    for w, probes in ((WL.simple_cubic_workload(), [(0, 0), (8, 120), (127, 3)]),
                      (WL.perovskite_workload(cells=5, nx=256, n_slices=2, n_phonons=1), [(2, 2), (101, 37)])):
        w.basis.kind = WL.BASIS_TRIG
        w.basis.coef_mode = 1
        _check_coefficients(w, probes, tol=1e-9)
    w = WL.simple_cubic_workload()
    w.basis.kind = WL.BASIS_TRIG
    w.basis.coef_mode = 1
    region = WL.Region(0, 0, 6, 5, (2, 2))
    ctx, spec, basis = _host_objects(w)
    prm = O.params_from_workload(w)
    probes = O.region_probes(region.px0, region.py0, region.npx, region.npy, region.spacing_px,
                             w.grid.nx, w.grid.ny)
    for eps in (0.5, 0.3):
        L, err = lma.select_L(ctx, spec, w.probe, w.basis, region, 40, eps)
        L_ref, err_ref = O.select_L(dataclasses.replace(prm, L=40), probes, eps, 40)
        assert L == L_ref and abs(err - err_ref) < 1e-9, (eps, L, L_ref, err, err_ref)


def test_closed_form_trig_coefficients_are_rejected_where_they_do_not_apply():
    w = WL.simple_cubic_workload()
    w.basis.coef_mode = 1                       # Gaussian input waves: no closed form
    with pytest.raises(lma.LmaError) as e:
        _host_objects(w)
    assert e.value.status == lma.LMA_ERR_INVALID
    w.basis.kind = WL.BASIS_TRIG
    w.basis.in_spacing_px = (8, 8)              # 16 input waves per axis < 2n + 1 = 27
    w.basis.in_offset_px = (0, 0)
    with pytest.raises(lma.LmaError) as e:
        _host_objects(w)
    assert e.value.status == lma.LMA_ERR_INVALID and "2n + 1" in str(e.value)
    w.basis.coef_mode = 2
    with pytest.raises(lma.LmaError) as e:
        _host_objects(w)
    assert e.value.status == lma.LMA_ERR_INVALID


def test_least_squares_error_never_rises_with_L():
    """The L nearest input waves form nested sets (a fixed order), so the least-squares L2
    error of the probe approximation cannot rise with L (the error-versus-L figures of
    Sec. 4.2.3 fall in steps); probe, Gaussian and trigonometric input waves."""
    ctx = lma.Context(-1)
    for kind in (WL.BASIS_PROBE, WL.BASIS_GAUSS, WL.BASIS_TRIG):
        prev = np.inf
        for L in range(1, 25):
            w = WL.simple_cubic_workload()
            w.basis.kind = kind
            w.basis.L = L
            spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
            b = lma.Basis(ctx, spec, w.probe, w.basis)
            e = b.coefficients(0, 0)[3][0]
            assert e <= prev * (1 + 1e-12), (kind, L, e, prev)
            prev = e
            b.close()
            spec.close()


def test_header_is_plain_c():
    """include/lma.h is a C ABI: it compiles as strict C99 (gcc) with no C++ constructs."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    r = subprocess.run([gcc, "-std=c99", "-fsyntax-only", "-Wall", "-Wextra", "-pedantic", "-Werror", "-x", "c",
                        os.path.join(ROOT, "include", "lma.h")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_binding_fails_loudly_without_the_cuda_library(tmp_path):
    """No fallback: loading the binding's library from a path where it was not built raises
    (checked in a fresh process, since a loaded library is cached)."""
    import subprocess
    import sys
    missing = str(tmp_path / "liblma.so")
    code = ("from paper_2310_16829_gb300 import lma\n"
            "try:\n    lma.load(%r)\nexcept RuntimeError as e:\n    print('raised:', e)\n    raise SystemExit(3)\n" % missing)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 3 and "not built" in r.stdout, (r.returncode, r.stdout, r.stderr[-500:])


def test_realspace_gain_matches_the_dft_of_the_oracle_kernel():
    """lma_realspace_gain against numpy's DFT of the oracle's truncated kernel (Sec. 3.2):
    max |Q(k)| of the zero-padded K x K kernel on the W x W window; the untruncated kernel
    (K = W - 1 covers all but one row and column; K = 1 is the kernel's centre) bounds."""
    w = WL.perovskite_workload(n_phonons=1, n_slices=2)
    ctx, spec, basis = _host_objects(w)
    prm = O.params_from_workload(w)
    prop = O.fresnel_propagator(128, 128, prm.dy, prm.dx, prm.lam, prm.slice_dz, prm.bandlimit_frac)
    for K1, K2 in ((3, 3), (5, 9), (13, 13)):
        qK = O.realspace_kernel(prop, K1, K2)
        full = np.zeros((128, 128), complex)
        for iy, dy in enumerate(O.kernel_offsets(K2)):
            for ix, dx in enumerate(O.kernel_offsets(K1)):
                full[dy % 128, dx % 128] = qK[iy, ix]
        Q = np.abs(np.fft.fft2(full))
        band = O.bandlimit_mask(128, 128, prm.bandlimit_frac)
        ga, gb = basis.realspace_gain(K1, K2)
        assert abs(ga - Q.max()) < 1e-12 and abs(gb - Q[band].max()) < 1e-12, (K1, K2)
    # the centre alone is the propagator's mean; the full-but-one kernel is close to |P| <= 1
    ga, _ = basis.realspace_gain(1, 1)
    assert abs(ga - abs(prop.mean())) < 1e-12
    assert abs(basis.realspace_gain(127, 127)[0] - 1.0) < 0.05
    with pytest.raises(lma.LmaError):
        basis.realspace_gain(4, 3)



def test_selftest_wait_checks_its_arguments_before_the_device():
    """lma_selftest_wait rejects an unknown wait form with LMA_ERR_INVALID and needs a device
    for the known ones (host-only context: LMA_ERR_UNSUPPORTED)."""
    ctx = lma.Context(-1)
    assert ctx.selftest_wait(2) == lma.LMA_ERR_INVALID
    assert ctx.selftest_wait(-1) == lma.LMA_ERR_INVALID
    assert ctx.selftest_wait(0) == lma.LMA_ERR_UNSUPPORTED


def test_synth_tuning_read_reports_nothing_before_tuning():
    """lma_synth_tuning_read counts the tuned synthesis shapes (none in a fresh context) and
    checks its arguments."""
    ctx = lma.Context(-1)
    assert ctx.synth_tuning() == []
    n = ctypes.c_int32()
    assert ctx.lib.lma_synth_tuning_read(ctx.h, None, 1, ctypes.byref(n)) == lma.LMA_ERR_INVALID


def test_synth_form_and_buffer_limit_arguments():
    """lma_set_synth_mode takes LMA_SYNTH_AUTO, _GATHER and _GROUPED only, and
    lma_set_synth_buffer_limit a byte count >= 0 (0 restores the default); both are context
    state, set without a device."""
    ctx = lma.Context(-1)
    for m in (lma.LMA_SYNTH_GATHER, lma.LMA_SYNTH_GROUPED, lma.LMA_SYNTH_AUTO):
        ctx.set_synth_mode(m)
    for m in (-2, 2):
        assert ctx.lib.lma_set_synth_mode(ctx.h, m) == lma.LMA_ERR_INVALID
    ctx.set_synth_buffer_limit(1 << 20)
    ctx.set_synth_buffer_limit(0)
    assert ctx.lib.lma_set_synth_buffer_limit(ctx.h, -1) == lma.LMA_ERR_INVALID
    assert ctx.lib.lma_set_synth_mode(None, 0) == lma.LMA_ERR_INVALID
