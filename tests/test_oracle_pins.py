"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a direct sum,
a closed form, a value printed in the paper, brute force on a tiny input, an
invariant or a symmetry. They are chosen so that a plausible slip (a dropped
term, a wrong sign or index, a transposed operand) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import lma_oracle as O

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b))))


# --------------------------------------------------------------------------- transforms

def test_dft2_matches_direct_double_sum():
    rng = np.random.default_rng(1)
    n, m = 16, 12
    a = rng.normal(size=(m, n)) + 1j * rng.normal(size=(m, n))
    direct = np.zeros((m, n), dtype=np.complex128)
    ys, xs = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    for ky in range(m):
        for kx in range(n):
            direct[ky, kx] = np.sum(a * np.exp(-2j * np.pi * (ky * ys / m + kx * xs / n)))
    assert rel(O.dft2(a), direct) < 1e-13
    assert rel(O.idft2(O.dft2(a)), a) < 1e-14
    inv = np.zeros_like(direct)
    for y in range(m):
        for x in range(n):
            inv[y, x] = np.sum(direct * np.exp(2j * np.pi * (ys * y / m + xs * x / n))) / (m * n)
    assert rel(inv, a) < 1e-13


def test_frequencies_are_the_papers_centred_grid_in_fft_order():
    # Sec. 4.1: g(k) = (k - 1 - floor(X/2)) / l_x for k = 1..X (centred order)
    for n, l in ((16, 4.0), (15, 3.0), (128, 16.0)):
        centred = (np.arange(1, n + 1) - 1 - n // 2) / l
        assert np.allclose(np.fft.fftshift(O.freqs(n, l / n)), centred, rtol=0, atol=1e-15)


# --------------------------------------------------------------------------- propagation

def _gaussian(ny, nx, dy, dx, s, cy=0.0, cx=0.0):
    y = O.min_image(np.arange(ny), ny) * dy - cy
    x = O.min_image(np.arange(nx), nx) * dx - cx
    return np.exp(-(y[:, None] ** 2 + x[None, :] ** 2) / (2 * s * s)).astype(np.complex128)


def _free_gaussian(ny, nx, dy, dx, s, lam, z, cy=0.0, cx=0.0):
    """Closed form of the paraxial equation (Sec. 3.1, V = 0) for a Gaussian start.

    psi(0) = exp(-r^2 / 2 s^2)  ->  psi(z) = (s^2/Q) exp(-r^2 / 2Q), Q = s^2 + i lambda z / 2 pi.
    """
    q = s * s + 1j * lam * z / (2 * np.pi)
    y = O.min_image(np.arange(ny), ny) * dy - cy
    x = O.min_image(np.arange(nx), nx) * dx - cx
    r2 = y[:, None] ** 2 + x[None, :] ** 2
    return (s * s / q) * np.exp(-r2 / (2 * q))


def test_fresnel_propagation_of_a_gaussian_matches_closed_form():
    # non-square grid and pixels so that a transposed axis fails
    ny, nx, dy, dx = 192, 256, 0.11, 0.1
    s, lam, dz, n = 0.5, 0.025, 5.0, 10
    psi = _gaussian(ny, nx, dy, dx, s)
    prop = O.fresnel_propagator(ny, nx, dy, dx, lam, dz, 2.0 / 3.0)
    ex = O.multislice(psi, [np.ones((ny, nx))] * n, prop)
    assert rel(ex, _free_gaussian(ny, nx, dy, dx, s, lam, n * dz)) < 1e-11


def test_transmit_then_propagate_order_with_a_tilt():
    # Fig. multislice_pseudocode: transmission first, then propagation. A tilt
    # t = exp(2 pi i q.x) then propagation over z moves the Gaussian by lambda z q
    # and adds the phase exp(2 pi i q.x - i pi lambda z |q|^2).
    ny, nx, dy, dx = 256, 256, 0.1, 0.1
    s, lam, z = 0.5, 0.025, 40.0
    mq, nq = 9, -5
    qx, qy = mq / (nx * dx), nq / (ny * dy)
    y = np.arange(ny) * dy
    x = np.arange(nx) * dx
    tilt = np.exp(2j * np.pi * (qy * y[:, None] + qx * x[None, :]))
    psi0 = _gaussian(ny, nx, dy, dx, s)
    prop = O.fresnel_propagator(ny, nx, dy, dx, lam, z, 2.0 / 3.0)
    ex = O.multislice(psi0, [tilt], prop)
    # evaluate the closed form on the periodic grid with the tilt written on
    # min-image coordinates (tilt is periodic because q lies on the grid)
    ym = O.min_image(np.arange(ny), ny) * dy
    xm = O.min_image(np.arange(nx), nx) * dx
    phase = np.exp(2j * np.pi * (qy * ym[:, None] + qx * xm[None, :]) - 1j * np.pi * lam * z * (qx * qx + qy * qy))
    expect = phase * _free_gaussian(ny, nx, dy, dx, s, lam, z, cy=lam * z * qy, cx=lam * z * qx)
    assert rel(ex, expect) < 1e-10


def test_slices_compose_in_free_space():
    rng = np.random.default_rng(2)
    n, d, lam = 64, 0.1, 0.02
    mask = O.bandlimit_mask(n, n, 2.0 / 3.0)
    psi = O.idft2(mask * (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))))
    many = O.multislice(psi, [np.ones((n, n))] * 7, O.fresnel_propagator(n, n, d, d, lam, 1.5, 2 / 3))
    one = O.multislice(psi, [np.ones((n, n))], O.fresnel_propagator(n, n, d, d, lam, 7 * 1.5, 2 / 3))
    assert rel(many, one) < 1e-12


def test_constant_potential_is_a_global_phase():
    rng = np.random.default_rng(3)
    n, d, lam, sigma, v0, ns = 64, 0.1, 0.02, 7e-4, 37.0, 5
    psi = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    prop = O.fresnel_propagator(n, n, d, d, lam, 2.0, 2 / 3)
    free = O.multislice(psi, [np.ones((n, n))] * ns, prop)
    t = O.transmission(np.full((n, n), v0), sigma)
    tilted = O.multislice(psi, [t] * ns, prop)
    assert rel(tilted, np.exp(1j * ns * sigma * v0) * free) < 1e-13


def test_norm_identity_per_slice():
    # |t| = 1 and |P| = 1: each slice loses exactly the energy outside the mask
    rng = np.random.default_rng(4)
    n, d, lam, sigma = 64, 0.1, 0.02, 7e-4
    mask = O.bandlimit_mask(n, n, 2 / 3)
    prop = O.fresnel_propagator(n, n, d, d, lam, 2.0, 2 / 3)
    psi = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    for _ in range(3):
        t = O.transmission(rng.uniform(0, 500, size=(n, n)), sigma)
        nxt = O.multislice(psi, [t], prop)
        lost = np.sum(np.abs(O.dft2(t * psi)[~mask]) ** 2) / n ** 2
        assert abs(np.sum(np.abs(nxt) ** 2) - (np.sum(np.abs(psi) ** 2) - lost)) < 1e-9 * np.sum(np.abs(psi) ** 2)
        psi = nxt
    # band-limited input in free space keeps its norm
    bl = O.idft2(mask * O.dft2(psi))
    out = O.multislice(bl, [np.ones((n, n))] * 3, prop)
    assert abs(np.sum(np.abs(out) ** 2) / np.sum(np.abs(bl) ** 2) - 1) < 1e-13


def test_multislice_is_linear():
    rng = np.random.default_rng(5)
    n, d, lam, sigma = 48, 0.1, 0.02, 7e-4
    prop = O.fresnel_propagator(n, n, d, d, lam, 2.0, 2 / 3)
    ts = [O.transmission(rng.uniform(0, 300, size=(n, n)), sigma) for _ in range(4)]
    us = [rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)) for _ in range(3)]
    al = rng.normal(size=3) + 1j * rng.normal(size=3)
    lhs = O.multislice(sum(a * u for a, u in zip(al, us)), ts, prop)
    rhs = sum(a * O.multislice(u, ts, prop) for a, u in zip(al, us))
    assert rel(lhs, rhs) < 1e-13


def test_multislice_commutes_with_grid_shifts():
    rng = np.random.default_rng(6)
    n, d, lam, sigma = 48, 0.1, 0.02, 7e-4
    prop = O.fresnel_propagator(n, n, d, d, lam, 2.0, 2 / 3)
    ts = [O.transmission(rng.uniform(0, 300, size=(n, n)), sigma) for _ in range(3)]
    u = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    sh = (5, -11)
    a = np.roll(O.multislice(u, ts, prop), sh, axis=(0, 1))
    b = O.multislice(np.roll(u, sh, axis=(0, 1)), [np.roll(t, sh, axis=(0, 1)) for t in ts], prop)
    assert rel(a, b) < 1e-13


# --------------------------------------------------------------------------- physics model

def test_wavelength_and_gaussian_width_match_the_paper():
    g = GOLDEN["wavelength_200kV_A"]
    assert round(O.electron_wavelength(200e3), g["digits"]) == g["value"]
    s = GOLDEN["gaussian_sigma_A"]
    assert round(O.gaussian_width(s["inputs"]["lambda"], s["inputs"]["alpha_max"]), s["digits"]) == s["value"]


def test_workload_literals_match_the_formulas():
    from paper_2310_16829_gb300 import workloads as WL
    assert abs(WL.LAMBDA_300KV / O.electron_wavelength(300e3) - 1) < 1e-12
    assert abs(WL.SIGMA_300KV / O.interaction_constant(300e3) - 1) < 1e-12
    # the toy workload states rounded 200 kV constants
    assert abs(WL.LAMBDA_CFG0 - O.electron_wavelength(200e3)) < 1e-5
    assert abs(WL.SIGMA_CFG0 - O.interaction_constant(200e3)) < 1e-6


def test_probe_is_normalised_band_limited_and_shifts_by_modulation():
    ny, nx, d, lam, a = 96, 96, 0.1, 0.02, 0.03
    p0 = O.probe(ny, nx, d, d, lam, a, cs=1000.0, defocus=50.0)
    assert abs(np.sum(np.abs(p0) ** 2) - 1) < 1e-13
    k2 = O.k_squared(ny, nx, d, d)
    outside = lam * np.sqrt(k2) >= a
    assert np.max(np.abs(O.dft2(p0)[outside])) < 1e-12
    # aperture is strict and the aberration phase is applied: |spectrum| is flat inside
    spec = O.dft2(p0)
    inside = ~outside
    assert np.ptp(np.abs(spec[inside])) < 1e-10
    # eq. probe_wave_function with an integer-pixel p equals a roll of psi_0
    pshift = O.probe(ny, nx, d, d, lam, a, cs=1000.0, defocus=50.0, p=(7 * d, -3 * d))
    assert rel(pshift, np.roll(p0, (7, -3), axis=(0, 1))) < 1e-12


def test_aberration_phase_sign_and_powers():
    # chi = 1/2 pi Cs lambda^3 k^4 - pi Z lambda k^2 evaluated at two points
    lam = 0.02
    k2 = np.array([0.25, 4.0])
    chi_cs = O.aberration(k2, lam, 1e7, 0.0)
    chi_z = O.aberration(k2, lam, 0.0, 100.0)
    assert abs(chi_cs[1] / chi_cs[0] - 256.0) < 1e-12      # |k|^4
    assert abs(chi_z[1] / chi_z[0] - 16.0) < 1e-12         # |k|^2
    assert chi_z[0] < 0 and chi_cs[0] > 0
    assert abs(chi_cs[0] - 0.5 * np.pi * 1e7 * lam ** 3 * 0.0625) < 1e-12 * chi_cs[0]


def test_projected_potential_closed_forms():
    # one atom on a fine grid: v at its pixel is peak * sum(frac); the pixel sum
    # times dx dy is the truncated Gaussian integral 2 pi w^2 (1 - exp(-rc^2 / 2w^2))
    n, l = 512, 10.24
    d = l / n
    peak, fr, wd, rc = (250.0,), (0.7, 0.3), (0.15, 0.5), 3.0
    xa, ya = 20 * d, 230 * d     # exactly on pixel (x=20, y=230)
    v = O.projected_potential(np.array([xa]), np.array([ya]), np.array([0]), np.array([0]),
                              1, n, n, l, l, peak, fr, wd, rc)[0]
    assert abs(v[230, 20] - 250.0) < 1e-12
    assert v[20, 230] == 0.0   # not transposed
    integral = 250.0 * sum(f * 2 * np.pi * w * w * (1 - np.exp(-rc * rc / (2 * w * w))) for f, w in zip(fr, wd))
    assert abs(np.sum(v) * d * d / integral - 1) < 1e-8
    # periodic images: an atom across the boundary gives the same field shifted
    v2 = O.projected_potential(np.array([l - 3 * d]), np.array([0.5 * d]), np.array([0]), np.array([0]),
                               1, n, n, l, l, peak, fr, wd, rc)[0]
    v3 = O.projected_potential(np.array([30 * d]), np.array([0.5 * d]), np.array([0]), np.array([0]),
                               1, n, n, l, l, peak, fr, wd, rc)[0]
    assert rel(np.roll(v3, -33, axis=1), v2) < 1e-12
    # hard cutoff
    yy, xx = np.meshgrid(np.arange(n) * d, np.arange(n) * d, indexing="ij")
    ddx = (xx - xa) - l * np.round((xx - xa) / l)
    ddy = (yy - ya) - l * np.round((yy - ya) / l)
    r = np.sqrt(ddx ** 2 + ddy ** 2)
    assert np.all(v[r > rc + 1e-9] == 0.0) and np.all(v[r < rc - 1e-9] > 0.0)


def test_detector_reads_a_plane_wave():
    n, d, lam = 64, 0.1, 0.025
    m0, n0 = 5, -3
    k = math.hypot(m0 / (n * d), n0 / (n * d))
    y = np.arange(n) * d
    pw = np.exp(2j * np.pi * (n0 / (n * d) * y[:, None] + m0 / (n * d) * y[None, :])) / n
    inside = O.detector_mask(n, d, d, lam, lam * k * 0.99, lam * k * 1.01, 2 / 3)
    assert abs(O.detect(pw, inside) - 1.0) < 1e-13
    assert O.detect(pw, O.detector_mask(n, d, d, lam, lam * k * 1.01, 1.0, 2 / 3)) < 1e-25
    # an annulus ending just below the wave's angle does not see it
    assert O.detect(pw, O.detector_mask(n, d, d, lam, 0.0, lam * k * 0.999999, 2 / 3)) < 1e-25


def test_detector_over_all_frequencies_is_parseval():
    rng = np.random.default_rng(7)
    psi = rng.normal(size=(32, 32)) + 1j * rng.normal(size=(32, 32))
    assert abs(O.detect(psi, np.ones((32, 32), bool)) / np.sum(np.abs(psi) ** 2) - 1) < 1e-13


def _plane_wave(ny, nx, d, m0, n0):
    """Unit-norm plane wave exp(2 pi i (m0 x / (nx d) + n0 y / (ny d))) on an ny x nx grid."""
    y = np.arange(ny)[:, None] * d
    x = np.arange(nx)[None, :] * d
    return np.exp(2j * np.pi * (m0 * x / (nx * d) + n0 * y / (ny * d))) / math.sqrt(nx * ny)


def test_rings_put_a_plane_wave_in_its_ring_only():
    # 3D STEM of Sec. 3.1: consecutive rings of width r from 0
    n, d, lam, width = 64, 0.1, 0.025, 0.004
    m0, n0 = 5, -3
    ang = lam * math.hypot(m0 / (n * d), n0 / (n * d))
    pw = _plane_wave(n, n, d, m0, n0)
    rings = O.ring_masks(n, d, d, lam, width, 30, 2 / 3)
    reads = np.array([O.detect(pw, m) for m in rings])
    a = int(ang // width)
    assert abs(reads[a] - 1.0) < 1e-13
    assert np.all(np.delete(reads, a) < 1e-25)


def test_rings_add_up_to_the_annulus_they_tile():
    rng = np.random.default_rng(3)
    n, d, lam, width, nr = 64, 0.1, 0.025, 0.0037, 21
    psi = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    total = sum(O.detect(psi, m) for m in O.ring_masks(n, d, d, lam, width, nr, 2 / 3))
    annulus = O.detect(psi, O.detector_mask(n, d, d, lam, 0.0, nr * width, 2 / 3))
    assert abs(total / annulus - 1) < 1e-12


def test_pattern_of_a_plane_wave_is_a_unit_delta_at_its_frequency():
    # non-square grid: a transposed axis or a sign slip moves the delta
    ny, nx, d = 48, 64, 0.1
    for m0, n0 in ((5, -3), (-7, 2)):
        pw = _plane_wave(ny, nx, d, m0, n0)
        for frac in (None, 2 / 3):
            pat = O.pattern(pw, 10, 6, frac)
            assert pat.shape == (13, 21)
            assert abs(pat[n0 + 6, m0 + 10] - 1.0) < 1e-13
            rest = pat.copy()
            rest[n0 + 6, m0 + 10] = 0
            assert np.all(rest < 1e-25)
    # a wave outside the bandlimit leaves nothing in the pattern (rounding noise only)
    pw = _plane_wave(64, 64, d, 30, 0)
    pat = O.pattern(pw, 31, 31, 2 / 3)
    assert pat[31, 61] == 0.0 and np.all(pat < 1e-25)
    assert abs(O.pattern(pw, 31, 31, None)[31, 61] - 1.0) < 1e-13


def test_pattern_summed_over_an_annulus_is_the_2d_reading():
    rng = np.random.default_rng(5)
    n, d, lam = 64, 0.1, 0.025
    psi = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    A = n // 2 - 1
    pat = O.pattern(psi, A, A, 2 / 3)
    ia = np.arange(-A, A + 1)
    k = np.hypot(ia[None, :] / (n * d), ia[:, None] / (n * d))
    for r1, r2 in ((0.0, 0.02), (0.01, 0.05), (0.03, 0.07)):
        sel = (lam * k >= r1) & (lam * k < r2)
        ref = O.detect(psi, O.detector_mask(n, d, d, lam, r1, r2, 2 / 3))
        assert abs(pat[sel].sum() / ref - 1) < 1e-12


def test_bandlimit_mask_is_the_integer_two_thirds_circle():
    for n in (64, 128, 256):
        m = O.bandlimit_mask(n, n, 2 / 3)
        i = O.signed_index(n)
        brute = np.array([[9 * (a * a + b * b) <= n * n for b in i] for a in i])
        assert np.array_equal(m, brute)


# --------------------------------------------------------------------------- LMA geometry

def test_input_lattice_count_matches_the_recompute_example():
    g = GOLDEN["input_lattice_count"]
    # 848 x 800 grid, probes every 2 px (P = (424, 400)), I = P + p/2, f = 2
    lat = O.input_lattice(848, 800, (2, 2), (1, 1), 2)
    assert lat.shape[0] == g["value"]
    assert 424 * 400 == GOLDEN["probe_count"]["value"]
    assert len(set(map(tuple, lat.tolist()))) == g["value"]


def test_nearest_translates_form_complete_shells():
    lat = O.input_lattice(64, 64, (4, 4), (2, 2), 1)
    idx, offs = O.nearest_translates((0, 0), lat, 32, 64, 64)
    d2 = offs[:, 0] ** 2 + offs[:, 1] ** 2
    # brute force: all offsets (2 + 4a) in both axes, sorted by distance
    vals = sorted((x * x + y * y) for x in range(-30, 31) for y in range(-30, 31)
                  if x % 4 == 2 and y % 4 == 2)
    assert sorted(d2.tolist()) == vals[:32]
    assert set(np.unique(d2).tolist()) == {8, 40, 72, 104, 136}
    # returned indices address the same translates as the offsets
    assert np.array_equal(O.min_image(lat[idx, 0], 64), offs[:, 0])


def _small_params(**kw):
    base = dict(nx=64, ny=64, lx=8.0, ly=8.0, slice_dz=2.0, n_slices=3, lam=0.025, sigma=7.3e-4,
                bandlimit_frac=2 / 3, alpha_max=0.03, cs=0.0, defocus=0.0, kind=0, gauss_sigma=0.0,
                in_spacing=(4, 4), in_offset=(2, 2), f=1, L=8, W=64, D=64)
    base.update(kw)
    return O.LmaParams(**base)


def _direct_ls(prm, p, L):
    """Least squares written against absolute positions for probe p (no reuse)."""
    lat = O.input_lattice(prm.nx, prm.ny, prm.in_spacing, prm.in_offset, prm.f)
    idx, _ = O.nearest_translates(p, lat, L, prm.nx, prm.ny)
    psi = O.probe(prm.ny, prm.nx, prm.dy, prm.dx, prm.lam, prm.alpha_max, p=(p[1] * prm.dy, p[0] * prm.dx))
    uW = O.input_wave_window(prm.kind, prm.W, prm.ny, prm.nx, prm.dy, prm.dx, prm.lam, prm.alpha_max, 0, 0, 0)
    A = np.stack([O.embed_window(uW, int(lat[i, 1]) - prm.W // 2, int(lat[i, 0]) - prm.W // 2,
                                 prm.ny, prm.nx).ravel() for i in idx], 1)
    al = np.linalg.lstsq(A, psi.ravel(), rcond=None)[0]
    res = np.linalg.norm(psi.ravel() - A @ al)
    return al, res, A, psi.ravel()


def test_case1_same_coefficients_and_error_for_every_probe():
    # Case 1 (eq. lma_approximation_exit1): probes every 8 px, translates every 4 px
    prm = _small_params(W=32, D=32)
    ref = None
    for p in [(0, 0), (8, 16), (56, 40), (24, 56)]:
        al, res, _, _ = _direct_ls(prm, p, 12)
        if ref is None:
            ref = (al, res)
        assert rel(al, ref[0]) < 1e-9
        assert abs(res - ref[1]) < 1e-12
    orc = O.LmaOracle(_small_params(W=32, D=32, L=12))
    cs, _ = orc.coefficient_set((24, 56))
    assert rel(cs.alpha, ref[0]) < 1e-9


def test_case2_gives_c_times_d_coefficient_sets_reused_by_translation():
    # Case 2 (eq. lma_approximation_exit2): probes every 2 px, translates every 4 px
    prm = _small_params(W=32, D=32, L=10)
    orc = O.LmaOracle(prm)
    probes = O.region_probes(0, 0, 8, 8, (2, 2), 64, 64)
    for pr in probes:
        orc.coefficient_set((int(pr[0]), int(pr[1])))
    assert len(orc._sets) == 4
    al, _, _, _ = _direct_ls(prm, (6, 10), 10)      # a probe of class (0, 0), solved directly
    cs, _ = orc.coefficient_set((6, 10))
    assert rel(cs.alpha, al) < 1e-9


def test_least_squares_residual_is_orthogonal_and_matches_normal_equations():
    prm = _small_params(W=32, D=32)
    al, _, A, b = _direct_ls(prm, (0, 0), 6)
    r = b - A @ al
    assert np.max(np.abs(A.conj().T @ r)) < 1e-12 * np.linalg.norm(b) * np.max(np.abs(A))
    ne = np.linalg.solve(A.conj().T @ A, A.conj().T @ b)
    assert rel(ne, al) < 1e-8


def test_synthesis_placement_truncates_or_wraps():
    U = (np.arange(16).reshape(4, 4) + 1).astype(np.complex128)
    out = O.synthesize([U], np.array([2.0]), np.array([[1, -2]]), 4, cyclic=False)
    exp = np.zeros((4, 4), complex)
    exp[0:2, 1:4] = 2 * U[2:4, 0:3]
    assert np.array_equal(out, exp)
    out_c = O.synthesize([U], np.array([1.0]), np.array([[1, -2]]), 4, cyclic=True)
    assert np.array_equal(out_c, np.roll(U, (-2, 1), axis=(0, 1)))
    # a larger detection window centres the exit wave
    out_d = O.synthesize([U], np.array([1.0]), np.array([[0, 0]]), 8, cyclic=False)
    assert np.array_equal(out_d[2:6, 2:6], U) and np.sum(np.abs(out_d)) == np.sum(np.abs(U))


# --------------------------------------------------------------------------- LMA vs brute force

def _tiny_specimen(prm, seed=11, per_slice=3):
    rng = np.random.default_rng(seed)
    n = per_slice * prm.n_slices
    x = rng.uniform(0, prm.lx, n)
    y = rng.uniform(0, prm.ly, n)
    s = np.repeat(np.arange(prm.n_slices), per_slice).astype(np.int32)
    sp = rng.integers(0, 2, n).astype(np.int16)
    class A:
        pass
    a = A()
    a.x, a.y, a.slice, a.species = x, y, s, sp
    return a


class _Det:
    def __init__(self, r1, r2):
        self.r1, self.r2 = r1, r2


def test_lma_with_probe_input_waves_is_the_standard_algorithm():
    # Sec. 4.2.3: u = psi_0, I = P, f = 1, L = 1 retrieves the standard algorithm
    prm = _small_params(kind=1, in_spacing=(8, 8), in_offset=(0, 0), L=1, n_slices=4)
    at = _tiny_specimen(prm)
    orc = O.LmaOracle(prm)
    orc.set_specimen([at], (300.0, 150.0), (0.7, 0.3), (0.15, 0.5), 3.0)
    probes = O.region_probes(0, 0, 8, 8, (8, 8), 64, 64)
    dets = [_Det(0.0, 0.02), _Det(0.03, 0.066)]
    img = orc.image(dets, probes)
    std = O.standard_image(prm, orc.transmission_stack(0), dets, probes)
    assert rel(img, std) < 1e-12
    cs, _ = orc.coefficient_set((0, 0))
    assert cs.err_l2 < 1e-13 and abs(cs.alpha[0] - 1) < 1e-13


def test_lma_with_gaussian_waves_propagates_the_approximated_probe_exactly():
    # linearity (Sec. 4.2): with W = D = X, LMA is standard multislice of sum alpha u_i
    prm = _small_params(kind=0, L=12, n_slices=3)
    at = _tiny_specimen(prm, seed=12)
    orc = O.LmaOracle(prm)
    orc.set_specimen([at], (300.0, 150.0), (0.7, 0.3), (0.15, 0.5), 3.0)
    probes = O.region_probes(4, 0, 5, 3, (12, 20), 64, 64)

    def approx(p):
        cs, idx = orc.coefficient_set(p)
        full = np.zeros((64, 64), complex)
        for a, i in zip(cs.alpha, idx):
            full += a * O.embed_window(orc.uW, int(orc.lattice[i, 1]) - 32, int(orc.lattice[i, 0]) - 32, 64, 64)
        return full

    dets = [_Det(0.03, 0.066)]
    img = orc.image(dets, probes)
    std = O.standard_image(prm, orc.transmission_stack(0), dets, probes, psi_init=approx)
    assert rel(img, std) < 1e-12


def test_simple_cubic_image_has_crystal_period_and_4mm_symmetry():
    # simple-cubic 2x2 cells of 4 A on 64^2: image periodic with 32 px and 4mm symmetric
    prm = _small_params(L=32, n_slices=3, alpha_max=0.02)
    xs, ys, ss = [], [], []
    for s in range(prm.n_slices):
        for j in range(2):
            for i in range(2):
                xs.append(4.0 * i); ys.append(4.0 * j); ss.append(s)

    class A:
        pass
    at = A()
    at.x, at.y = np.array(xs), np.array(ys)
    at.slice, at.species = np.array(ss, np.int32), np.zeros(len(xs), np.int16)
    orc = O.LmaOracle(prm)
    orc.set_specimen([at], (300.0,), (0.7, 0.3), (0.15, 0.5), 3.0)
    probes = O.region_probes(0, 0, 16, 16, (4, 4), 64, 64)
    img = orc.image([_Det(0.03, 0.066)], probes)[0].reshape(16, 16)
    tol = 1e-10 * np.max(img)
    assert np.max(np.abs(img - np.roll(img, 8, axis=0))) < tol
    assert np.max(np.abs(img - np.roll(img, 8, axis=1))) < tol
    assert np.max(np.abs(img - img.T)) < tol
    mirror = img[:, (-np.arange(16)) % 16]
    assert np.max(np.abs(img - mirror)) < tol
    assert np.ptp(img) > 1e3 * tol   # not trivially constant


def test_3d_and_4d_images_agree_with_the_2d_image():
    # the same synthesized exit waves read three ways: rings tiling an annulus add up to
    # its 2D reading, and so does the 4D pattern summed over the annulus
    prm = _small_params(L=32, n_slices=3, alpha_max=0.02)

    class A:
        pass
    at = A()
    at.x, at.y = np.array([0.0, 4.0, 0.0, 4.0]), np.array([0.0, 0.0, 4.0, 4.0])
    at.slice, at.species = np.zeros(4, np.int32), np.zeros(4, np.int16)
    orc = O.LmaOracle(prm)
    orc.set_specimen([at], (300.0,), (0.7, 0.3), (0.15, 0.5), 3.0)
    probes = np.array([[0, 0], [6, 2], [33, 17]])
    width, nr = 0.005, 13
    rings = orc.image_rings(width, nr, probes)
    two_d = orc.image([_Det(0.02, 0.045), _Det(0.0, nr * width)], probes)
    assert rel(rings[4:9].sum(axis=0), two_d[0]) < 1e-12
    assert rel(rings.sum(axis=0), two_d[1]) < 1e-12
    A4 = prm.D // 2 - 1
    pat = orc.image_4d(A4, A4, probes)
    ia = np.arange(-A4, A4 + 1)
    ang = prm.lam * np.hypot(ia[None, :] / (prm.D * prm.dx), ia[:, None] / (prm.D * prm.dy))
    sel = (ang >= 0.02) & (ang < 0.045)
    assert rel(pat[:, sel].sum(axis=1), two_d[0]) < 1e-12


def test_edit_column_removes_or_swaps_only_that_column():
    x = np.array([0.01, 3.9, 7.99, 2.0, 0.05])
    y = np.array([0.02, 0.0, 7.98, 2.0, 0.03])
    s = np.array([0, 0, 1, 1, 2], np.int32)
    sp = np.array([0, 1, 0, 1, 2], np.int16)
    x2, y2, s2, sp2, nhit = O.edit_column(x, y, s, sp, 8.0, 8.0, 0.0, 0.0, 0.3, 0, 0)
    assert nhit == 3 and list(x2) == [3.9, 2.0]
    _, _, _, sp3, nhit = O.edit_column(x, y, s, sp, 8.0, 8.0, 0.0, 0.0, 0.3, 1, 2)
    assert nhit == 3 and list(sp3) == [2, 1, 2, 1, 2]


# --------------------------------------------------------------------------- partitions (Sec. 4.2.4)

def _resident_runs(sets, parts):
    """Count Multislice runs by simulating the store: each part keeps exactly its own
    translates; a translate is computed when the part needs it and the previous one did not."""
    runs, resident = 0, set()
    for part in parts:
        need = set().union(*[sets[q] for q in part])
        runs += len(need - resident)
        resident = need
    return runs


def test_partitions_cover_the_region_once_and_fit_the_memory_bound():
    prm = _small_params(L=12)
    npx, npy = 9, 7
    probes = O.region_probes(4, 8, npx, npy, (4, 4), prm.nx, prm.ny)
    sets = O.probe_translate_sets(prm, probes)
    total = len(frozenset().union(*sets))
    for M in (12, 20, 37, 60, total):
        for parts in (O.partition_rows(sets, npx, npy, M), O.partition_rectangles(sets, npx, npy, M),
                      O.partition_rectangles(sets, npx, npy, M, column_major=True),
                      O.partition_rectangles(sets, npx, npy, M, period=(2, 3)),
                      O.partition_greedy(sets, npx, npy, M, start=31)):
            flat = sorted(q for p in parts for q in p)
            assert flat == list(range(npx * npy))
            assert all(len(frozenset().union(*[sets[q] for q in p])) <= M for p in parts)
            T = O.partition_cost(sets, parts)
            assert T == _resident_runs(sets, parts)
            assert total <= T <= sum(len(s) for s in sets)
    # enough memory for everything: one part, the minimum number of runs
    for parts in (O.partition_rows(sets, npx, npy, total), O.partition_rectangles(sets, npx, npy, total),
                  O.partition_greedy(sets, npx, npy, total, start=5)):
        assert len(parts) == 1 and O.partition_cost(sets, parts) == total


def test_greedy_partition_hand_worked():
    # 3 x 3 probes each needing only its own translate, M = 3, start at the centre; derived
    # by hand from the rule (fewest translates, ties by (b, a); dead end -> first unassigned)
    sets = [frozenset([q]) for q in range(9)]
    parts = O.partition_greedy(sets, 3, 3, 3, start=4)
    assert parts == [[4, 0, 1], [2, 5, 7], [3, 6, 8]]
    assert O.partition_cost(sets, parts) == 9


def test_rectangle_partition_hand_worked():
    # 5 x 4 probes, own translates, M = 6: largest area 6, squarest tie (2x3 vs 3x2) -> wider 3x2
    sets = [frozenset([q]) for q in range(20)]
    parts = O.partition_rectangles(sets, 5, 4, 6)
    assert parts == [[0, 1, 2, 5, 6, 7], [3, 4, 8, 9], [10, 11, 12, 15, 16, 17], [13, 14, 18, 19]]
    cm = O.partition_rectangles(sets, 5, 4, 6, column_major=True)
    assert cm == [parts[0], parts[2], parts[1], parts[3]]
    rows = O.partition_rows(sets, 5, 4, 6)
    assert rows == [[0, 1, 2, 3, 4, 5], [6, 7, 8, 9, 10, 11], [12, 13, 14, 15, 16, 17], [18, 19]]


# --------------------------------------------------------------------------- real-space propagation

def test_convolution_matches_a_direct_double_sum():
    rng = np.random.default_rng(11)
    n = 10
    psi = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    q = rng.normal(size=(3, 5)) + 1j * rng.normal(size=(3, 5))     # K2 = 3 (y), K1 = 5 (x)
    direct = np.zeros_like(psi)
    for y in range(n):
        for x in range(n):
            for iy, dy in enumerate((-1, 0, 1)):
                for ix, dx in enumerate((-2, -1, 0, 1, 2)):
                    direct[y, x] += q[iy, ix] * psi[(y - dy) % n, (x - dx) % n]
    assert rel(O.convolve_periodic(psi, q), direct) < 1e-13


def test_full_kernel_convolution_is_the_fourier_propagation():
    rng = np.random.default_rng(12)
    n, d, lam = 32, 0.1, 0.025
    prop = O.fresnel_propagator(n, n, d, d, lam, 2.0, 2 / 3)
    psi = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    t = [np.exp(1j * rng.normal(size=(n, n))) for _ in range(3)]
    q = O.realspace_kernel(prop, n, n)
    assert rel(O.multislice_realspace(psi, t, q), O.multislice(psi, t, prop)) < 1e-12
    # a 1 x 1 kernel multiplies by q(0) = the mean of the propagator
    q1 = O.realspace_kernel(prop, 1, 1)
    assert abs(q1[0, 0] - prop.mean()) < 1e-15
    # the truncated kernel approximates the propagation, better as it grows (the discrete
    # Fresnel kernel is a chirp with the bandlimit's rings, so the decay is slow)
    wave = O.probe(n, n, d, d, lam, 0.02)
    ref = O.multislice(wave, t[:1], prop)
    errs = [rel(O.multislice_realspace(wave, t[:1], O.realspace_kernel(prop, K, K)), ref) for K in (5, 9, 17, 31)]
    assert all(a > b for a, b in zip(errs, errs[1:])) and errs[0] < 0.5


# --------------------------------------------------------------------------- partial coherence, L from a target error

def _toy_specimen(orc):
    class A:
        pass
    at = A()
    at.x, at.y = np.array([0.0, 4.0, 0.0, 4.0]), np.array([0.0, 0.0, 4.0, 4.0])
    at.slice, at.species = np.zeros(4, np.int32), np.zeros(4, np.int16)
    orc.set_specimen([at], (300.0,), (0.7, 0.3), (0.15, 0.5), 3.0)
    return orc


def test_coherent_image_is_the_weighted_average_of_fresh_images():
    # Gaussian input waves do not depend on the focus: every variant's image from scratch
    # (new probe, coefficients and exit waves) must equal the shared-exit-wave result
    import dataclasses
    prm = _small_params(L=16, n_slices=2, alpha_max=0.025)
    probes = np.array([[0, 0], [6, 10], [33, 17]])
    dets = [_Det(0.0, 0.02), _Det(0.03, 0.066)]
    variants = [(-40.0, 0.0, 1.0), (0.0, 0.0, 2.0), (55.0, 0.0, 0.5)]
    got = _toy_specimen(O.LmaOracle(prm)).image_coherent(dets, probes, variants)
    ref = np.zeros_like(got)
    for dz, cs, wgt in variants:
        fresh = _toy_specimen(O.LmaOracle(dataclasses.replace(prm, defocus=dz, cs=cs)))
        ref += wgt / 3.5 * fresh.image(dets, probes)
    assert rel(got, ref) < 1e-12
    # one variant with the basis's own probe is the plain image
    orc = _toy_specimen(O.LmaOracle(prm))
    assert rel(orc.image_coherent(dets, probes, [(prm.defocus, prm.cs, 3.0)]), orc.image(dets, probes)) < 1e-14


def test_select_L_is_the_smallest_L_meeting_the_target():
    prm = _small_params(L=8)
    probes = O.region_probes(0, 0, 4, 4, (4, 4), prm.nx, prm.ny)
    lat = O.input_lattice(prm.nx, prm.ny, prm.in_spacing, prm.in_offset, prm.f)
    psi0 = O.probe(prm.ny, prm.nx, prm.dy, prm.dx, prm.lam, prm.alpha_max, prm.cs, prm.defocus)
    uW = O.input_wave_window(prm.kind, prm.W, prm.ny, prm.nx, prm.dy, prm.dx, prm.lam, prm.alpha_max,
                             prm.cs, prm.defocus, prm.gauss_sigma)

    def err(L):
        return O.coefficients(psi0, uW, O.nearest_translates((0, 0), lat, L, prm.nx, prm.ny)[1]).err_sup

    for eps in (0.75, 0.6, 0.5, 0.45):
        L, e = O.select_L(prm, probes, eps, 40)
        assert 1 <= L and e <= eps and abs(e - err(L)) < 1e-15
        assert L == 1 or err(L - 1) > eps
    assert O.select_L(prm, probes, 1e-9, 3)[0] == 0
    # u = probe on I = P: the probe is one of the input waves, L = 1 is exact (Sec. 4.2.3)
    import dataclasses
    pp = dataclasses.replace(prm, kind=1, in_offset=(0, 0))
    L, e = O.select_L(pp, probes, 1e-12, 4)
    assert L == 1 and e < 1e-12


def test_realspace_lma_with_the_full_kernel_is_the_fourier_lma():
    prm = _small_params(L=8, n_slices=2, alpha_max=0.03)
    probes = np.array([[0, 0], [6, 10]])
    dets = [_Det(0.0, 0.02), _Det(0.03, 0.066)]
    fourier = _toy_specimen(O.LmaOracle(prm)).image(dets, probes)
    full = _toy_specimen(O.LmaOracle(prm, realspace=(prm.W, prm.W))).image(dets, probes)
    assert rel(full, fourier) < 1e-12
    small = _toy_specimen(O.LmaOracle(prm, realspace=(5, 5))).image(dets, probes)
    assert 1e-6 < rel(small, fourier) < 1.0      # an approximation, not the Fourier image


# --------------------------------------------------------------------------- trigonometric input waves

def test_trig_polynomial_has_the_stated_coefficients():
    # phi_n sampled at M >= 2n + 1 points of one period: its DFT holds cos(k pi / (2n + 2)) at
    # |k| <= n (times M) and nothing else; phi_n(0) = cot(pi / (4n + 4))
    for n, M in ((3, 16), (7, 32), (12, 25)):
        t = 2 * math.pi * np.arange(M) / M
        c = np.fft.fft(O.trig_poly(n, t)) / M
        for k in range(M):
            kk = k if k <= M // 2 else k - M
            expect = math.cos(kk * math.pi / (2 * n + 2)) if abs(kk) <= n else 0.0
            assert abs(c[k] - expect) < 1e-12, (n, k)
        assert abs(O.trig_poly(n, np.zeros(1))[0] - 1 / math.tan(math.pi / (4 * n + 4))) < 1e-12


def test_trig_input_waves_tensor_and_radial():
    W, n_grid, d, lam, amax = 32, 64, 0.1, 0.025, 0.02
    n = O.trig_degree(lam, amax, n_grid * d)
    assert n == round(amax * n_grid * d / lam)
    u = O.input_wave_window(2, W, n_grid, n_grid, d, d, lam, amax, 0.0, 0.0, 0.0)
    phi = O.trig_poly(n, 2 * math.pi * (np.arange(W) - W // 2) / n_grid)
    assert np.allclose(u.real, np.outer(phi, phi), atol=1e-13, rtol=0) and np.all(u.imag == 0)
    assert abs(u[W // 2, W // 2] - (1 / math.tan(math.pi / (4 * n + 4))) ** 2) < 1e-10
    ur = O.input_wave_window(3, W, n_grid, n_grid, d, d, lam, amax, 0.0, 0.0, 0.0)
    off = np.arange(W) - W // 2
    r = np.hypot(off[:, None], off[None, :])
    for a, b in ((3, 4), (0, 5), (5, 12), (6, 8)):     # equal radii -> equal values
        pts = [(a, b), (b, a), (-a, b), (a, -b)]
        vals = [ur[W // 2 + y, W // 2 + x] for y, x in pts]
        assert np.ptp(np.real(vals)) < 1e-13
    assert abs(ur[W // 2, W // 2 + 5] - ur[W // 2 + 3, W // 2 + 4]) < 1e-13 and r[W // 2 + 3, W // 2 + 4] == 5


# ---- closed-form coefficients of the tensor trigonometric input waves (Sec. 2, Sec. 4.2.3) ----

def test_trig_basis_matrix_maps_translate_coefficients_to_fourier_coefficients():
    """Brute force: sample sum_j a_j phi_n(t - 2 pi j / (2n + 1)) on 4n + 8 points, take its
    Fourier coefficients with numpy's FFT, and compare with M a; M^-1 is the matrix inverse."""
    rng = np.random.default_rng(41)
    for n in (1, 3, 7):
        a = rng.standard_normal(2 * n + 1) + 1j * rng.standard_normal(2 * n + 1)
        npts = 4 * n + 8
        t = 2 * np.pi * np.arange(npts) / npts
        f = sum(a[j] * O.trig_poly(n, t - 2 * np.pi * j / (2 * n + 1)) for j in range(2 * n + 1))
        c = np.fft.fft(f) / npts
        c_k = c[np.mod(np.arange(-n, n + 1), npts)]
        M = O.trig_basis_matrix(n)
        assert np.max(np.abs(M @ a - c_k)) < 1e-12 * np.max(np.abs(c_k))
        Minv = O.trig_basis_inverse(n)
        assert np.max(np.abs(Minv - np.linalg.inv(M))) < 1e-12 * np.max(np.abs(Minv))
        assert np.max(np.abs(Minv @ M - np.eye(2 * n + 1))) < 1e-12


def _trig_full_period_translates(n, N, offsets):
    """Columns u_j on the full N x N grid: phi_n(2 pi (x - d_x) / N) phi_n(2 pi (y - d_y) / N)."""
    x = np.arange(N)
    cols = []
    for dx_, dy_ in offsets:
        ux = O.trig_poly(n, 2 * np.pi * (x - dx_) / N)
        uy = O.trig_poly(n, 2 * np.pi * (x - dy_) / N)
        cols.append(np.outer(uy, ux).ravel())
    return np.stack(cols, axis=1)


def test_trig_closed_coefficients_reconstruct_every_band_limited_wave():
    """A random wave with DFT coefficients only at |k_x|, |k_y| <= n is rebuilt exactly from all
    full-period translates of the lattice, for m = 2n + 1 translates per axis (the paper's
    M^-1) and for denser lattices on power-of-two grids (m = 8, 16 > 2n + 1), with zero and
    nonzero lattice offsets; least squares (numpy's minimum-norm solution) over the same
    translates gives the same coefficients."""
    rng = np.random.default_rng(42)
    for n, N, m, off in ((2, 15, 5, (0, 0)), (3, 28, 7, (1, 2)), (3, 16, 8, (1, 0)), (2, 32, 16, (0, 1))):
        s = N // m
        spec = np.zeros((N, N), dtype=np.complex128)
        ks = np.mod(np.arange(-n, n + 1), N)
        spec[ks[:, None], ks[None, :]] = rng.standard_normal((2 * n + 1, 2 * n + 1)) + \
            1j * rng.standard_normal((2 * n + 1, 2 * n + 1))
        f = np.fft.ifft2(spec)
        offsets = np.array([(off[0] + jx * s, off[1] + jy * s) for jy in range(m) for jx in range(m)])
        a = O.trig_closed_coefficients(f, n, offsets, (m, m))
        A = _trig_full_period_translates(n, N, offsets)
        assert np.max(np.abs(A @ a - f.ravel())) < 1e-12 * np.max(np.abs(f))
        a_ls = np.linalg.lstsq(A, f.ravel(), rcond=None)[0]
        assert np.max(np.abs(a_ls - a)) < 1e-10 * np.max(np.abs(a))


def test_trig_closed_coefficients_of_a_probe_on_a_periodic_window():
    """W = N (the window is the whole period): a probe whose aperture lies inside |k| <= n is
    represented with zero error by the closed-form coefficients of all translates, and the
    coefficients decay away from the probe (the translates are localized)."""
    n, s = 3, 4
    N = s * (2 * n + 1)
    dx = 0.5
    lam = 0.02508
    alpha = 2.5 * lam / (N * dx)          # aperture radius 2.5 Fourier pixels < n
    psi0 = O.probe(N, N, dx, dx, lam, alpha)
    uW = O.input_wave_window(2, N, N, N, dx, dx, lam, alpha, 0.0, 0.0, 0.0, degree=n)
    offsets = np.array([(jx * s - (N // 2 // s) * s, jy * s - (N // 2 // s) * s)
                        for jy in range(2 * n + 1) for jx in range(2 * n + 1)])
    cs = O.coefficients_closed(psi0, uW, offsets, n)
    assert cs.err_sup < 1e-12 and cs.err_l2 < 1e-12
    d = np.hypot(offsets[:, 0], offsets[:, 1])
    assert np.abs(cs.alpha[d == 0]).max() > 4 * np.abs(cs.alpha[d >= 3 * s]).max()


# ---- helpers: detector masks, coefficient classes, window crops ----

def test_detector_masks_are_annuli_of_the_right_size():
    """r1 <= lambda |k| < r2 on the D x D window: 4-fold symmetric, empty outside the bandlimit,
    and an annulus inside the band holds pi (k2^2 - k1^2) Fourier pixels up to its rim
    (k = r / (lambda q), q = 1 / (D dx)); a mistaken angle scale (k instead of lambda k, a lost
    factor 2 pi, pixels in place of Angstrom) moves the count far outside that bound."""
    D, dx, lam = 128, 0.125, 0.02508
    q = 1.0 / (D * dx)
    for r1, r2 in ((0.0, 0.02), (0.02, 0.05), (0.03, 0.066)):
        m = O.detector_mask(D, dx, dx, lam, r1, r2, 2 / 3)
        assert np.array_equal(m, m.T) and np.array_equal(m, np.roll(m[::-1, :], 1, axis=0))
        k1, k2 = r1 / (lam * q), r2 / (lam * q)
        area = np.pi * (k2 ** 2 - k1 ** 2)
        assert abs(m.sum() - area) <= 2 * np.pi * (k1 + k2) + 4, (r1, r2, m.sum(), area)
    outside = O.detector_mask(D, dx, dx, lam, 0.0, 1.0, 2 / 3) ^ O.detector_mask(D, dx, dx, lam, 0.0, 1.0, None)
    assert not np.any(outside & O.bandlimit_mask(D, D, 2 / 3))


def test_coefficient_classes_follow_case_1_and_case_2():
    """Sec. 4.2.1: probes on the input lattice's period share one coefficient set (Case 1,
    R = cP); probes every p = r / c pixels fall into c x d classes (Case 2)."""
    probes1 = [(x, y) for x in range(0, 64, 4) for y in range(0, 64, 4)]
    assert len({O.class_key(p, (4, 4), (2, 2), 1) for p in probes1}) == 1
    probes2 = [(x, y) for x in range(0, 64, 2) for y in range(0, 64, 1)]
    assert len({O.class_key(p, (4, 4), (2, 2), 1) for p in probes2}) == 2 * 4
    # f = 2 keeps every other input wave: the period doubles
    assert len({O.class_key(p, (4, 4), (2, 2), 2) for p in probes1}) == 4


def test_periodic_crop_and_embed_window_invert_each_other():
    rng = np.random.default_rng(43)
    a = rng.standard_normal((16, 24)) + 1j * rng.standard_normal((16, 24))
    win = O.periodic_crop(a, -3, 20, 8, 8)                 # wraps on both axes
    full = O.embed_window(win, -3, 20, 16, 24)
    iy = np.mod(-3 + np.arange(8), 16)
    ix = np.mod(20 + np.arange(8), 24)
    keep = np.zeros((16, 24), bool)
    keep[iy[:, None], ix[None, :]] = True
    assert np.array_equal(full[keep], a[keep]) and not np.any(full[~keep])


def test_l_nearest_sets_reproduce_the_paper_partition_counts():
    """Sec. 4.2.4 prints the minimum number of Multislice runs T_P = |union of I_{f,p,L}| of a
    48 x 48 sub-image: 1077 for L = 75 and 953 for L = 51 (u = probe, I = P + p/2, f = 2,
    512 pixels, 158 probes per axis). With probes and input waves on whole pixels (floor of
    their positions), I_f keeping the even input waves and the sub-image at probes 1..48,
    the oracle's L-nearest rule gives both numbers."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    gv = g["partition_minimum_runs"]
    X, P = 512, 158
    axis = np.array([int(np.floor((k + 0.5) * X / P)) for k in range(0, P, 2)])
    lattice = np.stack(np.meshgrid(axis, axis, indexing="xy"), axis=-1).reshape(-1, 2)
    probes = [int(np.floor(i * X / P)) for i in range(1, 49)]
    for L, key in ((75, "L75"), (51, "L51")):
        union = set()
        for py in probes:
            for px in probes:
                idx, _ = O.nearest_translates((px, py), lattice, L, X, X)
                union.update(int(i) for i in idx)
        assert len(union) == gv[key], (L, len(union))


def test_row_by_row_partition_of_the_paper_at_L51():
    """Sec. 4.2.4's partition figure, bottom row (L = 51): row by row gives l = 12 parts and
    T = 953, the union itself, so no translate is recomputed. The caption gives no M; in the
    whole-pixel geometry of the partition-count pin, M = 280 reproduces the printed pair. A
    cost that drops the overlap term gives 3350; a part that overruns M fails the bound check."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    gv = g["partition_row_by_row_L51"]
    X, P = 512, 158
    axis = np.array([int(np.floor((k + 0.5) * X / P)) for k in range(0, P, 2)])
    lattice = np.stack(np.meshgrid(axis, axis, indexing="xy"), axis=-1).reshape(-1, 2)
    probes = [int(np.floor(i * X / P)) for i in range(1, 49)]
    sets = [frozenset(int(i) for i in O.nearest_translates((px, py), lattice, 51, X, X)[0])
            for py in probes for px in probes]
    parts = O.partition_rows(sets, 48, 48, 280)
    assert len(parts) == gv["parts"]
    assert all(len(frozenset().union(*[sets[q] for q in part])) <= 280 for part in parts)
    assert O.partition_cost(sets, parts) == gv["T"]


def test_cost_model_reproduces_the_realspace_crossover_of_the_paper():
    """Sec. 4.2.1: on a 2048^2 domain with a 25 x 25 kernel, real-space propagation on X/f
    windows costs no more than Fourier propagation iff f >= 4. The two image costs are
    compared for every f from 1 to 8, and the closed-form crossover falls in (3, 4]. Natural
    logarithms would move the boundary to f = 5, a dropped factor 1/2 to f = 6, and Fourier
    runs costed on the X' x Y' windows would make real space never cheaper."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    gv = g["realspace_crossover"]
    X, Y, K = gv["X"], gv["Y"], (gv["K1"], gv["K2"])
    n_I, N, n_P, L = 4096, 100, 16384, 32
    cheaper = [f for f in range(1, 9)
               if O.lma_ops(n_I, f, N, X, Y, n_P, L, X // f, Y // f, K=K)
               <= O.lma_ops(n_I, f, N, X, Y, n_P, L, X // f, Y // f)]
    assert cheaper == list(range(gv["f_min"], 9))
    c = O.realspace_crossover_f(X, Y, *K)
    assert gv["f_min"] - 1 < c <= gv["f_min"]
    # at f = 1 on the full domain the first summands stand in the per-run ratio of Sec. 3.2
    r = O.multislice_ops(1, X, Y, K) / O.multislice_ops(1, X, Y)
    assert abs(r - (1 + 625) / (2 + 2 * 22)) < 1e-12


@pytest.mark.parametrize("L", [8, 16, 48])
def test_image_error_is_bounded_by_the_probe_approximation_error(L):
    """Sec. 4.2.3 observes image errors below the probe approximation error. With W = D = X it
    is a theorem: transmission (|t| = 1) and the bandlimited propagator (|P| <= 1) never raise
    the L2 norm, so multislice maps the probe residual psi_p - sum alpha u to an exit-wave
    residual no larger; a reading is the squared norm of a projection of the spectrum (1/D^2
    Parseval), so |sqrt(I_LMA) - sqrt(I_std)| <= err_l2 for a unit-norm probe, per probe and
    detector. Probe input waves on a 2-pixel lattice give errors of 0 to 6 %, and the bound
    is nearly attained (up to 0.97 of it), so a misplaced translate or a wrongly normalised
    residual or reading breaks it."""
    prm = _small_params(kind=1, L=L, n_slices=3, in_spacing=(2, 2), in_offset=(1, 1))
    at = _tiny_specimen(prm, seed=21)
    orc = O.LmaOracle(prm)
    orc.set_specimen([at], (300.0, 150.0), (0.7, 0.3), (0.15, 0.5), 3.0)
    probes = O.region_probes(3, 1, 4, 4, (5, 7), 64, 64)
    dets = [_Det(0.0, 0.02), _Det(0.02, 0.05), _Det(0.0, 1.0)]
    img = orc.image(dets, probes)
    std = O.standard_image(prm, orc.transmission_stack(0), dets, probes)
    errs = np.array([orc.coefficient_set(tuple(int(v) for v in p))[0].err_l2 for p in probes])
    assert 1e-3 < errs.max() < 0.1
    gap = np.abs(np.sqrt(img) - np.sqrt(std))
    assert np.all(gap <= errs[None, :] * (1 + 1e-12) + 1e-14), (gap / errs[None, :]).max()
