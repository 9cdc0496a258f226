"""Plain FP64 CPU oracle for the Lattice Multislice Algorithm (LMA) hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. The CUDA library never
calls it and shares no code, table or constant with it.

Everything is numpy float64 / complex128, written for a reader who checks it
against the paper by eye: no blocking, no fusion, no reordering. Library
primitives used as steps: ``numpy.fft`` (DFT), ``numpy.linalg.lstsq`` (least
squares), ``numpy.lexsort`` (ordering).

Conventions (fixed here because the paper leaves them open):
  * arrays are indexed [y, x]; pixel j sits at j*dx, periodic boundaries
    (Sec. 3.1: the simulation domain is periodic because of the DFT);
  * frequencies are in FFT order, k_m = m'/(n*d) with m' = m for m < n/2 else
    m - n; this is the paper's centred g(k) of Sec. 4.1 after an fftshift;
  * the forward DFT is unnormalised with kernel exp(-2 pi i k.x), the inverse
    carries 1/n^2 (numpy's convention);
  * the bandlimit mask keeps (m'/nx)^2 + (n'/ny)^2 <= (frac/2)^2 (2/3 of
    Nyquist by default). The paper does not discuss anti-aliasing; the mask is
    applied in the propagation step only;
  * the detector collects r1 <= lambda*|k| < r2 on the detection window,
    intersected with the same bandlimit mask (eq. for 2D STEM, Sec. 3.1).

Parity pins for every function live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, List, Sequence, Tuple

import numpy as np

# CODATA 2018 exact / recommended values (SI).
_H = 6.62607015e-34
_C = 299792458.0
_M0 = 9.1093837015e-31
_E = 1.602176634e-19


# ----------------------------------------------------------------------------
# electron optics constants
# ----------------------------------------------------------------------------

def electron_wavelength(voltage: float) -> float:
    """Relativistic electron wavelength in Angstrom for an accelerating voltage in V.

    lambda = h c / sqrt(E (2 m0 c^2 + E)), E = e V. The paper quotes
    lambda = 0.0250793 A for 200 kV (captions of the Sec. 4.2.3 figures).
    """
    energy = _E * voltage
    mc2 = _M0 * _C * _C
    return _H * _C / math.sqrt(energy * (2.0 * mc2 + energy)) * 1e10


def interaction_constant(voltage: float) -> float:
    """Beam-sample interaction constant sigma of eq. schroedinger_equation, rad/(V*A).

    sigma = 2 pi / (lambda V) * (m0 c^2 + E) / (2 m0 c^2 + E).
    """
    energy = _E * voltage
    mc2 = _M0 * _C * _C
    lam = electron_wavelength(voltage)
    return 2.0 * math.pi / (lam * voltage) * (mc2 + energy) / (2.0 * mc2 + energy)


def gaussian_width(lam: float, alpha_max: float) -> float:
    """Gaussian input-wave width sigma = lambda / (2 alpha_max) (Sec. 4.2.3, Gaussians)."""
    return lam / (2.0 * alpha_max)


# ----------------------------------------------------------------------------
# grids and transforms
# ----------------------------------------------------------------------------

def signed_index(n: int) -> np.ndarray:
    """m' for m = 0..n-1 in FFT order (m' = m for m < n/2, else m - n)."""
    m = np.arange(n)
    return np.where(m < (n + 1) // 2, m, m - n)


def freqs(n: int, d: float) -> np.ndarray:
    """Spatial frequencies k_m = m' / (n d) in FFT order (1/Angstrom)."""
    return signed_index(n) / (n * d)


def dft2(a: np.ndarray) -> np.ndarray:
    """Unnormalised forward 2D DFT with kernel exp(-2 pi i k.x)."""
    return np.fft.fft2(a)


def idft2(a: np.ndarray) -> np.ndarray:
    """Inverse 2D DFT with the 1/(nx ny) factor."""
    return np.fft.ifft2(a)


def k_squared(ny: int, nx: int, dy: float, dx: float) -> np.ndarray:
    """|k|^2 on the [ny, nx] frequency grid."""
    ky = freqs(ny, dy)[:, None]
    kx = freqs(nx, dx)[None, :]
    return ky * ky + kx * kx


def bandlimit_mask(ny: int, nx: int, frac: float) -> np.ndarray:
    """Circular bandlimit: (m'/nx)^2 + (n'/ny)^2 <= (frac/2)^2, decided in FP64.

    For a square n-point window and frac = 2/3 this is 9 (m'^2 + n'^2) <= n^2.
    """
    my = signed_index(ny)[:, None] / ny
    mx = signed_index(nx)[None, :] / nx
    if ny == nx:
        # exact integer form for square windows: 4 (m'^2 + n'^2) <= frac^2 n^2
        iy = signed_index(ny)[:, None].astype(np.int64)
        ix = signed_index(nx)[None, :].astype(np.int64)
        return (4 * (iy * iy + ix * ix)).astype(np.float64) <= frac * frac * nx * nx
    return my * my + mx * mx <= 0.25 * frac * frac


# ----------------------------------------------------------------------------
# physics model (Sec. 3.1 and Sec. 3.2)
# ----------------------------------------------------------------------------

def aberration(k2: np.ndarray, lam: float, cs: float, defocus: float) -> np.ndarray:
    """chi(k) = 1/2 pi Cs lambda^3 |k|^4 - pi Z lambda |k|^2 (eq. aberration_function)."""
    return 0.5 * math.pi * cs * lam ** 3 * k2 * k2 - math.pi * defocus * lam * k2


def aperture(k2: np.ndarray, lam: float, alpha_max: float) -> np.ndarray:
    """A(k) = 1 iff lambda |k| < alpha_max (eq. aperture_function, strict)."""
    return (lam * np.sqrt(k2) < alpha_max).astype(np.float64)


def probe(ny: int, nx: int, dy: float, dx: float, lam: float, alpha_max: float,
          cs: float = 0.0, defocus: float = 0.0, p: Tuple[float, float] = (0.0, 0.0)
          ) -> np.ndarray:
    """STEM probe psi_p^init on the full periodic grid (eq. probe_wave_function).

    Fourier values exp(-i chi) A mu_{-p}, mu_p(k) = exp(2 pi i k.p) (Sec. 4.1),
    inverse DFT, then normalised so that sum |psi|^2 = 1. ``p`` = (py, px) in
    Angstrom.
    """
    k2 = k_squared(ny, nx, dy, dx)
    ky = freqs(ny, dy)[:, None]
    kx = freqs(nx, dx)[None, :]
    spec = np.exp(-1j * aberration(k2, lam, cs, defocus)) * aperture(k2, lam, alpha_max)
    spec = spec * np.exp(-2j * math.pi * (ky * p[0] + kx * p[1]))
    psi = idft2(spec)
    return psi / math.sqrt(float(np.sum(np.abs(psi) ** 2)))


def fresnel_propagator(ny: int, nx: int, dy: float, dx: float, lam: float, dz: float,
                       frac: float | None) -> np.ndarray:
    """Fourier-space propagation factor for one slice of thickness dz.

    The propagation term of eq. schroedinger_equation, d psi/dz = (i lambda/4pi)
    Laplacian psi, becomes d psi^/dz = -i pi lambda |k|^2 psi^ for the forward
    DFT exp(-2 pi i k.x); over dz this is exp(-i pi lambda dz |k|^2), the DFT of
    the real-space kernel q of Sec. 3.2. Multiplied by the bandlimit mask when
    ``frac`` is given.
    """
    prop = np.exp(-1j * math.pi * lam * dz * k_squared(ny, nx, dy, dx))
    if frac is not None:
        prop = prop * bandlimit_mask(ny, nx, frac)
    return prop


def kernel_offsets(K: int) -> np.ndarray:
    """Offsets -floor(K/2) .. K - 1 - floor(K/2) of a K-pixel kernel axis (K = n covers every
    residue of an n-pixel periodic axis once)."""
    return np.arange(K) - K // 2


def realspace_kernel(prop: np.ndarray, K1: int, K2: int) -> np.ndarray:
    """q discretized to K1 x K2 pixels (Sec. 3.2, complexity paragraph): the real-space
    kernel of the window's Fourier propagator, q = IDFT(prop), at the offsets
    kernel_offsets(K2) (y) x kernel_offsets(K1) (x), shape (K2, K1). With K1 = K2 = n the
    convolution with it is the Fourier-space propagation exactly."""
    q = idft2(prop)
    ny, nx = prop.shape
    oy, ox = kernel_offsets(K2), kernel_offsets(K1)
    return q[np.ix_(oy % ny, ox % nx)]


def convolve_periodic(psi: np.ndarray, qK: np.ndarray) -> np.ndarray:
    """(q * psi)(x) = sum over kernel offsets d of q(d) psi(x - d), periodic on the window."""
    K2, K1 = qK.shape
    out = np.zeros_like(psi)
    for iy, dy in enumerate(kernel_offsets(K2)):
        for ix, dx in enumerate(kernel_offsets(K1)):
            out += qK[iy, ix] * np.roll(psi, (int(dy), int(dx)), axis=(0, 1))
    return out


def multislice_realspace(psi: np.ndarray, t: Sequence[np.ndarray], qK: np.ndarray) -> np.ndarray:
    """The multislice pseudocode with the propagation step as a real-space convolution
    with the K1 x K2 kernel: for each slice transmit, then convolve."""
    for ts in t:
        psi = convolve_periodic(ts * psi, qK)
    return psi


def projected_potential(x: np.ndarray, y: np.ndarray, slc: np.ndarray, species: np.ndarray,
                        n_slices: int, ny: int, nx: int, ly: float, lx: float,
                        peak: Sequence[float], term_frac: Sequence[float],
                        term_width: Sequence[float], r_cut: float) -> np.ndarray:
    """Projected potential v_s(x) per slice (V*A) on the periodic grid.

    v_s(x_j) = sum over atoms a of slice s, over periodic images with r < r_cut,
    of peak[species(a)] * sum_t term_frac[t] exp(-r^2 / (2 term_width[t]^2)).
    The integral over the slice of Sec. 3.2 (v_eps) is given directly as this
    Gaussian-sum model.
    """
    dx = lx / nx
    dy = ly / ny
    v = np.zeros((n_slices, ny, nx), dtype=np.float64)
    jx_lo_off = int(math.ceil(r_cut / dx)) + 1
    jy_lo_off = int(math.ceil(r_cut / dy)) + 1
    for a in range(x.shape[0]):
        xa, ya, s = float(x[a]), float(y[a]), int(slc[a])
        # unwrapped pixel indices around the atom: each one is one (pixel, image) pair
        cx = int(math.floor(xa / dx))
        cy = int(math.floor(ya / dy))
        jx = np.arange(cx - jx_lo_off, cx + jx_lo_off + 1)
        jy = np.arange(cy - jy_lo_off, cy + jy_lo_off + 1)
        rx = jx * dx - xa
        ry = jy * dy - ya
        r2 = ry[:, None] ** 2 + rx[None, :] ** 2
        inside = r2 < r_cut * r_cut
        val = np.zeros_like(r2)
        for f, w in zip(term_frac, term_width):
            val += f * np.exp(-r2 / (2.0 * w * w))
        val = np.where(inside, float(peak[int(species[a])]) * val, 0.0)
        np.add.at(v[s], (np.mod(jy, ny)[:, None], np.mod(jx, nx)[None, :]), val)
    return v


def transmission(v: np.ndarray, sigma: float) -> np.ndarray:
    """t = exp(i sigma v_eps) (Sec. 3.2)."""
    return np.exp(1j * sigma * v)


def multislice(psi: np.ndarray, t: Sequence[np.ndarray], prop: np.ndarray) -> np.ndarray:
    """Standard multislice (Fig. multislice_pseudocode): for each slice, transmit then propagate."""
    psi = np.array(psi, dtype=np.complex128)
    for ts in t:
        psi = psi * ts
        psi = idft2(prop * dft2(psi))
    return psi


def periodic_crop(a: np.ndarray, oy: int, ox: int, h: int, w: int) -> np.ndarray:
    """a[(oy + 0..h-1) mod ny, (ox + 0..w-1) mod nx] (last two axes)."""
    ny, nx = a.shape[-2], a.shape[-1]
    iy = np.mod(oy + np.arange(h), ny)
    ix = np.mod(ox + np.arange(w), nx)
    return a[..., iy[:, None], ix[None, :]]


def detector_mask(n: int, dy: float, dx: float, lam: float, r1: float, r2: float,
                  frac: float | None) -> np.ndarray:
    """Pixels of an n x n window with r1 <= lambda |k| < r2, intersected with the bandlimit."""
    ang = lam * np.sqrt(k_squared(n, n, dy, dx))
    m = (ang >= r1) & (ang < r2)
    if frac is not None:
        m &= bandlimit_mask(n, n, frac)
    return m


def detect(psi: np.ndarray, mask: np.ndarray) -> float:
    """2D STEM reading (Sec. 3.1): (1/n^2) sum over the detector of |DFT(psi)|^2.

    With a unit-norm probe this is the fraction of the incident intensity that
    reaches the detector.
    """
    spec = dft2(psi)
    return float(np.sum(np.abs(spec[mask]) ** 2) / psi.size)


def ring_masks(n: int, dy: float, dx: float, lam: float, width: float, n_rings: int,
               frac: float | None) -> List[np.ndarray]:
    """3D STEM detector (Sec. 3.1): ring a collects a*width <= lambda |k| < (a+1)*width,
    a = 0..n_rings-1, each intersected with the bandlimit like the 2D detector."""
    return [detector_mask(n, dy, dx, lam, a * width, (a + 1) * width, frac) for a in range(n_rings)]


def pattern(psi: np.ndarray, A: int, B: int, frac: float | None) -> np.ndarray:
    """4D STEM reading (Sec. 3.1): |DFT(psi)|^2 / n^2 at the frequencies (a, b) * (1/(n dx),
    1/(n dy)) for a = -A..A, b = -B..B, shape (2B+1, 2A+1) indexed [b + B, a + A]; zero
    outside the bandlimit. With a unit-norm wave the entries are fractions of the incident
    intensity, and summing them over an annulus gives the 2D STEM reading."""
    ny, nx = psi.shape
    spec = np.abs(dft2(psi)) ** 2 / psi.size
    if frac is not None:
        spec = np.where(bandlimit_mask(ny, nx, frac), spec, 0.0)
    out = np.zeros((2 * B + 1, 2 * A + 1), dtype=np.float64)
    for b in range(-B, B + 1):
        for a in range(-A, A + 1):
            out[b + B, a + A] = spec[b % ny, a % nx]
    return out


# ----------------------------------------------------------------------------
# LMA geometry (Sec. 4.2.1, 4.2.2)
# ----------------------------------------------------------------------------

def input_lattice(nx: int, ny: int, spacing: Tuple[int, int], offset: Tuple[int, int],
                  f: int) -> np.ndarray:
    """Pixel positions of I_f (Sec. 4.2.1, option (i)), shape (R_y/f * R_x/f, 2) as (x, y).

    I = {a r_x e1 + b r_y e2 + I_offset}, with R_x r_x = X covering the periodic
    domain, and I_f keeps every f-th point in both directions. Raster order:
    index = b * (R_x/f) + a.
    """
    sx, sy = spacing
    if nx % sx or ny % sy:
        raise ValueError("input lattice does not cover the grid")
    rx, ry = nx // sx, ny // sy
    if rx % f or ry % f:
        raise ValueError("R must be a multiple of f")
    a = np.arange(rx // f)
    b = np.arange(ry // f)
    xs = (offset[0] + a * f * sx) % nx
    ys = (offset[1] + b * f * sy) % ny
    out = np.empty((ys.size * xs.size, 2), dtype=np.int64)
    out[:, 0] = np.tile(xs, ys.size)
    out[:, 1] = np.repeat(ys, xs.size)
    return out


def min_image(d: np.ndarray, n: int) -> np.ndarray:
    """Signed minimum-image offset in [-n/2, n/2)."""
    return np.mod(d + n // 2, n) - n // 2


def nearest_translates(p: Tuple[int, int], lattice: np.ndarray, L: int, nx: int, ny: int
                       ) -> Tuple[np.ndarray, np.ndarray]:
    """I_{f,p,L}: the L input waves closest to p (Sec. 4.2.1, option (iii)).

    Distance is the periodic minimum-image distance. Ties are broken by
    (distance^2, dy, dx) ascending on the signed offsets. Returns (indices into
    ``lattice``, offsets (L, 2) as (dx, dy) in pixels).
    """
    if L > lattice.shape[0]:
        raise ValueError("L exceeds |I_f|")
    ddx = min_image(lattice[:, 0] - p[0], nx)
    ddy = min_image(lattice[:, 1] - p[1], ny)
    d2 = ddx * ddx + ddy * ddy
    order = np.lexsort((ddx, ddy, d2))[:L]
    return order, np.stack([ddx[order], ddy[order]], axis=1)


def class_key(p: Tuple[int, int], spacing: Tuple[int, int], offset: Tuple[int, int], f: int
              ) -> Tuple[int, int]:
    """Position of p relative to the I_f lattice; probes with equal keys share coefficients.

    Case 1 (R = cP) gives a single key, Case 2 (P = cR) gives c*d keys
    (eqs. lma_approximation_exit1 / exit2).
    """
    return ((p[0] - offset[0]) % (f * spacing[0]), (p[1] - offset[1]) % (f * spacing[1]))


def trig_poly(n: int, t: np.ndarray) -> np.ndarray:
    """phi_n(t) = sum_{k=-n..n} e^{ikt} cos(k pi / (2n + 2)) (Sec. 4.2.3, trigonometric
    polynomials), real and even: 1 + 2 sum_{k=1..n} cos(k t) cos(k pi / (2n + 2))."""
    out = np.ones_like(t, dtype=np.float64)
    for k in range(1, n + 1):
        out = out + 2.0 * np.cos(k * t) * math.cos(k * math.pi / (2 * n + 2))
    return out


def trig_degree(lam: float, alpha_max: float, lx: float) -> int:
    """n = (alpha_max / lambda) / q with the Fourier pixel q = 1 / l_x, rounded to an integer."""
    return int(round(alpha_max * lx / lam))


def input_wave_window(kind: int, W: int, ny: int, nx: int, dy: float, dx: float, lam: float,
                      alpha_max: float, cs: float, defocus: float, gauss_sigma: float,
                      degree: int = 0) -> np.ndarray:
    """The input wave u sampled on a W x W window with its centre at window pixel (W/2, W/2).

    kind 0: Gaussian g_sigma (Sec. 4.2.3, Gaussians), sigma = lambda/(2 alpha_max)
    unless given; kind 1: the probe itself, u = psi_0^init (Sec. 4.2.3); kind 2: the tensor
    product phi_n(2 pi x / l_x) phi_n(2 pi y / l_y) of trigonometric polynomials; kind 3: the
    radial phi_n(2 pi |v| / l_x). Degree n = ``degree`` or trig_degree(). Offsets from the
    centre run over [-W/2, W/2), taken periodically on the full grid.
    """
    off = np.arange(W) - W // 2
    if kind in (2, 3):
        n = degree if degree > 0 else trig_degree(lam, alpha_max, nx * dx)
        if kind == 2:
            return np.outer(trig_poly(n, 2 * math.pi * off / ny), trig_poly(n, 2 * math.pi * off / nx)
                            ).astype(np.complex128)
        r = np.sqrt((off[:, None] * dy) ** 2 + (off[None, :] * dx) ** 2)
        return trig_poly(n, 2 * math.pi * r / (nx * dx)).astype(np.complex128)
    if kind == 0:
        s = gauss_sigma if gauss_sigma > 0 else gaussian_width(lam, alpha_max)
        ry = off * dy
        rx = off * dx
        r2 = ry[:, None] ** 2 + rx[None, :] ** 2
        return np.exp(-r2 / (2.0 * s * s)).astype(np.complex128)
    if kind == 1:
        p0 = probe(ny, nx, dy, dx, lam, alpha_max, cs, defocus)
        return periodic_crop(p0, -(W // 2), -(W // 2), W, W)
    raise ValueError("unknown input wave kind")


def embed_window(wave: np.ndarray, oy: int, ox: int, ny: int, nx: int) -> np.ndarray:
    """Place a W x W window wave with origin (oy, ox) on the full periodic grid (zeros elsewhere)."""
    full = np.zeros((ny, nx), dtype=np.complex128)
    W = wave.shape[0]
    iy = np.mod(oy + np.arange(W), ny)
    ix = np.mod(ox + np.arange(W), nx)
    full[iy[:, None], ix[None, :]] += wave
    return full


@dataclass
class CoefficientSet:
    alpha: np.ndarray        # (L,) complex128
    offsets: np.ndarray      # (L, 2) int (dx, dy) of each translate relative to the probe
    err_l2: float            # relative Euclidean error of the probe approximation
    err_sup: float           # relative supremum error


def coefficients(psi0: np.ndarray, uW: np.ndarray, offsets: np.ndarray) -> CoefficientSet:
    """Least-squares coefficients for one probe (eqs. lma_approximation_exit1_0 / exit2_0).

    Relative coordinates: the probe ``psi0`` is centred at pixel (0, 0) of the
    full periodic grid and translate j sits at ``offsets[j]``; its window is
    [offset - W/2, offset + W/2). Solves min_alpha ||psi0 - sum_j alpha_j u_j||_2
    over the whole grid.
    """
    ny, nx = psi0.shape
    W = uW.shape[0]
    cols = [embed_window(uW, int(o[1]) - W // 2, int(o[0]) - W // 2, ny, nx).ravel()
            for o in offsets]
    A = np.stack(cols, axis=1)
    b = psi0.ravel()
    alpha = np.linalg.lstsq(A, b, rcond=None)[0]
    approx = A @ alpha
    err_l2 = float(np.linalg.norm(b - approx) / np.linalg.norm(b))
    err_sup = float(np.max(np.abs(b - approx)) / np.max(np.abs(b)))
    return CoefficientSet(alpha=alpha, offsets=np.asarray(offsets, dtype=np.int64),
                          err_l2=err_l2, err_sup=err_sup)


def trig_modulation_matrix(n: int) -> np.ndarray:
    """W[k, j] = exp(-2 pi i j k / (2n + 1)), k = -n..n (rows), j = 0..2n (columns).

    Sec. 2 writes the entries without the imaginary unit; with it, W carries the
    coefficients of the elementary waves e^{ikt} into those of the 2n + 1 equispaced
    translates t_j = 2 pi j / (2n + 1) (the reading taken here)."""
    k = np.arange(-n, n + 1)[:, None]
    j = np.arange(2 * n + 1)[None, :]
    return np.exp(-2j * math.pi * j * k / (2 * n + 1))


def trig_basis_matrix(n: int) -> np.ndarray:
    """M with c = M a: the coefficients c_k of a polynomial in T_n from the coefficients a_j of
    its expansion in the translates phi_n(t - t_j). phi_n(t - t_j) = sum_k w_k e^{-ik t_j} e^{ikt}
    with w_k = cos(k pi / (2n + 2)), so M = diag(w) W (Sec. 2 prints W diag(w))."""
    w = np.cos(np.arange(-n, n + 1) * math.pi / (2 * n + 2))
    return w[:, None] * trig_modulation_matrix(n)


def trig_basis_inverse(n: int) -> np.ndarray:
    """M^-1 = W^* diag(1 / w) / (2n + 1), from W W^* = (2n + 1) I. Sec. 2 prints the factor
    1 / (2n + 1)^2 and the factors in the other order; in two dimensions the tensor product
    of two of these carries 1 / (2n + 1)^2."""
    w = np.cos(np.arange(-n, n + 1) * math.pi / (2 * n + 2))
    return trig_modulation_matrix(n).conj().T / w[None, :] / (2 * n + 1)


def trig_closed_coefficients(psi0: np.ndarray, n: int, offsets: np.ndarray,
                             m: Tuple[int, int] | None = None) -> np.ndarray:
    """Closed-form coefficients of the tensor trigonometric input waves (Sec. 2, Sec. 4.2.3:
    no least squares) for the probe ``psi0`` centred at pixel (0, 0) of the full N_y x N_x
    grid and translates at ``offsets`` (dx, dy) relative to it, on a lattice of m = (m_x, m_y)
    translates per axis (default 2n + 1).

    With u(x, y) = phi_n(2 pi x / N_x) phi_n(2 pi y / N_y) and m = 2n + 1 translates per
    period, the probe's part in T_n x T_n (its DFT coefficients with |k_x|, |k_y| <= n) is
    sum_j a_j u_j with a_j the two-dimensional M^-1 applied to those coefficients; in the
    coordinates of the translate offset d = X_j - p this is
      a(d) = (m_x m_y)^-1 sum_{|k_x|,|k_y|<=n} P(k) / (N_x N_y w_kx w_ky) e^{2 pi i (k_x d_x / N_x + k_y d_y / N_y)},
    P the DFT of psi0. For m > 2n + 1 (a denser lattice, as on power-of-two grids, which
    2n + 1 never divides) the same sum with 1 / (m_x m_y) is again exact: the lattice sum of
    e^{2 pi i (k' - k) X_j / N} vanishes for k' != k when |k' - k| <= 2n < m; it is the
    minimum-norm representation. The DFT is numpy's; the sum is written out."""
    ny, nx = psi0.shape
    mx, my = m if m is not None else (2 * n + 1, 2 * n + 1)
    P = dft2(psi0)
    ks = np.arange(-n, n + 1)
    w = np.cos(ks * math.pi / (2 * n + 2))
    G = P[np.mod(ks, ny)[:, None], np.mod(ks, nx)[None, :]] / (nx * ny * w[:, None] * w[None, :])
    out = np.empty(len(offsets), dtype=np.complex128)
    for j, (dx_, dy_) in enumerate(np.asarray(offsets)):
        ph = np.exp(2j * math.pi * (ks[:, None] * dy_ / ny + ks[None, :] * dx_ / nx))
        out[j] = np.sum(G * ph) / (mx * my)
    return out


def coefficients_closed(psi0: np.ndarray, uW: np.ndarray, offsets: np.ndarray, n: int,
                        m: Tuple[int, int] | None = None) -> CoefficientSet:
    """Coefficient set with the closed-form trigonometric coefficients (lattice of m translates
    per axis) and the errors of the windowed approximation, measured as for the least-squares
    sets."""
    ny, nx = psi0.shape
    W = uW.shape[0]
    alpha = trig_closed_coefficients(psi0, n, offsets, m)
    approx = np.zeros((ny, nx), dtype=np.complex128)
    for a, o in zip(alpha, offsets):
        approx += a * embed_window(uW, int(o[1]) - W // 2, int(o[0]) - W // 2, ny, nx)
    err_l2 = float(np.linalg.norm(psi0 - approx) / np.linalg.norm(psi0))
    err_sup = float(np.max(np.abs(psi0 - approx)) / np.max(np.abs(psi0)))
    return CoefficientSet(alpha=alpha, offsets=np.asarray(offsets, dtype=np.int64),
                          err_l2=err_l2, err_sup=err_sup)


# ----------------------------------------------------------------------------
# LMA steps (Fig. lma_pseudocode)
# ----------------------------------------------------------------------------

def translate_exit_wave(uW: np.ndarray, t_full: np.ndarray, prop_W: np.ndarray,
                        pos: Tuple[int, int]) -> np.ndarray:
    """Step 1 for one input wave: multislice of u_i on its W x W window.

    The window is [i - W/2, i + W/2) of the periodic grid (option (ii)); the
    slices of ``t_full`` are cropped to it.
    """
    W = uW.shape[0]
    ts = periodic_crop(t_full, pos[1] - W // 2, pos[0] - W // 2, W, W)
    return multislice(uW, ts, prop_W)


def synthesize(U: Sequence[np.ndarray], alpha: np.ndarray, offsets: np.ndarray, D: int,
               cyclic: bool) -> np.ndarray:
    """Step 2: Psi_p = sum_j alpha_j U_{i_j} on the D x D window centred at p.

    U_{i_j} has its own window [i_j - W/2, i_j + W/2); relative to the probe
    window [p - D/2, p + D/2) it is shifted by offsets[j] + (D - W)/2 and
    truncated to the probe window. When the windows are the whole periodic grid
    (``cyclic``) the placement is a cyclic shift.
    """
    psi = np.zeros((D, D), dtype=np.complex128)
    for Uj, a, o in zip(U, alpha, offsets):
        W = Uj.shape[0]
        sx = int(o[0]) + (D - W) // 2
        sy = int(o[1]) + (D - W) // 2
        if cyclic:
            psi += a * np.roll(Uj, shift=(sy, sx), axis=(0, 1))
            continue
        y0, y1 = max(0, sy), min(D, sy + W)
        x0, x1 = max(0, sx), min(D, sx + W)
        if y0 < y1 and x0 < x1:
            psi[y0:y1, x0:x1] += a * Uj[y0 - sy:y1 - sy, x0 - sx:x1 - sx]
    return psi


@dataclass
class LmaParams:
    nx: int
    ny: int
    lx: float
    ly: float
    slice_dz: float
    n_slices: int
    lam: float
    sigma: float
    bandlimit_frac: float
    alpha_max: float
    cs: float
    defocus: float
    kind: int
    gauss_sigma: float
    in_spacing: Tuple[int, int]
    in_offset: Tuple[int, int]
    f: int
    L: int
    W: int
    D: int
    trig_degree: int = 0      # input wave kinds 2, 3: degree n of phi_n (0: from alpha_max l_x / lambda)
    coef_mode: int = 0        # 0: least squares; 1: closed-form trigonometric coefficients (kind 2)

    @property
    def degree(self) -> int:
        return self.trig_degree if self.trig_degree > 0 else trig_degree(self.lam, self.alpha_max, self.lx)

    @property
    def lattice_m(self) -> Tuple[int, int]:
        """Input waves per axis of the I_f lattice."""
        return (self.nx // (self.in_spacing[0] * self.f), self.ny // (self.in_spacing[1] * self.f))

    @property
    def dx(self) -> float:
        return self.lx / self.nx

    @property
    def dy(self) -> float:
        return self.ly / self.ny

    @property
    def cyclic(self) -> bool:
        return self.W == self.nx and self.W == self.ny and self.D == self.W


class LmaOracle:
    """The LMA image pipeline of Fig. lma_pseudocode in FP64.

    Construct with the grid, probe and basis parameters; call ``image`` with
    per-phonon atom lists, the potential model, detectors and probe positions.
    Exit waves are cached per (phonon, translate) so that sampled probes share
    propagations.
    """

    def __init__(self, prm: LmaParams, realspace: Tuple[int, int] | None = None):
        """``realspace`` = (K1, K2): propagate with the K1 x K2 real-space kernel instead of
        the Fourier step (Sec. 3.2)."""
        self.prm = prm
        p = prm
        self.lattice = input_lattice(p.nx, p.ny, p.in_spacing, p.in_offset, p.f)
        self.uW = input_wave_window(p.kind, p.W, p.ny, p.nx, p.dy, p.dx, p.lam, p.alpha_max,
                                    p.cs, p.defocus, p.gauss_sigma, p.trig_degree)
        self.prop_W = fresnel_propagator(p.W, p.W, p.dy, p.dx, p.lam, p.slice_dz,
                                         p.bandlimit_frac)
        self.qK = realspace_kernel(self.prop_W, realspace[0], realspace[1]) if realspace else None
        self._psi0 = None
        self._sets: Dict[Tuple[int, int], CoefficientSet] = {}
        self._t: Dict[int, np.ndarray] = {}
        self._U: Dict[Tuple[int, int], np.ndarray] = {}

    # -- coefficients -------------------------------------------------------
    @property
    def psi0(self) -> np.ndarray:
        if self._psi0 is None:
            p = self.prm
            self._psi0 = probe(p.ny, p.nx, p.dy, p.dx, p.lam, p.alpha_max, p.cs, p.defocus)
        return self._psi0

    def coefficient_set(self, p: Tuple[int, int]) -> Tuple[CoefficientSet, np.ndarray]:
        """Coefficients for probe pixel p and the lattice indices of its L translates."""
        prm = self.prm
        key = class_key(p, prm.in_spacing, prm.in_offset, prm.f)
        idx, offs = nearest_translates(p, self.lattice, prm.L, prm.nx, prm.ny)
        if key not in self._sets:
            if prm.coef_mode == 1:
                self._sets[key] = coefficients_closed(self.psi0, self.uW, offs, prm.degree, prm.lattice_m)
            else:
                self._sets[key] = coefficients(self.psi0, self.uW, offs)
        cs = self._sets[key]
        if not np.array_equal(cs.offsets, offs):
            raise AssertionError("coefficient reuse broken: offsets differ inside a class")
        return cs, idx

    # -- specimen -----------------------------------------------------------
    def set_specimen(self, phonons: Sequence, peak, term_frac, term_width, r_cut):
        self._phonons = list(phonons)
        self._pot = (tuple(peak), tuple(term_frac), tuple(term_width), float(r_cut))
        self._t.clear()
        self._U.clear()

    def transmission_stack(self, phi: int) -> np.ndarray:
        if phi not in self._t:
            p = self.prm
            at = self._phonons[phi]
            peak, tf, tw, rc = self._pot
            v = projected_potential(at.x, at.y, at.slice, at.species, p.n_slices, p.ny, p.nx,
                                    p.ly, p.lx, peak, tf, tw, rc)
            self._t[phi] = transmission(v, p.sigma)
        return self._t[phi]

    def exit_wave(self, phi: int, i: int) -> np.ndarray:
        if (phi, i) not in self._U:
            pos = (int(self.lattice[i, 0]), int(self.lattice[i, 1]))
            if self.qK is None:
                self._U[(phi, i)] = translate_exit_wave(self.uW, self.transmission_stack(phi),
                                                        self.prop_W, pos)
            else:
                W = self.prm.W
                ts = periodic_crop(self.transmission_stack(phi), pos[1] - W // 2, pos[0] - W // 2, W, W)
                self._U[(phi, i)] = multislice_realspace(self.uW, ts, self.qK)
        return self._U[(phi, i)]

    # -- image ----------------------------------------------------------------
    # the three steps after propagation; a restatement in another precision overrides them
    def _synthesize(self, U, alpha, offsets) -> np.ndarray:
        return synthesize(U, alpha, offsets, self.prm.D, self.prm.cyclic)

    def _detect(self, psi: np.ndarray, mask: np.ndarray) -> float:
        return detect(psi, mask)

    def _pattern(self, psi: np.ndarray, A: int, B: int) -> np.ndarray:
        return pattern(psi, A, B, self.prm.bandlimit_frac)

    def pixel(self, phi: int, p: Tuple[int, int], masks: Sequence[np.ndarray]) -> List[float]:
        cs, idx = self.coefficient_set(p)
        U = [self.exit_wave(phi, int(i)) for i in idx]
        psi = self._synthesize(U, cs.alpha, cs.offsets)
        return [self._detect(psi, m) for m in masks]

    def detector_masks(self, detectors) -> List[np.ndarray]:
        p = self.prm
        return [detector_mask(p.D, p.dy, p.dx, p.lam, d.r1, d.r2, p.bandlimit_frac)
                for d in detectors]

    def image(self, detectors, probes: np.ndarray) -> np.ndarray:
        """Phonon-averaged readings, shape (n_det, n_probes); probes (n, 2) pixel (x, y)."""
        masks = self.detector_masks(detectors)
        out = np.zeros((len(masks), probes.shape[0]), dtype=np.float64)
        nphi = len(self._phonons)
        for phi in range(nphi):
            for k, pr in enumerate(probes):
                out[:, k] += self.pixel(phi, (int(pr[0]), int(pr[1])), masks)
        return out / nphi

    def image_coherent(self, detectors, probes: np.ndarray, variants: Sequence[Tuple[float, float, float]]
                       ) -> np.ndarray:
        """Partial coherence (Sec. 1: the simulation repeated with slightly different probe
        parameters and averaged): for each variant (defocus, C_s, weight) the coefficients
        are fitted to that probe with the same input waves, and the images are averaged with
        the normalised weights. The exit waves do not depend on the probe, so every variant
        reuses them."""
        p = self.prm
        masks = self.detector_masks(detectors)
        wsum = float(sum(v[2] for v in variants))
        out = np.zeros((len(masks), probes.shape[0]), dtype=np.float64)
        nphi = len(self._phonons)
        for defocus, cs_v, weight in variants:
            psi0 = probe(p.ny, p.nx, p.dy, p.dx, p.lam, p.alpha_max, cs_v, defocus)
            sets: Dict[Tuple[int, int], CoefficientSet] = {}
            img = np.zeros_like(out)
            for phi in range(nphi):
                for k, pr in enumerate(probes):
                    q = (int(pr[0]), int(pr[1]))
                    key = class_key(q, p.in_spacing, p.in_offset, p.f)
                    idx, offs = nearest_translates(q, self.lattice, p.L, p.nx, p.ny)
                    if key not in sets:
                        sets[key] = (coefficients_closed(psi0, self.uW, offs, self.prm.degree, self.prm.lattice_m)
                                     if self.prm.coef_mode == 1 else coefficients(psi0, self.uW, offs))
                    U = [self.exit_wave(phi, int(i)) for i in idx]
                    psi = self._synthesize(U, sets[key].alpha, offs)
                    img[:, k] += [self._detect(psi, m) for m in masks]
            out += (weight / wsum) * img / nphi
        return out

    def image_rings(self, width: float, n_rings: int, probes: np.ndarray) -> np.ndarray:
        """3D STEM image (Sec. 3.1), shape (n_rings, n_probes): the 2D image with one ring
        per detector, averaged over configurations."""
        p = self.prm
        masks = ring_masks(p.D, p.dy, p.dx, p.lam, width, n_rings, p.bandlimit_frac)
        out = np.zeros((n_rings, probes.shape[0]), dtype=np.float64)
        nphi = len(self._phonons)
        for phi in range(nphi):
            for k, pr in enumerate(probes):
                out[:, k] += self.pixel(phi, (int(pr[0]), int(pr[1])), masks)
        return out / nphi

    def image_4d(self, A: int, B: int, probes: np.ndarray) -> np.ndarray:
        """4D STEM image (Sec. 3.1), shape (n_probes, 2B+1, 2A+1): the diffraction pattern of
        each synthesized exit wave on its D x D window, averaged over configurations."""
        out = np.zeros((probes.shape[0], 2 * B + 1, 2 * A + 1), dtype=np.float64)
        nphi = len(self._phonons)
        for phi in range(nphi):
            for k, pr in enumerate(probes):
                cs, idx = self.coefficient_set((int(pr[0]), int(pr[1])))
                U = [self.exit_wave(phi, int(i)) for i in idx]
                psi = self._synthesize(U, cs.alpha, cs.offsets)
                out[k] += self._pattern(psi, A, B)
        return out / nphi


def select_L(prm: LmaParams, probes: np.ndarray, eps_sup: float, L_max: int) -> Tuple[int, float]:
    """Smallest L (1..L_max) whose probe approximation error in the supremum norm, relative
    to the probe's maximum, is at most eps_sup for every probe class of `probes` (the
    parameter choice of Sec. 4.2.6: a target error fixes L), with the coefficients of
    ``prm.coef_mode``. Returns (L, worst error), or (0, error at L_max) when no L reaches
    the target."""
    lat = input_lattice(prm.nx, prm.ny, prm.in_spacing, prm.in_offset, prm.f)
    psi0 = probe(prm.ny, prm.nx, prm.dy, prm.dx, prm.lam, prm.alpha_max, prm.cs, prm.defocus)
    uW = input_wave_window(prm.kind, prm.W, prm.ny, prm.nx, prm.dy, prm.dx, prm.lam, prm.alpha_max,
                           prm.cs, prm.defocus, prm.gauss_sigma, prm.trig_degree)
    reps = {}
    for q in probes:
        key = class_key((int(q[0]), int(q[1])), prm.in_spacing, prm.in_offset, prm.f)
        reps.setdefault(key, (int(q[0]), int(q[1])))
    def fit(offs):
        if prm.coef_mode == 1:
            return coefficients_closed(psi0, uW, offs, prm.degree, prm.lattice_m)
        return coefficients(psi0, uW, offs)

    err = float("inf")
    for L in range(1, L_max + 1):
        err = max(fit(nearest_translates(q, lat, L, prm.nx, prm.ny)[1]).err_sup for q in reps.values())
        if err <= eps_sup:
            return L, err
    return 0, err


def region_probes(px0: int, py0: int, npx: int, npy: int, spacing: Tuple[int, int],
                  nx: int, ny: int) -> np.ndarray:
    """Probe lattice points of a region (row-major, x fastest), pixel (x, y) mod grid."""
    a = np.arange(npx)
    b = np.arange(npy)
    xs = np.mod(px0 + a * spacing[0], nx)
    ys = np.mod(py0 + b * spacing[1], ny)
    out = np.empty((npy * npx, 2), dtype=np.int64)
    out[:, 0] = np.tile(xs, npy)
    out[:, 1] = np.repeat(ys, npx)
    return out


def standard_image(prm: LmaParams, t_full: np.ndarray, detectors, probes: np.ndarray,
                   psi_init=None) -> np.ndarray:
    """Brute force (Fig. multislice_pseudocode per probe) on the full grid, D = X.

    ``psi_init`` (optional callable p -> full-grid wave) replaces the probe,
    e.g. by its LMA approximation.
    """
    p = prm
    prop = fresnel_propagator(p.ny, p.nx, p.dy, p.dx, p.lam, p.slice_dz, p.bandlimit_frac)
    masks = []
    for d in detectors:
        ang = p.lam * np.sqrt(k_squared(p.ny, p.nx, p.dy, p.dx))
        m = (ang >= d.r1) & (ang < d.r2) & bandlimit_mask(p.ny, p.nx, p.bandlimit_frac)
        masks.append(m)
    out = np.zeros((len(masks), probes.shape[0]))
    for k, pr in enumerate(probes):
        if psi_init is None:
            psi = probe(p.ny, p.nx, p.dy, p.dx, p.lam, p.alpha_max, p.cs, p.defocus,
                        p=(pr[1] * p.dy, pr[0] * p.dx))
        else:
            psi = psi_init((int(pr[0]), int(pr[1])))
        ex = multislice(psi, t_full, prop)
        for j, m in enumerate(masks):
            out[j, k] = float(np.sum(np.abs(dft2(ex)[m]) ** 2) / ex.size)
    return out


# ----------------------------------------------------------------------------
# local recompute (Sec. 4.2.6)
# ----------------------------------------------------------------------------

# ----------------------------------------------------------------------------
# memory-bounded partition of the probe region (Sec. 4.2.4)
# ----------------------------------------------------------------------------

def probe_translate_sets(prm: "LmaParams", probes: np.ndarray) -> List[frozenset]:
    """I_{f,p,L} of every probe (lattice indices), probes (n, 2) pixel (x, y)."""
    lat = input_lattice(prm.nx, prm.ny, prm.in_spacing, prm.in_offset, prm.f)
    return [frozenset(int(i) for i in nearest_translates((int(q[0]), int(q[1])), lat, prm.L, prm.nx, prm.ny)[0])
            for q in probes]


def multislice_ops(n_slices: int, X: int, Y: int, K: Tuple[int, int] | None = None) -> float:
    """Operation count of one multislice run on an X x Y domain (Sec. 3.2): N (2XY + 2XY log XY)
    with the propagation step in Fourier space, N (XY + XY K1 K2) with the K1 x K2 real-space
    kernel. log is base 2 (the 2048^2 crossover example of Sec. 4.2.1 holds only in that base)."""
    xy = float(X) * float(Y)
    if K is None:
        return n_slices * (2.0 * xy + 2.0 * xy * math.log2(xy))
    return n_slices * (xy + xy * K[0] * K[1])


def lma_ops(n_I: int, f: int, n_slices: int, X: int, Y: int, n_P: int, L: int, Xp: int, Yp: int,
            K: Tuple[int, int] | None = None) -> float:
    """T_LMA of Sec. 4.2.1, coefficient precomputation excluded: |I_f| = |I| / f^2 multislice
    runs plus |P| L X'Y' for the linear combinations. As the two formulas are printed, the
    Fourier variant runs multislice on the X x Y domain and the real-space variant (K given)
    on the X' x Y' domain."""
    runs = n_I / f ** 2
    per_run = multislice_ops(n_slices, X, Y) if K is None else multislice_ops(n_slices, Xp, Yp, K)
    return runs * per_run + float(n_P) * L * Xp * Yp


def realspace_crossover_f(X: int, Y: int, K1: int, K2: int) -> float:
    """The f from which real-space propagation on X/f x Y/f windows costs no more than Fourier
    propagation on the X x Y domain (Sec. 4.2.1): sqrt((1 + K1 K2) / (2 (1 + log XY)))."""
    return math.sqrt(0.5 * (1.0 + K1 * K2) / (1.0 + math.log2(float(X) * float(Y))))


def partition_cost(sets: Sequence[frozenset], parts: Sequence[Sequence[int]]) -> int:
    """T_{P_1..P_l} of Sec. 4.2.4: Multislice runs when the parts are computed in order and
    only the solutions shared by consecutive parts are kept."""
    unions = [frozenset().union(*[sets[q] for q in part]) for part in parts]
    return sum(len(u) for u in unions) - sum(len(unions[j] & unions[j + 1]) for j in range(len(unions) - 1))


def partition_rows(sets: Sequence[frozenset], npx: int, npy: int, M: int) -> List[List[int]]:
    """Row by row (Sec. 4.2.4, strategy 1): probes in raster order (a fastest); a probe
    joins the current part while the part's translates stay within M, else it starts the
    next part. Probe index = b * npx + a."""
    parts: List[List[int]] = []
    cur: List[int] = []
    union: set = set()
    for q in range(npx * npy):
        if cur and len(union | sets[q]) > M:
            parts.append(cur)
            cur, union = [], set()
        cur.append(q)
        union |= sets[q]
    if cur:
        parts.append(cur)
    return parts


def _tiles(npx: int, npy: int, w: int, h: int, column_major: bool) -> List[List[int]]:
    """The w x h tiling from (0, 0); tiles at the right and bottom edges are clipped."""
    xs = list(range(0, npx, w))
    ys = list(range(0, npy, h))
    order = [(x0, y0) for x0 in xs for y0 in ys] if column_major else [(x0, y0) for y0 in ys for x0 in xs]
    return [[b * npx + a for b in range(y0, min(y0 + h, npy)) for a in range(x0, min(x0 + w, npx))]
            for x0, y0 in order]


def partition_rectangles(sets: Sequence[frozenset], npx: int, npy: int, M: int,
                         column_major: bool = False, period: Tuple[int, int] = (1, 1)) -> List[List[int]]:
    """Rectangles (Sec. 4.2.4, strategy 2): tiles of one shape w x h from probe (0, 0),
    clipped at the right and bottom edges, in row-major (or column-major) order.

    The shape has the largest area w h such that a w x h tile anchored at every phase
    (ax, ay), 0 <= ax < period[0], 0 <= ay < period[1], needs at most M translates (the
    probe/lattice geometry repeats every `period` probes, so every full tile of the tiling
    is a translate of one of these; clipped tiles are subsets). For each width the height
    grows while all phase tiles fit; ties go to the squarer shape, then the wider one.
    """
    def fits(w: int, h: int) -> bool:
        for ay in range(period[1]):
            for ax in range(period[0]):
                u = set()
                for b in range(ay, min(ay + h, npy)):
                    for a in range(ax, min(ax + w, npx)):
                        u |= sets[b * npx + a]
                if len(u) > M:
                    return False
        return True

    best = None
    for w in range(1, npx + 1):
        if not fits(w, 1):
            break
        h = 1
        while h < npy and fits(w, h + 1):
            h += 1
        key = (w * h, -abs(w - h), w)
        if best is None or key > best[0]:
            best = (key, w, h)
    return _tiles(npx, npy, best[1], best[2], column_major)


def partition_greedy(sets: Sequence[frozenset], npx: int, npy: int, M: int, start: int = 0
                     ) -> List[List[int]]:
    """Greedy (Sec. 4.2.4, strategy 3): from the start probe, repeatedly add the unassigned
    neighbour (8-neighbourhood, inside the region) of the last added probe whose addition
    gives the fewest translates, ties by (b, a); the part closes when that neighbour would
    exceed M, and the next part starts with it. A probe with no unassigned neighbour
    continues with the first unassigned probe in raster order."""
    n = npx * npy
    assigned = [False] * n
    parts: List[List[int]] = []
    cur: List[int] = []
    union: set = set()
    nxt = start
    while True:
        q = nxt
        if cur and len(union | sets[q]) > M:
            parts.append(cur)
            cur, union = [], set()
        cur.append(q)
        union |= sets[q]
        assigned[q] = True
        if len(cur) + sum(len(p) for p in parts) == n:
            break
        a, b = q % npx, q // npx
        cand = []
        for bb in range(b - 1, b + 2):
            for aa in range(a - 1, a + 2):
                if 0 <= aa < npx and 0 <= bb < npy and not assigned[bb * npx + aa]:
                    r = bb * npx + aa
                    cand.append((len(union) + len(sets[r] - union), bb, aa, r))
        nxt = min(cand)[3] if cand else assigned.index(False)
    parts.append(cur)
    return parts


def edit_column(x: np.ndarray, y: np.ndarray, slc: np.ndarray, species: np.ndarray,
                lx: float, ly: float, cx: float, cy: float, r_site: float, op: int,
                new_species: int):
    """Change one atomic column: atoms whose lateral minimum-image distance to
    (cx, cy) is below r_site are removed (op 0) or given ``new_species`` (op 1)."""
    ddx = x - cx
    ddy = y - cy
    ddx = ddx - lx * np.round(ddx / lx)
    ddy = ddy - ly * np.round(ddy / ly)
    hit = ddx * ddx + ddy * ddy < r_site * r_site
    if op == 0:
        keep = ~hit
        return x[keep], y[keep], slc[keep], species[keep], int(hit.sum())
    if op == 1:
        sp = species.copy()
        sp[hit] = new_species
        return x.copy(), y.copy(), slc.copy(), sp, int(hit.sum())
    raise ValueError("unknown edit op")


def params_from_workload(w) -> LmaParams:
    """Flatten a ``workloads.Workload`` (duck-typed) into LmaParams."""
    g, b, pr = w.grid, w.basis, w.probe
    return LmaParams(nx=g.nx, ny=g.ny, lx=g.lx, ly=g.ly, slice_dz=g.slice_dz,
                     n_slices=g.n_slices, lam=g.lam, sigma=g.sigma,
                     bandlimit_frac=g.bandlimit_frac, alpha_max=pr.alpha_max, cs=pr.cs,
                     defocus=pr.defocus, kind=b.kind, gauss_sigma=b.gauss_sigma,
                     in_spacing=tuple(b.in_spacing_px), in_offset=tuple(b.in_offset_px),
                     f=b.f, L=b.L, W=b.window, D=b.det_window,
                     trig_degree=getattr(b, "trig_degree", 0), coef_mode=getattr(b, "coef_mode", 0))
