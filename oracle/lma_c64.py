"""Complex64 restatement of the oracle's LMA pipeline: the rounding floor of single precision.

TEST INFRASTRUCTURE ONLY, under the same rule as ``lma_oracle``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import it. It is not a
reference for values; ``lma_oracle`` (FP64) is.

Why it exists. The GPU path computes in complex64. A detector reading that carries a small
part of the beam (the HAADF annulus of a thin crystal holds 1e-7..1e-4 of it) cannot be
computed to 1e-4 relative error in that precision: the rounding of every 2D DFT is a white
noise spread over the whole spectrum, and the part of it that lands on the annulus is an
absolute error of the reading. To tell that floor from a kernel error, the tests run the
oracle's steps once more with every array held in complex64 -- input wave, transmission,
propagator, coefficients, exit waves, synthesized wave, spectrum -- and every DFT in single
precision, then measure this restatement's error against the FP64 oracle on the same inputs.
That is the error complex64 arithmetic alone makes, whatever the order of its operations.

The steps, their order and their inputs are the oracle's (Fig. multislice_pseudocode,
Fig. lma_pseudocode, Sec. 3.1); only the precision differs:
  * the transmission is the oracle's t = exp(i sigma v) rounded once to complex64;
  * the least-squares coefficients are the oracle's, rounded once to complex64;
  * DFTs are ``scipy.fft`` in single precision (it keeps complex64 in and out);
  * a detector reading sums |DFT|^2 in float32 (pairwise), divided by n^2 in float32.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np
import scipy.fft as _sf

from . import lma_oracle as O

C64 = np.complex64
F32 = np.float32


def dft2(a: np.ndarray) -> np.ndarray:
    """Unnormalised forward 2D DFT in single precision (complex64 in and out)."""
    out = _sf.fft2(np.asarray(a, dtype=C64))
    assert out.dtype == C64
    return out


def idft2(a: np.ndarray) -> np.ndarray:
    """Inverse 2D DFT with the 1/n^2 factor, in single precision."""
    out = _sf.ifft2(np.asarray(a, dtype=C64))
    assert out.dtype == C64
    return out


def multislice(psi: np.ndarray, t: Sequence[np.ndarray], prop: np.ndarray) -> np.ndarray:
    """``lma_oracle.multislice`` in complex64: for each slice, transmit then propagate."""
    psi = np.asarray(psi, dtype=C64)
    prop = np.asarray(prop, dtype=C64)
    for ts in t:
        psi = psi * np.asarray(ts, dtype=C64)
        psi = idft2(prop * dft2(psi))
    return psi


def convolve_periodic(psi: np.ndarray, qK: np.ndarray) -> np.ndarray:
    """``lma_oracle.convolve_periodic`` in complex64."""
    K2, K1 = qK.shape
    qK = np.asarray(qK, dtype=C64)
    out = np.zeros(psi.shape, dtype=C64)
    for iy, dy in enumerate(O.kernel_offsets(K2)):
        for ix, dx in enumerate(O.kernel_offsets(K1)):
            out += qK[iy, ix] * np.roll(psi, (int(dy), int(dx)), axis=(0, 1))
    return out


def multislice_realspace(psi: np.ndarray, t: Sequence[np.ndarray], qK: np.ndarray) -> np.ndarray:
    """``lma_oracle.multislice_realspace`` in complex64."""
    psi = np.asarray(psi, dtype=C64)
    for ts in t:
        psi = convolve_periodic(np.asarray(ts, dtype=C64) * psi, qK)
    return psi


def translate_exit_wave(uW: np.ndarray, t_full: np.ndarray, prop_W: np.ndarray,
                        pos: Tuple[int, int]) -> np.ndarray:
    """``lma_oracle.translate_exit_wave`` in complex64 (window [i - W/2, i + W/2))."""
    W = uW.shape[0]
    ts = O.periodic_crop(t_full, pos[1] - W // 2, pos[0] - W // 2, W, W)
    return multislice(uW, ts, prop_W)


def synthesize(U: Sequence[np.ndarray], alpha: np.ndarray, offsets: np.ndarray, D: int,
               cyclic: bool) -> np.ndarray:
    """``lma_oracle.synthesize`` in complex64, with the coefficients rounded once."""
    psi = np.zeros((D, D), dtype=C64)
    for Uj, a, o in zip(U, np.asarray(alpha, dtype=C64), offsets):
        W = Uj.shape[0]
        sx = int(o[0]) + (D - W) // 2
        sy = int(o[1]) + (D - W) // 2
        if cyclic:
            psi += a * np.roll(np.asarray(Uj, dtype=C64), shift=(sy, sx), axis=(0, 1))
            continue
        y0, y1 = max(0, sy), min(D, sy + W)
        x0, x1 = max(0, sx), min(D, sx + W)
        if y0 < y1 and x0 < x1:
            psi[y0:y1, x0:x1] += a * np.asarray(Uj, dtype=C64)[y0 - sy:y1 - sy, x0 - sx:x1 - sx]
    return psi


def intensity(psi: np.ndarray) -> np.ndarray:
    """|DFT(psi)|^2 in float32."""
    spec = dft2(psi)
    return spec.real * spec.real + spec.imag * spec.imag


def detect(psi: np.ndarray, mask: np.ndarray) -> float:
    """``lma_oracle.detect`` in single precision: (1/n^2) sum over the detector of |DFT|^2."""
    e = intensity(psi)
    return float(np.sum(e[mask], dtype=F32) / F32(psi.size))


def pattern(psi: np.ndarray, A: int, B: int, frac: float | None) -> np.ndarray:
    """``lma_oracle.pattern`` in single precision."""
    ny, nx = psi.shape
    spec = intensity(psi) / F32(psi.size)
    if frac is not None:
        spec = np.where(O.bandlimit_mask(ny, nx, frac), spec, F32(0.0))
    out = np.zeros((2 * B + 1, 2 * A + 1), dtype=np.float64)
    for b in range(-B, B + 1):
        for a in range(-A, A + 1):
            out[b + B, a + A] = spec[b % ny, a % nx]
    return out


class LmaOracleC64(O.LmaOracle):
    """``LmaOracle`` with every step of the image pipeline in complex64.

    Geometry (lattice, nearest translates, coefficient classes) and the FP64 inputs
    (probe, input wave, transmission, least-squares coefficients) are the oracle's; each
    is rounded once to complex64 where the pipeline first uses it.
    """

    def __init__(self, prm: O.LmaParams, realspace: Tuple[int, int] | None = None):
        super().__init__(prm, realspace)
        self._t32: Dict[int, np.ndarray] = {}

    def transmission_stack_c64(self, phi: int) -> np.ndarray:
        if phi not in self._t32:
            self._t32[phi] = self.transmission_stack(phi).astype(C64)
        return self._t32[phi]

    def set_specimen(self, phonons: Sequence, peak, term_frac, term_width, r_cut):
        super().set_specimen(phonons, peak, term_frac, term_width, r_cut)
        self._t32 = {}

    def exit_wave(self, phi: int, i: int) -> np.ndarray:
        if (phi, i) not in self._U:
            pos = (int(self.lattice[i, 0]), int(self.lattice[i, 1]))
            t = self.transmission_stack_c64(phi)
            if self.qK is None:
                self._U[(phi, i)] = translate_exit_wave(self.uW, t, self.prop_W, pos)
            else:
                W = self.prm.W
                ts = O.periodic_crop(t, pos[1] - W // 2, pos[0] - W // 2, W, W)
                self._U[(phi, i)] = multislice_realspace(self.uW, ts, self.qK)
        return self._U[(phi, i)]

    def _synthesize(self, U, alpha, offsets) -> np.ndarray:
        return synthesize(U, alpha, offsets, self.prm.D, self.prm.cyclic)

    def _detect(self, psi: np.ndarray, mask: np.ndarray) -> float:
        return detect(psi, mask)

    def _pattern(self, psi: np.ndarray, A: int, B: int) -> np.ndarray:
        return pattern(psi, A, B, self.prm.bandlimit_frac)


def floor_scale(ref: np.ndarray, emu: np.ndarray) -> np.ndarray:
    """kappa per detector row: the envelope of |emu - ref| / sqrt(ref) over the row's readings.

    A reading I = (1/n^2) sum_det |Psi|^2 perturbed by a white rounding noise dPsi changes by
    2 Re sum Psi* dPsi + sum |dPsi|^2, whose first term grows as sqrt(I) times the noise on
    the detector; kappa sqrt(I) is therefore the envelope of the complex64 error of a row.
    kappa is the largest normalised error of the row, but at least three times its root mean
    square, so that a row of few readings (whose largest error is a poor estimate of the
    envelope) does not understate it.
    """
    ref = np.atleast_2d(np.asarray(ref, dtype=np.float64))
    ref = ref.reshape(ref.shape[0], -1)
    emu = np.asarray(emu, dtype=np.float64).reshape(ref.shape)
    pos = ref > 0
    q = np.where(pos, np.abs(emu - ref) / np.sqrt(np.where(pos, ref, 1.0)), 0.0)
    n = np.maximum(pos.sum(axis=1), 1)
    rms = np.sqrt(np.sum(q * q, axis=1) / n)
    return np.maximum(np.max(q, axis=1), 3.0 * rms)


def floor_bound(ref: np.ndarray, emu: np.ndarray, tol: float, margin: float = 3.0) -> np.ndarray:
    """Per reading: max(tol * ref, margin * kappa_row * sqrt(ref)), the larger of the relative
    bound and ``margin`` times the complex64 envelope of its detector row."""
    ref2 = np.atleast_2d(np.asarray(ref, dtype=np.float64))
    ref2 = ref2.reshape(ref2.shape[0], -1)
    kap = floor_scale(ref2, emu)
    return np.maximum(tol * ref2, margin * kap[:, None] * np.sqrt(np.maximum(ref2, 0.0)))
