"""ctypes binding of the LMA C-ABI (include/lma.h).

Argument marshalling only: every step of the path runs in the CUDA library
``_build/liblma.so``, built in-tree by ``paper_2310_16829_gb300.build``. There
is no fallback: ``load()`` raises if the library is missing.

Array arguments may be numpy arrays (host memory) or torch CUDA tensors
(device memory, passed by ``data_ptr()``); streams are torch streams or raw
``cudaStream_t`` integers.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblma.so")

LMA_OK = 0
LMA_ERR_INVALID = 1
LMA_ERR_OOM = 2
LMA_ERR_CUDA = 3
LMA_ERR_TIMEOUT = 4
LMA_ERR_UNSUPPORTED = 5
STATUS_NAMES = {0: "LMA_OK", 1: "LMA_ERR_INVALID", 2: "LMA_ERR_OOM", 3: "LMA_ERR_CUDA",
                4: "LMA_ERR_TIMEOUT", 5: "LMA_ERR_UNSUPPORTED"}

LMA_BASIS_GAUSS = 0
LMA_BASIS_PROBE = 1
LMA_BASIS_TRIG = 2
LMA_BASIS_TRIG_RADIAL = 3
LMA_COEF_LSQ = 0
LMA_COEF_TRIG_CLOSED = 1
LMA_PREC_C64 = 0
LMA_PREC_FP16_STORE = 1
LMA_PREC_MIXED = 2
LMA_EDIT_REMOVE = 0
LMA_EDIT_SET_SPECIES = 1
LMA_IMAGE_RECOMPUTE = 1
LMA_MAX_RINGS = 256
LMA_MAX_VARIANTS = 32
LMA_IMAGE_GRAPH = 2
LMA_IMAGE_AUTOTUNE = 4
LMA_PART_ROWS = 0
LMA_PART_RECTANGLES = 1
LMA_PART_RECTANGLES_COLUMN_MAJOR = 2
LMA_PART_GREEDY = 3
LMA_SLICE_AUTO = -1
LMA_SLICE_ONE_PER_ITEM = 0
LMA_SLICE_PERSISTENT = 1
LMA_SLICE_DYNAMIC = 2
LMA_SYNTH_AUTO = -1
LMA_SYNTH_GATHER = 0
LMA_SYNTH_GROUPED = 1
SLICE_MODE_NAMES = {0: "one_per_item", 1: "persistent", 2: "dynamic"}

# every symbol include/lma.h declares (checked by the CPU tests)
EXPORTS = [
    "lma_create", "lma_destroy", "lma_last_error",
    "lma_create_specimen", "lma_free_specimen", "lma_specimen_set_atoms", "lma_transmission",
    "lma_create_basis", "lma_free_basis", "lma_basis_get_info", "lma_basis_coefficients",
    "lma_propagate_basis", "lma_exit_wave",
    "lma_image", "lma_image_rings", "lma_image_4d", "lma_image_many", "lma_edit_column",
    "lma_affected_probes",
    "lma_profile_enable", "lma_profile_read", "lma_readout_noalloc", "lma_realspace_gain",
    "lma_set_slice_mode", "lma_tuning_read", "lma_partition", "lma_image_partitioned",
    "lma_image_coherent", "lma_select_L", "lma_image_realspace", "lma_selftest_wait", "lma_synth_tuning_read",
    "lma_set_synth_mode", "lma_set_synth_buffer_limit",
]


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("lx", C.c_double), ("ly", C.c_double),
                ("slice_dz", C.c_double), ("n_slices", C.c_int32), ("lam", C.c_double),
                ("sigma", C.c_double), ("bandlimit_frac", C.c_double)]


class Potential(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("peak", C.POINTER(C.c_double)), ("n_terms", C.c_int32),
                ("term_frac", C.POINTER(C.c_double)), ("term_width", C.POINTER(C.c_double)),
                ("r_cut", C.c_double)]


class Atoms(C.Structure):
    _fields_ = [("n_atoms", C.c_int64), ("x", C.POINTER(C.c_double)), ("y", C.POINTER(C.c_double)),
                ("slice", C.POINTER(C.c_int32)), ("species", C.POINTER(C.c_int16))]


class Probe(C.Structure):
    _fields_ = [("alpha_max", C.c_double), ("cs", C.c_double), ("defocus", C.c_double)]


class BasisDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("gauss_sigma", C.c_double), ("in_spacing_px", C.c_int32 * 2),
                ("in_offset_px", C.c_int32 * 2), ("f", C.c_int32), ("L", C.c_int32),
                ("window", C.c_int32), ("det_window", C.c_int32), ("precision", C.c_int32),
                ("phonon_batch", C.c_int32), ("trig_degree", C.c_int32), ("coef_mode", C.c_int32)]


class Detector(C.Structure):
    _fields_ = [("r1", C.c_double), ("r2", C.c_double)]


class Region(C.Structure):
    _fields_ = [("px0", C.c_int32), ("py0", C.c_int32), ("npx", C.c_int32), ("npy", C.c_int32),
                ("spacing_px", C.c_int32 * 2)]


class PartitionDesc(C.Structure):
    _fields_ = [("strategy", C.c_int32), ("start", C.c_int32), ("max_resident", C.c_int64)]


class BasisInfo(C.Structure):
    _fields_ = [("n_translates", C.c_int64), ("nax", C.c_int32), ("nay", C.c_int32),
                ("n_sets", C.c_int32), ("L", C.c_int32), ("window", C.c_int32),
                ("det_window", C.c_int32), ("gauss_sigma", C.c_double),
                ("exit_wave_bytes", C.c_int64), ("phonon_batch", C.c_int32)]


class KernelStat(C.Structure):
    _fields_ = [("launches", C.c_int64), ("total_ms", C.c_double), ("units", C.c_int64)]


class Profile(C.Structure):
    _fields_ = [("potential", KernelStat), ("slice", KernelStat), ("synth", KernelStat),
                ("finalize", KernelStat), ("allocations", C.c_int64)]

    def as_dict(self):
        d = {k: {"launches": int(getattr(self, k).launches), "total_ms": float(getattr(self, k).total_ms),
                 "units": int(getattr(self, k).units)} for k, _ in self._fields_ if k != "allocations"}
        d["allocations"] = int(self.allocations)
        return d


class Tuning(C.Structure):
    _fields_ = [("n_jobs", C.c_int32), ("half", C.c_int32), ("even", C.c_int32), ("n_items", C.c_int64),
                ("translate_slices", C.c_int64), ("mode", C.c_int32), ("ms", C.c_double * 3)]

    def as_dict(self):
        return {"n_jobs": int(self.n_jobs), "half": bool(self.half), "even": bool(self.even),
                "n_items": int(self.n_items), "translate_slices": int(self.translate_slices),
                "mode": SLICE_MODE_NAMES.get(int(self.mode), int(self.mode)),
                "ms": {SLICE_MODE_NAMES[m]: float(self.ms[m]) for m in range(3)}}


class SynthTuning(C.Structure):
    _fields_ = [("readout", C.c_int32), ("half", C.c_int32), ("n_items", C.c_int64), ("L", C.c_int32),
                ("window", C.c_int32), ("strip", C.c_int32), ("persistent", C.c_int32), ("grouped", C.c_int32),
                ("group_x", C.c_int32), ("group_y", C.c_int32), ("group_shape", (C.c_int32 * 2) * 2),
                ("ms", C.c_double * 8)]

    def variant_name(self, v: int) -> str:
        if v < 6:
            return f"strip{16 << (v // 2)}_{'persistent' if v % 2 else 'per_probe'}"
        gx, gy = self.group_shape[v - 6][0], self.group_shape[v - 6][1]
        return f"grouped_{gx}x{gy}"

    def as_dict(self):
        return {"readout": ("annuli", "labels", "pattern")[int(self.readout)], "half": bool(self.half),
                "n_items": int(self.n_items), "L": int(self.L), "window": int(self.window),
                "strip": int(self.strip), "persistent": bool(self.persistent), "grouped": bool(self.grouped),
                "group": [int(self.group_x), int(self.group_y)] if self.grouped else None,
                "ms": {self.variant_name(v): float(self.ms[v]) for v in range(8) if self.ms[v] > 0}}


class LmaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_VP = C.c_void_p
_SIGS = {
    "lma_create": (C.c_int32, [C.c_int32, C.POINTER(_VP)]),
    "lma_destroy": (None, [_VP]),
    "lma_last_error": (C.c_char_p, [_VP]),
    "lma_create_specimen": (C.c_int32, [_VP, C.POINTER(Grid), C.POINTER(Potential), C.POINTER(Atoms),
                                        C.c_int32, C.POINTER(_VP)]),
    "lma_free_specimen": (C.c_int32, [_VP]),
    "lma_specimen_set_atoms": (C.c_int32, [_VP, _VP, C.POINTER(Atoms), C.c_int32]),
    "lma_profile_enable": (C.c_int32, [_VP, C.c_int32]),
    "lma_profile_read": (C.c_int32, [_VP, C.POINTER(Profile)]),
    "lma_transmission": (C.c_int32, [_VP, _VP, C.c_int32, _VP, _VP]),
    "lma_create_basis": (C.c_int32, [_VP, _VP, C.POINTER(Probe), C.POINTER(BasisDesc), C.POINTER(_VP)]),
    "lma_free_basis": (C.c_int32, [_VP]),
    "lma_basis_get_info": (C.c_int32, [_VP, C.POINTER(BasisInfo)]),
    "lma_basis_coefficients": (C.c_int32, [_VP, _VP, C.c_int32, C.c_int32, _VP, _VP, _VP, _VP]),
    "lma_propagate_basis": (C.c_int32, [_VP, _VP, _VP, C.c_int32, _VP]),
    "lma_exit_wave": (C.c_int32, [_VP, _VP, C.c_int64, _VP, _VP]),
    "lma_image": (C.c_int32, [_VP, _VP, _VP, C.POINTER(Detector), C.c_int32, C.POINTER(Region),
                              C.c_uint32, _VP, _VP]),
    "lma_image_rings": (C.c_int32, [_VP, _VP, _VP, C.c_double, C.c_int32, C.POINTER(Region), C.c_uint32,
                                    _VP, _VP]),
    "lma_image_4d": (C.c_int32, [_VP, _VP, _VP, C.c_int32, C.c_int32, C.POINTER(Region), C.c_uint32, _VP,
                                 _VP]),
    "lma_image_many": (C.c_int32, [_VP, C.c_int32, C.POINTER(_VP), C.POINTER(_VP), C.POINTER(Detector),
                                   C.c_int32, C.POINTER(Region), C.c_uint32, C.POINTER(_VP), _VP]),
    "lma_edit_column": (C.c_int32, [_VP, _VP, _VP, C.c_double, C.c_double, C.c_double, C.c_int32,
                                    C.c_int16, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "lma_affected_probes": (C.c_int32, [_VP, _VP, C.POINTER(Region), _VP, C.POINTER(C.c_int64)]),
    "lma_realspace_gain": (C.c_int32, [_VP, _VP, C.c_int32, C.c_int32, _VP, _VP]),
    "lma_selftest_wait": (C.c_int32, [_VP, C.c_int32, _VP]),
    "lma_readout_noalloc": (C.c_int32, [_VP, _VP, _VP, C.POINTER(Detector), C.c_int32, C.POINTER(Region),
                                        _VP, _VP]),
    "lma_set_slice_mode": (C.c_int32, [_VP, C.c_int32]),
    "lma_set_synth_mode": (C.c_int32, [_VP, C.c_int32]),
    "lma_set_synth_buffer_limit": (C.c_int32, [_VP, C.c_int64]),
    "lma_image_realspace": (C.c_int32, [_VP, _VP, _VP, C.c_int32, C.c_int32, C.POINTER(Detector), C.c_int32,
                                        C.POINTER(Region), C.c_uint32, _VP, _VP]),
    "lma_image_coherent": (C.c_int32, [_VP, _VP, _VP, C.POINTER(Probe), C.POINTER(C.c_double), C.c_int32,
                                       C.POINTER(Detector), C.c_int32, C.POINTER(Region), C.c_uint32, _VP, _VP]),
    "lma_select_L": (C.c_int32, [_VP, _VP, C.POINTER(Probe), C.POINTER(BasisDesc), C.POINTER(Region), C.c_int32,
                                 C.c_double, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "lma_partition": (C.c_int32, [_VP, _VP, C.POINTER(Region), C.POINTER(PartitionDesc), _VP,
                                  C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "lma_image_partitioned": (C.c_int32, [_VP, _VP, _VP, C.POINTER(Detector), C.c_int32, C.POINTER(Region),
                                          C.POINTER(PartitionDesc), C.c_uint32, _VP, _VP]),
    "lma_tuning_read": (C.c_int32, [_VP, C.POINTER(Tuning), C.c_int32, C.POINTER(C.c_int32)]),
    "lma_synth_tuning_read": (C.c_int32, [_VP, C.POINTER(SynthTuning), C.c_int32, C.POINTER(C.c_int32)]),
}

_LIB: Optional[C.CDLL] = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"LMA CUDA library not built: {path} is missing "
                           "(run __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return int(a.data_ptr())
    raise TypeError(f"unsupported buffer type {type(a)}")


def _stream(s) -> int:
    if s is None:
        return 0
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    return int(s)


class Context:
    """An lma_ctx; device = -1 gives a host-only context."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = _VP()
        st = self.lib.lma_create(device, C.byref(h))
        if st != LMA_OK:
            raise LmaError(st, f"lma_create({device}) failed")
        self.h = h
        self.device = device

    def check(self, st: int) -> None:
        if st != LMA_OK:
            raise LmaError(st, self.lib.lma_last_error(self.h).decode())

    def profile_enable(self, on: bool = True) -> None:
        self.check(self.lib.lma_profile_enable(self.h, 1 if on else 0))

    def profile_read(self) -> dict:
        p = Profile()
        self.check(self.lib.lma_profile_read(self.h, C.byref(p)))
        return p.as_dict()

    def selftest_wait(self, which: int, stream=None) -> int:
        """Run the slice kernels' bounded mbarrier wait on a phase that never completes (0: in
        one warp, 1: in the 16 warps of a CTA); returns the status code, LMA_ERR_TIMEOUT when
        the wait gave up as it should."""
        return self.lib.lma_selftest_wait(self.h, which, _stream(stream))

    def set_slice_mode(self, mode: int) -> None:
        self.check(self.lib.lma_set_slice_mode(self.h, mode))

    def set_synth_mode(self, mode: int) -> None:
        """LMA_SYNTH_AUTO, LMA_SYNTH_GATHER or LMA_SYNTH_GROUPED (same readings bit for bit)."""
        self.check(self.lib.lma_set_synth_mode(self.h, mode))

    def set_synth_buffer_limit(self, nbytes: int) -> None:
        """Largest probe-wave buffer of the grouped synthesis (0: the default, 2 GiB)."""
        self.check(self.lib.lma_set_synth_buffer_limit(self.h, nbytes))

    def tuning(self) -> list:
        n = C.c_int32()
        self.check(self.lib.lma_tuning_read(self.h, None, 0, C.byref(n)))
        recs = (Tuning * max(1, n.value))()
        self.check(self.lib.lma_tuning_read(self.h, recs, n.value, C.byref(n)))
        return [recs[i].as_dict() for i in range(n.value)]

    def synth_tuning(self) -> list:
        n = C.c_int32()
        self.check(self.lib.lma_synth_tuning_read(self.h, None, 0, C.byref(n)))
        recs = (SynthTuning * max(1, n.value))()
        self.check(self.lib.lma_synth_tuning_read(self.h, recs, n.value, C.byref(n)))
        return [recs[i].as_dict() for i in range(n.value)]

    def close(self) -> None:
        if self.h:
            self.lib.lma_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Specimen:
    """An lma_specimen built from a ``workloads.Workload`` (or its parts)."""

    def __init__(self, ctx: Context, grid, potential, phonons: Sequence):
        self.ctx = ctx
        self.grid = grid
        g = Grid(grid.nx, grid.ny, grid.lx, grid.ly, grid.slice_dz, grid.n_slices, grid.lam,
                 grid.sigma, grid.bandlimit_frac)
        self._keep: List = []
        peak = _f64(potential.peak)
        frac = _f64(potential.term_frac)
        width = _f64(potential.term_width)
        self._keep += [peak, frac, width]
        pot = Potential(len(peak), peak.ctypes.data_as(C.POINTER(C.c_double)), len(frac),
                        frac.ctypes.data_as(C.POINTER(C.c_double)),
                        width.ctypes.data_as(C.POINTER(C.c_double)), potential.r_cut)
        arr = self._atoms_array(phonons)
        h = _VP()
        ctx.check(ctx.lib.lma_create_specimen(ctx.h, C.byref(g), C.byref(pot), arr, len(phonons),
                                              C.byref(h)))
        self._keep = []   # the library copied everything
        self.h = h
        self.n_phonons = len(phonons)

    def _atoms_array(self, phonons):
        arr = (Atoms * len(phonons))()
        for k, at in enumerate(phonons):
            x, y = _f64(at.x), _f64(at.y)
            s = np.ascontiguousarray(at.slice, dtype=np.int32)
            sp = np.ascontiguousarray(at.species, dtype=np.int16)
            self._keep += [x, y, s, sp]
            arr[k] = Atoms(x.shape[0], x.ctypes.data_as(C.POINTER(C.c_double)),
                           y.ctypes.data_as(C.POINTER(C.c_double)),
                           s.ctypes.data_as(C.POINTER(C.c_int32)),
                           sp.ctypes.data_as(C.POINTER(C.c_int16)))
        return arr

    def set_atoms(self, phonons: Sequence) -> None:
        arr = self._atoms_array(phonons)
        try:
            self.ctx.check(self.ctx.lib.lma_specimen_set_atoms(self.ctx.h, self.h, arr, len(phonons)))
        finally:
            self._keep = []

    def transmission(self, phonon: int, out=None, stream=None) -> np.ndarray:
        g = self.grid
        if out is None:
            out = np.empty((g.n_slices, g.ny, g.nx), dtype=np.complex64)
        self.ctx.check(self.ctx.lib.lma_transmission(self.ctx.h, self.h, phonon, _ptr(out),
                                                     _stream(stream)))
        return out

    def edit_column(self, basis: Optional["Basis"], cx: float, cy: float, r_site: float, op: int,
                    new_species: int = 0):
        n_changed = C.c_int64()
        n_stale = C.c_int64()
        self.ctx.check(self.ctx.lib.lma_edit_column(self.ctx.h, self.h, basis.h if basis else None,
                                                    cx, cy, r_site, op, new_species,
                                                    C.byref(n_changed), C.byref(n_stale)))
        return int(n_changed.value), int(n_stale.value)

    def close(self):
        if self.h:
            self.ctx.lib.lma_free_specimen(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _region(r) -> Region:
    return Region(r.px0, r.py0, r.npx, r.npy, (C.c_int32 * 2)(*r.spacing_px))


class Basis:
    """An lma_basis (input-wave lattice, coefficients, resident exit waves)."""

    def __init__(self, ctx: Context, spec: Specimen, probe, desc):
        self.ctx = ctx
        self.spec = spec
        pr = Probe(probe.alpha_max, probe.cs, probe.defocus)
        d = BasisDesc(desc.kind, desc.gauss_sigma, (C.c_int32 * 2)(*desc.in_spacing_px),
                      (C.c_int32 * 2)(*desc.in_offset_px), desc.f, desc.L, desc.window,
                      desc.det_window, getattr(desc, "precision", LMA_PREC_C64),
                      getattr(desc, "phonon_batch", 0), getattr(desc, "trig_degree", 0),
                      getattr(desc, "coef_mode", LMA_COEF_LSQ))
        h = _VP()
        ctx.check(ctx.lib.lma_create_basis(ctx.h, spec.h, C.byref(pr), C.byref(d), C.byref(h)))
        self.h = h
        self.L = desc.L
        self.W = desc.window
        self.alpha_max = probe.alpha_max

    def info(self) -> BasisInfo:
        i = BasisInfo()
        self.ctx.check(self.ctx.lib.lma_basis_get_info(self.h, C.byref(i)))
        return i

    def coefficients(self, px: int, py: int):
        L = self.L
        al = np.empty(2 * L, dtype=np.float64)
        off = np.empty(2 * L, dtype=np.int32)
        tr = np.empty(L, dtype=np.int64)
        err = np.empty(2, dtype=np.float64)
        self.ctx.check(self.ctx.lib.lma_basis_coefficients(self.ctx.h, self.h, px, py, _ptr(al),
                                                           _ptr(off), _ptr(tr), _ptr(err)))
        return al[0::2] + 1j * al[1::2], off.reshape(L, 2), tr, err

    def propagate(self, phonon: int, stream=None) -> None:
        self.ctx.check(self.ctx.lib.lma_propagate_basis(self.ctx.h, self.spec.h, self.h, phonon,
                                                        _stream(stream)))

    def exit_wave(self, translate: int, out=None, stream=None) -> np.ndarray:
        if out is None:
            out = np.empty((self.W, self.W), dtype=np.complex64)
        self.ctx.check(self.ctx.lib.lma_exit_wave(self.ctx.h, self.h, translate, _ptr(out),
                                                  _stream(stream)))
        return out

    def image(self, detectors, region, out=None, recompute: bool = False, stream=None,
              autotune: bool = False):
        dets = (Detector * len(detectors))(*[Detector(d.r1, d.r2) for d in detectors])
        if out is None:
            out = np.empty((len(detectors), region.npy, region.npx), dtype=np.float64)
        reg = _region(region)
        flags = (LMA_IMAGE_RECOMPUTE if recompute else 0) | (LMA_IMAGE_AUTOTUNE if autotune else 0)
        self.ctx.check(self.ctx.lib.lma_image(self.ctx.h, self.spec.h, self.h, dets, len(detectors),
                                              C.byref(reg), flags, _ptr(out), _stream(stream)))
        return out

    def image_rings(self, ring_width: float, n_rings: int, region, out=None, recompute: bool = False,
                    stream=None):
        """3D STEM image [n_rings][npy][npx]: ring a covers [a w, (a + 1) w) rad."""
        if out is None:
            out = np.empty((n_rings, region.npy, region.npx), dtype=np.float64)
        reg = _region(region)
        flags = LMA_IMAGE_RECOMPUTE if recompute else 0
        self.ctx.check(self.ctx.lib.lma_image_rings(self.ctx.h, self.spec.h, self.h, ring_width, n_rings,
                                                    C.byref(reg), flags, _ptr(out), _stream(stream)))
        return out

    def image_4d(self, half_x: int, half_y: int, region, out=None, recompute: bool = False, stream=None):
        """4D STEM image [npy][npx][2 half_y + 1][2 half_x + 1] (float32)."""
        if out is None:
            out = np.empty((region.npy, region.npx, 2 * half_y + 1, 2 * half_x + 1), dtype=np.float32)
        reg = _region(region)
        flags = LMA_IMAGE_RECOMPUTE if recompute else 0
        self.ctx.check(self.ctx.lib.lma_image_4d(self.ctx.h, self.spec.h, self.h, half_x, half_y,
                                                 C.byref(reg), flags, _ptr(out), _stream(stream)))
        return out

    def image_realspace(self, K1: int, K2: int, detectors, region, out=None, stream=None):
        """Image with the propagation step as a K1 x K2 real-space convolution."""
        dets = (Detector * len(detectors))(*[Detector(d.r1, d.r2) for d in detectors])
        if out is None:
            out = np.empty((len(detectors), region.npy, region.npx), dtype=np.float64)
        reg = _region(region)
        self.ctx.check(self.ctx.lib.lma_image_realspace(self.ctx.h, self.spec.h, self.h, K1, K2, dets,
                                                        len(detectors), C.byref(reg), 0, _ptr(out),
                                                        _stream(stream)))
        return out

    def realspace_gain(self, K1: int, K2: int):
        """(max_k |Q(k)|, max over the bandlimit) of the K1 x K2 real-space kernel (host)."""
        ga, gb = C.c_double(), C.c_double()
        self.ctx.check(self.ctx.lib.lma_realspace_gain(self.ctx.h, self.h, K1, K2, C.byref(ga), C.byref(gb)))
        return ga.value, gb.value

    def image_coherent(self, variants, detectors, region, out=None, recompute: bool = False, stream=None):
        """Partially coherent image: variants = [(defocus, cs, weight), ...] of the basis probe
        (same aperture), averaged with the normalised weights from one set of exit waves."""
        n = len(variants)
        probes = (Probe * n)(*[Probe(self.alpha_max, cs, dz) for dz, cs, _ in variants])
        wts = (C.c_double * n)(*[w for _, _, w in variants])
        dets = (Detector * len(detectors))(*[Detector(d.r1, d.r2) for d in detectors])
        if out is None:
            out = np.empty((len(detectors), region.npy, region.npx), dtype=np.float64)
        reg = _region(region)
        flags = LMA_IMAGE_RECOMPUTE if recompute else 0
        self.ctx.check(self.ctx.lib.lma_image_coherent(self.ctx.h, self.spec.h, self.h, probes, wts, n, dets,
                                                       len(detectors), C.byref(reg), flags, _ptr(out),
                                                       _stream(stream)))
        return out

    def partition(self, region, strategy: int, max_resident: int, start: int = 0):
        """Partition of a probe region under a memory bound (Sec. 4.2.4): (part index per
        probe [npy][npx], number of parts, Multislice runs T, peak resident waves)."""
        part = np.empty((region.npy, region.npx), dtype=np.int32)
        n = C.c_int32()
        runs = C.c_int64()
        peak = C.c_int64()
        reg = _region(region)
        d = PartitionDesc(strategy, start, max_resident)
        self.ctx.check(self.ctx.lib.lma_partition(self.ctx.h, self.h, C.byref(reg), C.byref(d), _ptr(part),
                                                  C.byref(n), C.byref(runs), C.byref(peak)))
        return part, int(n.value), int(runs.value), int(peak.value)

    def image_partitioned(self, detectors, region, strategy: int, max_resident: int, start: int = 0,
                          out=None, stream=None):
        """2D image with an exit-wave store of max_resident waves per configuration."""
        dets = (Detector * len(detectors))(*[Detector(d.r1, d.r2) for d in detectors])
        if out is None:
            out = np.empty((len(detectors), region.npy, region.npx), dtype=np.float64)
        reg = _region(region)
        d = PartitionDesc(strategy, start, max_resident)
        self.ctx.check(self.ctx.lib.lma_image_partitioned(self.ctx.h, self.spec.h, self.h, dets, len(detectors),
                                                          C.byref(reg), C.byref(d), 0, _ptr(out),
                                                          _stream(stream)))
        return out

    def readout_noalloc(self, exit_waves, detectors, region, out, stream=None):
        """Readings of one configuration from caller-held exit waves, without device allocation.

        ``exit_waves`` and ``out`` are device buffers owned by the caller (e.g. torch CUDA
        tensors); the library uses a fixed scratch array instead of allocating.
        """
        dets = (Detector * len(detectors))(*[Detector(d.r1, d.r2) for d in detectors])
        reg = _region(region)
        self.ctx.check(self.ctx.lib.lma_readout_noalloc(self.ctx.h, self.h, _ptr(exit_waves), dets,
                                                        len(detectors), C.byref(reg), _ptr(out),
                                                        _stream(stream)))
        return out

    def affected_probes(self, region) -> np.ndarray:
        mask = np.empty((region.npy, region.npx), dtype=np.uint8)
        n = C.c_int64()
        reg = _region(region)
        self.ctx.check(self.ctx.lib.lma_affected_probes(self.ctx.h, self.h, C.byref(reg), _ptr(mask),
                                                        C.byref(n)))
        return mask

    def close(self):
        if self.h:
            self.ctx.lib.lma_free_basis(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def select_L(ctx: Context, spec: "Specimen", probe, desc, region, L_max: int, eps_sup: float):
    """Smallest L <= L_max whose probe approximation error (supremum norm, relative) meets
    eps_sup over the region's coefficient classes: (L or 0, error)."""
    pr = Probe(probe.alpha_max, probe.cs, probe.defocus)
    d = BasisDesc(desc.kind, desc.gauss_sigma, (C.c_int32 * 2)(*desc.in_spacing_px),
                  (C.c_int32 * 2)(*desc.in_offset_px), desc.f, desc.L, desc.window,
                  desc.det_window, getattr(desc, "precision", LMA_PREC_C64), getattr(desc, "phonon_batch", 0),
                  getattr(desc, "trig_degree", 0), getattr(desc, "coef_mode", LMA_COEF_LSQ))
    reg = _region(region)
    L = C.c_int32()
    err = C.c_double()
    ctx.check(ctx.lib.lma_select_L(ctx.h, spec.h, C.byref(pr), C.byref(d), C.byref(reg), L_max, eps_sup,
                                   C.byref(L), C.byref(err)))
    return int(L.value), float(err.value)


def image_many(ctx: Context, bases, detectors, regions, outs, recompute: bool = True,
               graph: bool = False, stream=None, autotune: bool = False):
    """lma_image_many over several (specimen, basis) pairs; ``outs`` are per-basis buffers
    [n_det][npy][npx] float64 (device tensors when ``graph``)."""
    n = len(bases)
    specs = (_VP * n)(*[b.spec.h.value for b in bases])
    hs = (_VP * n)(*[b.h.value for b in bases])
    dets = (Detector * len(detectors))(*[Detector(d.r1, d.r2) for d in detectors])
    regs = (Region * n)(*[_region(r) for r in regions])
    ptrs = (_VP * n)(*[_ptr(o) for o in outs])
    flags = ((LMA_IMAGE_RECOMPUTE if recompute else 0) | (LMA_IMAGE_GRAPH if graph else 0) |
             (LMA_IMAGE_AUTOTUNE if autotune else 0))
    ctx.check(ctx.lib.lma_image_many(ctx.h, n, specs, hs, dets, len(detectors), regs, flags, ptrs,
                                     _stream(stream)))
    return outs
