"""The oracle's image readings evaluated over the host's cores.

TEST AND BASELINE INFRASTRUCTURE ONLY, under the same rule as ``lma_oracle``: only
``tests/`` and the CPU legs of ``bench.py`` may import it.

The exit waves of different (configuration, translate) pairs are independent (Fig.
lma_pseudocode, step 1), and so are the readings of different probes (step 2). ``readings``
hands them to worker processes started with 'spawn' (no worker inherits a CUDA context),
which call the oracle's own functions, unchanged: ``projected_potential`` and
``transmission`` per configuration, ``translate_exit_wave`` per translate, ``synthesize``
and ``detect`` per probe. Transmission stacks and exit waves pass between the processes
through memory-mapped files; the phonon average is summed in configuration order in the
parent. Each reading is therefore the same value, bit for bit, as ``LmaOracle.image`` gives.
With ``c64`` the workers also run the complex64 restatement (``lma_c64``) on the same inputs.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import shutil
import tempfile
import time
from concurrent.futures import ProcessPoolExecutor
from typing import Dict, List, Sequence

import numpy as np

from . import lma_c64 as C
from . import lma_oracle as O

_G: Dict = {}


def _init(state: Dict) -> None:
    _G.clear()
    _G.update(state)
    _G["maps"] = {}


def _map(name: str, dtype, shape, mode: str = "r+") -> np.ndarray:
    key = (name, mode)
    if key not in _G["maps"]:
        _G["maps"][key] = np.memmap(os.path.join(_G["dir"], name), dtype=dtype, mode=mode, shape=shape)
    return _G["maps"][key]


def _t_task(jp: int) -> float:
    """Transmission stack of configuration number jp of the call (step a1)."""
    t0 = time.perf_counter()
    prm = _G["prm"]
    x, y, s, sp = _G["atoms"][jp]
    peak, tf, tw, rc = _G["pot"]
    v = O.projected_potential(x, y, s, sp, prm.n_slices, prm.ny, prm.nx, prm.ly, prm.lx, peak, tf, tw, rc)
    t = _map(f"t{jp}", np.complex128, (prm.n_slices, prm.ny, prm.nx), "w+")
    t[:] = O.transmission(v, prm.sigma)
    t.flush()
    return time.perf_counter() - t0


def _u_task(job) -> float:
    """Exit wave of one translate for one configuration (step a3), FP64 and optionally complex64."""
    t0 = time.perf_counter()
    jp, i, slot = job
    prm = _G["prm"]
    W = prm.W
    t = _map(f"t{jp}", np.complex128, (prm.n_slices, prm.ny, prm.nx), "r")
    pos = (int(_G["lattice"][i, 0]), int(_G["lattice"][i, 1]))
    n = _G["n_slots"]
    u = _map("u64", np.complex128, (_G["n_phis"], n, W, W))
    u[jp, slot] = O.translate_exit_wave(_G["uW"], t, _G["prop_W"], pos)
    if _G["c64"]:
        u32 = _map("u32", np.complex64, (_G["n_phis"], n, W, W))
        u32[jp, slot] = C.translate_exit_wave(_G["uW"], t, _G["prop_W"], pos)
    return time.perf_counter() - t0


def _p_task(job):
    """Readings of one probe for one configuration (steps a4, a5)."""
    t0 = time.perf_counter()
    jp, k = job
    prm = _G["prm"]
    W = prm.W
    n = _G["n_slots"]
    alpha, offsets, slots = _G["tables"][k]
    u = _map("u64", np.complex128, (_G["n_phis"], n, W, W))
    psi = O.synthesize([u[jp, s] for s in slots], alpha, offsets, prm.D, prm.cyclic)
    r64 = [O.detect(psi, m) for m in _G["masks"]]
    r32 = None
    if _G["c64"]:
        u32 = _map("u32", np.complex64, (_G["n_phis"], n, W, W))
        psi32 = C.synthesize([u32[jp, s] for s in slots], alpha, offsets, prm.D, prm.cyclic)
        r32 = [C.detect(psi32, m) for m in _G["masks"]]
    return jp, k, r64, r32, time.perf_counter() - t0


def default_workers() -> int:
    return max(1, min(os.cpu_count() or 1, 64))


def readings(w, detectors, probes: np.ndarray, phis: Sequence[int] | None = None, c64: bool = False,
             workers: int | None = None, tmpdir: str | None = None) -> Dict:
    """Phonon-averaged oracle readings of ``probes`` ((n, 2) pixel (x, y)) over the
    configurations ``phis`` of workload ``w`` (all by default), computed by ``workers``
    processes.

    Returns {"ref": (n_det, n) FP64 readings, "emu": the complex64 restatement's readings
    (with ``c64``) or None, "translates": exit waves per configuration, "workers",
    "seconds": wall time per phase ("transmission", "exit_waves", "probes", "coefficients"),
    "cpu_seconds": summed worker time per phase}.
    """
    prm = O.params_from_workload(w)
    phis = list(range(len(w.phonons))) if phis is None else [int(p) for p in phis]
    workers = default_workers() if workers is None else max(1, int(workers))
    probes = np.asarray(probes, dtype=np.int64).reshape(-1, 2)
    secs, cpu = {}, {}

    t0 = time.perf_counter()
    orc = O.LmaOracle(prm)
    orc.set_specimen(w.phonons, w.potential.peak, w.potential.term_frac, w.potential.term_width,
                     w.potential.r_cut)
    sets = [orc.coefficient_set((int(p[0]), int(p[1]))) for p in probes]
    needed = sorted({int(i) for _, idx in sets for i in idx})
    slot_of = {i: s for s, i in enumerate(needed)}
    tables = [(cs.alpha, cs.offsets, [slot_of[int(i)] for i in idx]) for cs, idx in sets]
    masks = orc.detector_masks(detectors)
    secs["coefficients"] = time.perf_counter() - t0

    own_dir = tmpdir is None
    d = tempfile.mkdtemp(prefix="lma_oracle_") if own_dir else tmpdir
    state = {"prm": prm, "uW": orc.uW, "prop_W": orc.prop_W, "lattice": orc.lattice, "masks": masks,
             "tables": tables, "dir": d, "n_slots": len(needed), "n_phis": len(phis), "c64": bool(c64),
             "atoms": [(w.phonons[p].x, w.phonons[p].y, w.phonons[p].slice, w.phonons[p].species) for p in phis],
             "pot": (tuple(w.potential.peak), tuple(w.potential.term_frac), tuple(w.potential.term_width),
                     float(w.potential.r_cut))}
    ref = np.zeros((len(masks), probes.shape[0]), dtype=np.float64)
    emu = np.zeros_like(ref) if c64 else None
    try:
        W = prm.W
        # the exit-wave files are created here, so that every worker maps them whole
        np.memmap(os.path.join(d, "u64"), dtype=np.complex128, mode="w+",
                  shape=(len(phis), len(needed), W, W)).flush()
        if c64:
            np.memmap(os.path.join(d, "u32"), dtype=np.complex64, mode="w+",
                      shape=(len(phis), len(needed), W, W)).flush()
        ctx = mp.get_context("spawn")
        with ProcessPoolExecutor(max_workers=workers, mp_context=ctx, initializer=_init,
                                 initargs=(state,)) as ex:
            t0 = time.perf_counter()
            cpu["transmission"] = sum(ex.map(_t_task, range(len(phis))))
            secs["transmission"] = time.perf_counter() - t0
            jobs = [(jp, i, slot_of[i]) for jp in range(len(phis)) for i in needed]
            t0 = time.perf_counter()
            ch = max(1, len(jobs) // (8 * workers))
            cpu["exit_waves"] = sum(ex.map(_u_task, jobs, chunksize=ch))
            secs["exit_waves"] = time.perf_counter() - t0
            pjobs = [(jp, k) for jp in range(len(phis)) for k in range(probes.shape[0])]
            t0 = time.perf_counter()
            ch = max(1, len(pjobs) // (8 * workers))
            res = {}
            cpu["probes"] = 0.0
            for jp, k, r64, r32, dt in ex.map(_p_task, pjobs, chunksize=ch):
                res[(jp, k)] = (r64, r32)
                cpu["probes"] += dt
            secs["probes"] = time.perf_counter() - t0
        # phonon average, summed in configuration order (as LmaOracle.image)
        for jp in range(len(phis)):
            for k in range(probes.shape[0]):
                r64, r32 = res[(jp, k)]
                ref[:, k] += r64
                if c64:
                    emu[:, k] += r32
        ref /= len(phis)
        if c64:
            emu /= len(phis)
    finally:
        if own_dir:
            shutil.rmtree(d, ignore_errors=True)
    return {"ref": ref, "emu": emu, "translates": len(needed), "workers": workers,
            "seconds": secs, "cpu_seconds": cpu}


def subregion_probes(region, a0: int, b0: int, n: int, nx: int, ny: int) -> np.ndarray:
    """Pixel positions of the n x n probes of ``region`` starting at probe (a0, b0), row-major."""
    return O.region_probes(region.px0 + a0 * region.spacing_px[0], region.py0 + b0 * region.spacing_px[1],
                           n, n, region.spacing_px, nx, ny)


def cpu_model() -> str:
    """The host CPU's model name, as lscpu (or /proc/cpuinfo) reports it."""
    try:
        import subprocess
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"
