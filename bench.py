#!/usr/bin/env python
"""Benchmark of the LMA hot path on GB300: HAADF pixels/s of the full image pipeline.

One step = one pass of the whole path over the ABO3 workload (512^2 grid,
50 slices of 2 A, 8 frozen-phonon configurations, 128 x 128 probes, Gaussian
input waves on a 4-px lattice, L = 32, W = D = 128, complex64): for every
configuration the transmission is built (step a1), all 16384 translates are
propagated (a3), every probe is synthesized and read out (a4, a5), and the
readings are averaged in FP64 (a6). ``value`` is measured with the atoms
already resident in HBM and the image written to device memory; ``e2e`` runs
the same step through the public API with host buffers (new atom lists
uploaded, image copied back) inside the timed region.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm).
"""
from __future__ import annotations

import os

# Concurrent streams (the serving lanes) each need their own hardware work queue: with
# fewer queues than streams, a stream's kernels can wait behind another stream's kernels
# that share its queue. Set before CUDA initializes.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import argparse
import dataclasses
import json
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2310_16829_gb300 import workloads as WL  # noqa: E402

METRIC = "HAADF pixels/s (LMA mixed vs FP32, ≤1e-3 rel err); p50/p99 column-edit latency"
UNIT = "pixels/s"
# algorithmic work of one translate-slice on a 128 x 128 window: two 2D FFTs at
# 5 N log2 N flops (N = W^2) plus the transmission and propagator products at 6 flops each
W = 128
FLOPS_PER_TRANSLATE_SLICE = 2 * 5 * W * W * 14 + 12 * W * W   # 2,490,368
FP32_LANES_PER_SM = 128
# FP32 throughput reached by independent scalar FMA chains (152 x 4 CTAs of 256 threads) on this
# pool's GB300 at 2070 MHz: the practical ceiling beside the derived peak
FMA_MICROBENCH_TFLOPS = 74.3
# DRAM bytes (read + write) of one k_slice launch of one configuration (16384 translates x 50
# slices) from an ncu capture, with the SHA-256 of the kernel source it was taken on. The bench
# launch carries all configurations, so the figure is scaled by translate-slices (reads and the
# exit-wave writes both grow in proportion). It is reported only while the kernel source is
# the one captured; any change makes it null until a new capture is recorded here.
K_SLICE_TRAFFIC_CAPTURE = {"bytes": 506711808 + 2110760192, "translate_slices": 16384 * 50,
                           "source_sha256": "e007a227a1df6ee8842b4b3bbab88e6d1ffdb4a6f55732d1dd0afae383a8dfc9"}
KERNEL_SOURCE = os.path.join(ROOT, "paper_2310_16829_gb300", "csrc", "lma_kernels.cu")


def _kernel_source_sha() -> str:
    import hashlib
    return hashlib.sha256(open(KERNEL_SOURCE, "rb").read()).hexdigest()


def _sm_count(torch) -> int:
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ----------------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.active = False

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.active = True
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            if self.active:
                self.lines.append(line.strip())

    def stop(self) -> dict:
        self.active = False
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _gpu_id(torch) -> str:
    try:
        p = torch.cuda.get_device_properties(torch.cuda.current_device())
        return "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
    except Exception:
        return os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]


# ----------------------------------------------------------------------------------- oracle sample
SUB = 16   # probes per side of the CPU sample's subregion


def oracle_sample(w, workers: int, seed: int, c64: bool = False) -> dict:
    """Time the FP64 oracle, as it stands, on a bounded sample of the workload.

    The sample is one configuration: its transmission stack, the exit waves of every
    translate that a seeded 16 x 16-probe subregion needs, and those probes' synthesis and
    detection, spread over ``workers`` host processes (``oracle.pool``). The full-job time is
    extrapolated linearly in translates and probes:
    N_phi * (T_t + |I_f| * T_translate + |P| * T_probe), with the per-translate and per-probe
    wall times of the sample.
    """
    from oracle import pool as OP
    rng = np.random.default_rng(seed)
    a0 = int(rng.integers(0, w.region.npx - SUB + 1))
    b0 = int(rng.integers(0, w.region.npy - SUB + 1))
    probes = OP.subregion_probes(w.region, a0, b0, SUB, w.grid.nx, w.grid.ny)
    t0 = time.perf_counter()
    r = OP.readings(w, w.detectors, probes, phis=[0], c64=c64, workers=workers)
    wall = time.perf_counter() - t0
    sec = r["seconds"]
    n_tr = (w.grid.nx // (w.basis.in_spacing_px[0] * w.basis.f)) * (w.grid.ny // (w.basis.in_spacing_px[1] * w.basis.f))
    t_tr = sec["exit_waves"] / r["translates"]
    t_probe = sec["probes"] / len(probes)
    n_phi = len(w.phonons)
    full = n_phi * (sec["transmission"] + n_tr * t_tr + w.n_pixels * t_probe)
    return {"value": w.n_pixels / full, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": (f"configuration 0 of {n_phi}: transmission stack, the {r['translates']} of {n_tr} "
                       f"translate exit waves that the {SUB} x {SUB}-probe subregion at probe ({a0}, {b0}) "
                       f"needs, and its {len(probes)} of {w.n_pixels} probes, on {workers} host "
                       f"process(es); full job extrapolated linearly ({full:.0f} s)"),
            "extrapolation": {"configurations": n_phi, "translates": n_phi * n_tr / r["translates"],
                              "probes": n_phi * w.n_pixels / len(probes)},
            "phase_seconds": sec, "sample_seconds": wall, "coefficient_setup_s": sec["coefficients"],
            "subregion": (a0, b0), "probes": probes, "ref": r["ref"], "emu": r["emu"]}


def cpu_baseline(w, seed: int) -> dict:
    """The oracle on one host core and on every host core (the same seeded subregion)."""
    from oracle import pool as OP
    n = OP.default_workers()
    one = oracle_sample(w, 1, seed)
    many = oracle_sample(w, n, seed)
    keep = ("value", "cores", "sample", "extrapolation", "phase_seconds", "sample_seconds")
    out = {k: many[k] for k in keep}
    out.update({"unit": UNIT, "kind": "oracle", "nproc": os.cpu_count(), "cpu_model": OP.cpu_model(),
                "one_core": {k: one[k] for k in keep},
                "speedup_all_cores": many["value"] / one["value"]})
    # the parity sample (untimed): the same probes once more with the complex64 restatement
    par = oracle_sample(w, n, seed, c64=True)
    assert np.array_equal(par["ref"], many["ref"])
    return out, par


def sample_parity(ctx, w, sample: dict) -> dict:
    """The oracle's readings of the CPU sample's subregion (configuration 0) against the GPU
    path's image of the same probes with the same configuration, outside the timed region,
    under the tests' criterion: 1e-4 relative, or three times the complex64 floor of the same
    pixels (the oracle's pipeline restated in complex64)."""
    import torch
    from oracle import lma_c64 as C
    from paper_2310_16829_gb300 import lma
    w1 = w.with_phonons(1)
    a0, b0 = sample["subregion"]
    sp = w1.region.spacing_px
    reg = WL.Region(w1.region.px0 + a0 * sp[0], w1.region.py0 + b0 * sp[1], SUB, SUB, sp)
    spec = lma.Specimen(ctx, w1.grid, w1.potential, w1.phonons)
    ref, emu = sample["ref"], sample["emu"]

    def errors(prec):
        b = lma.Basis(ctx, spec, w1.probe, dataclasses.replace(w1.basis, precision=prec))
        got = b.image(w1.detectors, reg, recompute=True).reshape(len(w1.detectors), -1)
        b.close()
        rel = np.abs(got - ref) / ref
        ratio = np.abs(got - ref) / C.floor_bound(ref, emu, 1e-4, 3.0)
        return float(rel.max()), float(ratio.max())

    rel, ratio = errors(WL.PREC_C64)
    rel_h, _ = errors(WL.PREC_FP16_STORE)
    spec.close()
    torch.cuda.synchronize()
    kap = C.floor_scale(ref, emu)
    rel_emu = float(np.max(np.abs(emu - ref) / ref))
    return {"probes": int(ref.shape[1]), "configurations": 1, "detectors": len(w1.detectors),
            "readings_of_beam": [float(ref.min()), float(ref.max())],
            "max_rel_err_vs_oracle": rel, "complex64_restatement_max_rel_err": rel_emu,
            "kappa": [float(k) for k in kap],
            "worst_error_over_bound": ratio, "bound": "max(1e-4 x reading, 3 x kappa x sqrt(reading))",
            "pass": ratio <= 1.0,
            "fp16_store": {"max_rel_err_vs_oracle": rel_h}}


def run_reference(args, w) -> None:
    """The reference arm: the oracle as it stands on the host's cores, each step one bounded
    sample (a seeded 16 x 16-probe subregion of configuration 0) extrapolated to the job."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import pool as OP
    n = OP.default_workers()
    vals, secs = [], []
    for step in range(args.warmup + args.steps):
        r = oracle_sample(w, n, seed=100 + step)
        if step >= args.warmup:
            vals.append(r["value"])
            secs.append(r["sample_seconds"])
    v = statistics.mean(vals)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name, "parallelism": f"{n} host processes"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": n, "kind": "oracle",
                             "sample": r["sample"], "cpu_model": OP.cpu_model(), "nproc": os.cpu_count()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def edit_latency(n_edits: int, seed_base: int = 3000) -> dict:
    """Single-column edit latency on the resident serving specimen.

    20 x 20 ABO3 cells on a 1024^2 grid, 100 slices of 2 A, one configuration,
    all 65536 exit waves resident. Each request edits one seeded column (remove
    or change species, every slice) and images the 64 x 64 probes (4 px
    spacing) centred on it; only exit waves whose window meets the changed
    pixels are re-propagated (Sec. 4.2.6). Latency = host wall time of
    lma_edit_column + lma_image with a host output, per request.
    """
    from paper_2310_16829_gb300 import lma
    w = WL.serving_workload()
    ctx = lma.Context(0)
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    t0 = time.perf_counter()
    basis.propagate(0)
    full = basis.image(w.detectors, w.region)
    t_full = time.perf_counter() - t0
    dx = w.grid.lx / w.grid.nx
    lat, stale = [], []
    for req in range(n_edits):
        cx, cy, op, spc = WL.edit_request(20, req, seed_base)
        px = int(round(cx / dx)) // 4 * 4
        py = int(round(cy / dx)) // 4 * 4
        region = WL.Region(px - 32 * 4, py - 32 * 4, 64, 64, (4, 4))
        a = time.perf_counter()
        _, n_stale = spec.edit_column(basis, cx, cy, 0.5, op, spc)
        img = basis.image(w.detectors, region)
        lat.append(time.perf_counter() - a)
        stale.append(n_stale)
        assert np.all(np.isfinite(img))
    lat_ms = np.array(lat) * 1e3
    return {"workload": w.name, "requests": n_edits, "region_probes": 64 * 64,
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "mean_ms": float(lat_ms.mean()), "translates_repropagated_mean": float(np.mean(stale)),
            "translates_resident": int(basis.info().n_translates),
            "full_image_s": t_full, "full_image_pixels": int(full.size)}


def serving_measure(n_requests: int, loads=(0.5, 0.8), seed: int = 4000) -> dict:
    """Continuous batching on the serving mix (paper_2310_16829_gb300/serving.py).

    Lanes: edits on the resident 1024^2 / 100-slice specimen (64 x 64-probe region per
    edit), and full 256 x 256-probe images of fresh seeded 256^2 (20 slices), 512^2
    (50 slices) and 1024^2 (100 slices) ABO3 specimens, two warm instances each.
    HBM budget 75 % of the free memory. Mix 90 % edits / 10 % full images. Arrivals
    Poisson at `loads` x the capacity estimated from measured service times.
    """
    import torch
    from paper_2310_16829_gb300 import serving as S
    sizes = {"full_256": (5, 256, 20), "full_512": (10, 512, 50), "full_1024": (20, 1024, 100)}

    def builder(cells, nx, ns):
        return lambda sd: WL.perovskite_workload(cells=cells, nx=nx, n_slices=ns, n_phonons=1,
                                                 seed_base=sd, probes=256)

    # warm pool: every instance the stream may use is allocated and warmed before the
    # first arrival (device allocation can synchronize the device)
    lanes = [S.edit_lane(WL.serving_workload(), min_instances=1)]
    lanes += [S.image_lane(k, builder(*v), max_instances=2, min_instances=2) for k, v in sizes.items()]
    free, _ = torch.cuda.mem_get_info()
    srv = S.Server(lanes, budget_bytes=int(0.75 * free))
    rng = np.random.default_rng(seed)
    edit_k = [0]

    def make_requests(n):
        reqs = []
        for _ in range(n):
            if rng.random() < 0.9:
                cx, cy, op, spc = WL.edit_request(20, 1000 + edit_k[0], seed)
                edit_k[0] += 1
                reqs.append(S.EditRequest(cx, cy, op, spc, region_probes=64))
            else:
                lane = list(sizes)[int(rng.integers(0, 3))]
                reqs.append(S.ImageRequest(lane, seed=int(rng.integers(1 << 30))))
        return reqs

    # calibration: two requests per type (the first brings the instance up); service time
    # of the second
    svc = {}
    for lane in ["edit"] + list(sizes):
        for rep in range(2):
            if lane == "edit":
                cx, cy, op, spc = WL.edit_request(20, 900 + rep, seed)
                req = S.EditRequest(cx, cy, op, spc, region_probes=64)
            else:
                req = S.ImageRequest(lane, seed=7 + rep)
            r = srv.submit(req).wait(600)
            if r.error is not None:
                raise r.error
        svc[lane] = r.t_done - r.t_start
    mean_svc = 0.9 * svc["edit"] + 0.1 * sum(svc[k] for k in sizes) / 3
    capacity = 1.0 / mean_svc
    out = {"service_ms": {k: 1e3 * v for k, v in svc.items()}, "capacity_req_per_s": capacity,
           "budget_GB": srv.budget / 1e9, "loads": {}}
    for load in loads:
        reqs = make_requests(n_requests)
        arr = S.poisson_arrivals(n_requests, load * capacity, seed + int(100 * load))
        t0 = time.perf_counter()
        res = S.run_stream(srv, reqs, arr)
        span = time.perf_counter() - t0
        pix = sum(int(r.image.shape[-1] * r.image.shape[-2]) for r in res if r.image is not None)
        summ = S.latency_summary(res)
        summ["pixels_per_s"] = pix / span
        summ["offered_req_per_s"] = load * capacity
        out["loads"][str(load)] = summ
    out["instances"] = {k: len(l.instances) for k, l in srv.lanes.items()}
    srv.close()
    return out


def batching_measure(n_phonons: int, steps: int) -> dict:
    """Batched form against the plain complex64 LMA, on two sets of specimens.

    Uneven sizes: ABO3 5x5 cells on 256^2 (20 slices), 10x10 on 512^2 (50 slices), 20x20
    on 1024^2 (100 slices), 64^2 / 128^2 / 256^2 probes every 4 px, `n_phonons` seeded
    frozen-phonon configurations each. Many small specimens: 16 of 2x2 cells on 128^2
    (10 slices) and 8 of 5x5 cells on 256^2 (20 slices), 2 configurations each, with the
    full input lattice and with the sub-lattice f = 4 (64 / 256 translates per specimen).
      plain:   one lma_image per specimen, one configuration per slice and synthesis
               launch (phonon batch 1), one CTA per translate.
      batched: one lma_image_many call: configurations in phonon batches (as many as fit
               in memory), the slice work of all specimens of a pass in one launch (mode
               chosen by the autotuner), the whole call replayed as one CUDA graph.
    Both run on one stream with device outputs and are timed with CUDA events; the
    outputs of the two forms are compared bitwise.
    """
    out = _batching_case(WL.batch_workloads(n_phonons), n_phonons, steps,
                         "abo3 256^2/20sl + 512^2/50sl + 1024^2/100sl, %d configurations each" % n_phonons)
    out["small_specimens"] = _batching_case(
        WL.small_batch_workloads(2), 2, max(steps, 3),
        "16 x abo3 128^2/10sl + 8 x abo3 256^2/20sl, 2 configurations each")
    out["small_specimens_f4"] = _batching_case(
        WL.small_batch_workloads(2, f=4), 2, max(steps, 3),
        "16 x abo3 128^2/10sl + 8 x abo3 256^2/20sl, 2 configurations each, input sub-lattice f = 4")
    return out


def _batching_case(ws, n_phonons: int, steps: int, label: str) -> dict:
    import torch
    from paper_2310_16829_gb300 import lma
    from dataclasses import replace
    pixels = sum(w.n_pixels for w in ws)
    ctx = lma.Context(0)
    st = torch.cuda.Stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def make(pb):
        objs = []
        for w in ws:
            spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
            objs.append((spec, lma.Basis(ctx, spec, w.probe, replace(w.basis, phonon_batch=pb))))
        return objs

    def outs():
        return [torch.empty((1, w.region.npy, w.region.npx), dtype=torch.float64, device="cuda:0")
                for w in ws]

    def timed(fn):
        ms = []
        for _ in range(steps):
            torch.cuda.synchronize()
            ev[0].record(st)
            fn()
            ev[1].record(st)
            ev[1].synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        return float(np.mean(ms))

    objs = make(1)
    o_plain = outs()

    def plain():
        for (spec, basis), w, o in zip(objs, ws, o_plain):
            basis.image(w.detectors, w.region, out=o, recompute=True, stream=st)

    plain()
    ms_plain = timed(plain)
    ref = [o.cpu().numpy() for o in o_plain]
    for spec, basis in objs:
        basis.close()
        spec.close()
    torch.cuda.synchronize()

    objs = make(0)
    bases = [b for _, b in objs]
    regions = [w.region for w in ws]
    o_b = outs()
    t0 = time.perf_counter()
    lma.image_many(ctx, bases, ws[0].detectors, regions, o_b, graph=True, autotune=True, stream=st)
    st.synchronize()
    first_s = time.perf_counter() - t0

    def batched():
        lma.image_many(ctx, bases, ws[0].detectors, regions, o_b, graph=True, stream=st)

    batched()
    ms_b = timed(batched)
    same = all(np.array_equal(o.cpu().numpy(), r) for o, r in zip(o_b, ref))
    info = [b.info() for b in bases]
    out = {"workload": label, "pixels": pixels, "steps": steps,
           "plain": {"ms": ms_plain, "pixels_per_s": pixels / (ms_plain / 1e3)},
           "batched": {"ms": ms_b, "pixels_per_s": pixels / (ms_b / 1e3),
                       "phonon_batch": [int(i.phonon_batch) for i in info],
                       "passes": int(max(-(-n_phonons // max(1, i.phonon_batch)) for i in info)),
                       "first_call_s": first_s},
           "speedup": ms_plain / ms_b, "bitwise_equal": bool(same),
           "tuning": ctx.tuning(), "synth_tuning": ctx.synth_tuning()}
    for spec, basis in objs:
        basis.close()
        spec.close()
    ctx.close()
    return out


def profile_case_realspace(K: int) -> None:
    """The benchmark workload with one configuration, imaged twice with the K x K real-space
    propagation step (for ncu captures of k_slice_rs)."""
    import torch
    from paper_2310_16829_gb300 import lma
    w = WL.perovskite_workload(n_phonons=1)
    ctx = lma.Context(0)
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    out = torch.empty((1, w.region.npy, w.region.npx), dtype=torch.float64, device="cuda")
    for _ in range(2):
        basis.image_realspace(K, K, w.detectors, w.region, out=out, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    print(json.dumps({"profile_case_realspace": w.name, "K": K, "mean_haadf": float(out.mean())}))


def replica_workload(rank: int):
    """Replicas: rank r images its own specimen, the benchmark workload with frozen-phonon
    seeds 1000 + 97 r + phi (rank 0 is the single-GPU workload)."""
    return WL.perovskite_workload(seed_base=1000 + 97 * rank)


def max_over_ranks(total_ms: float, world: int, dist=None, device: str = "cuda") -> float:
    """The slowest rank's timed total (every rank gets it); world = 1 returns it unchanged."""
    if world > 1:
        import torch
        t = torch.tensor([total_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms


def profile_case(precision: str = "c64", window: int = 128, synth: str = "gather") -> None:
    """The benchmark workload with one configuration, imaged twice with RECOMPUTE, in the
    given precision (c64, fp16_store or mixed: the tensor-core slice kernel k_slice_tc).
    window = 64 or 256: the ABO3 256^2 specimen (5 x 5 cells, 20 slices, 4096 translates) with
    that propagation window instead (k_slice_64 or k_slice_256; store 0.13 or 2.1 GB).

    Launch order per pass: k_potential, k_slice (or k_slice_tc), k_synth_detect, k_finalize;
    with synth = "grouped", k_synth_group and then k_synth_detect over its probe waves.
    Device footprint about 2.5 GB (exit waves 2.15 GB, padded transmission 164 MB), and with
    the grouped synthesis the probe waves (2.15 GB).
    """
    import torch
    from paper_2310_16829_gb300 import lma
    if window == 128:
        w = WL.perovskite_workload(n_phonons=1)
    else:
        w = WL.perovskite_workload(cells=5, nx=256, n_slices=20, n_phonons=1)
        w = dataclasses.replace(w, basis=dataclasses.replace(w.basis, window=window))
    prec = {"c64": WL.PREC_C64, "fp16_store": WL.PREC_FP16_STORE, "mixed": WL.PREC_MIXED}[precision]
    w = dataclasses.replace(w, basis=dataclasses.replace(w.basis, precision=prec))
    ctx = lma.Context(0)
    ctx.set_synth_mode(lma.LMA_SYNTH_GROUPED if synth == "grouped" else lma.LMA_SYNTH_GATHER)
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    out = torch.empty((1, w.region.npy, w.region.npx), dtype=torch.float64, device="cuda")
    for _ in range(2):
        basis.image(w.detectors, w.region, out=out, recompute=True, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": w.name, "mean_haadf": float(out.mean())}))


def approx_curves() -> None:
    """Probe approximation error against L and f for the input-wave kinds of Sec. 4.2.3 (the
    error-versus-L figures) and for windows W = 64, 128, 256: host FP64 coefficients through
    the C-ABI, for the probe at pixel (0, 0) of the E2-like geometry of
    workloads.probe_approximation_workload. Prints one JSON line; no GPU work."""
    from paper_2310_16829_gb300 import lma
    ctx = lma.Context(-1)
    Ls = (1, 2, 4, 8, 12, 16, 24, 32, 48, 64)
    cases = [("probe", WL.BASIS_PROBE, {}, (1, 2, 4), (64, 128, 256)),
             ("gauss_0.482A", WL.BASIS_GAUSS, {"gauss_sigma": 0.482}, (1, 2, 4), (128, 256)),
             ("trig_lsq", WL.BASIS_TRIG, {}, (1, 2), (128, 256)),
             ("trig_closed", WL.BASIS_TRIG, {"coef_mode": 1}, (1,), (128,))]
    out = {}
    t0 = time.perf_counter()
    for name, kind, extra, fs, Ws in cases:
        out[name] = {}
        for W in Ws:
            for f in fs:
                rows = []
                for L in Ls:
                    w = WL.probe_approximation_workload(kind, f, L, window=W, **extra)
                    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
                    b = lma.Basis(ctx, spec, w.probe, w.basis)
                    err = b.coefficients(0, 0)[3]
                    rows.append([L, float(err[0]), float(err[1])])
                    b.close()
                    spec.close()
                out[name][f"W{W}_f{f}"] = rows
    ctx.close()
    print(json.dumps({"approx_curves": out, "geometry": "512^2 over 62.416 A, 200 kV, Z = 100 A, C_s = -2000 A, "
                      "alpha_max = 26 mrad, input waves every 2 f px at offset 1 px, windows W x W, probe at (0, 0)",
                      "columns": ["L", "err_l2", "err_sup"], "seconds": time.perf_counter() - t0}))


# ----------------------------------------------------------------------------------- main arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lma", choices=["lma", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--edits", type=int, default=24, help="column-edit requests timed (0: skip)")
    ap.add_argument("--serving", type=int, default=60, help="requests per offered load (0: skip)")
    ap.add_argument("--no-realspace", dest="realspace", action="store_false",
                    help="skip the real-space propagation measurement")
    ap.add_argument("--no-coherence", dest="coherence", action="store_false",
                    help="skip the partial-coherence (focal series) measurement")
    ap.add_argument("--no-partition", dest="partition", action="store_false",
                    help="skip the memory-bounded (partitioned) image measurement")
    ap.add_argument("--no-stem34", dest="stem34", action="store_false",
                    help="skip the 3D (rings) and 4D (pattern) STEM readout timings")
    ap.add_argument("--no-windows", dest="windows", action="store_false",
                    help="skip the W = 64 / 128 / 256 window timings on the 1024^2 specimen")
    ap.add_argument("--batch-phonons", type=int, default=32,
                    help="configurations per specimen of the uneven three-specimen batch (0: skip)")
    ap.add_argument("--profile-case", action="store_true",
                    help="one configuration of the workload, two image passes (for ncu captures)")
    ap.add_argument("--profile-precision", default="c64", choices=["c64", "fp16_store", "mixed"],
                    help="precision of --profile-case")
    ap.add_argument("--profile-window", type=int, default=128, choices=[64, 128, 256],
                    help="propagation window of --profile-case (64 and 256 on a 256^2 specimen)")
    ap.add_argument("--profile-synth", default="gather", choices=["gather", "grouped"],
                    help="synthesis form of --profile-case")
    ap.add_argument("--profile-case-realspace", type=int, default=0, metavar="K",
                    help="one configuration imaged twice with the K x K real-space step (for ncu)")
    ap.add_argument("--approx-curves", action="store_true",
                    help="probe approximation error against L and f per input-wave kind (host only)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    w = WL.perovskite_workload()
    if args.profile_case:
        profile_case(args.profile_precision, args.profile_window, args.profile_synth)
        return
    if args.approx_curves:
        approx_curves()
        return
    if args.profile_case_realspace:
        profile_case_realspace(args.profile_case_realspace)
        return
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    from paper_2310_16829_gb300 import lma

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # replicas: every rank simulates its own specimen (independent phonon seeds)
    if rank:
        w = replica_workload(rank)
    ctx = lma.Context(local)
    stream = torch.cuda.current_stream()
    spec = lma.Specimen(ctx, w.grid, w.potential, w.phonons)
    basis = lma.Basis(ctx, spec, w.probe, w.basis)
    region, dets = w.region, w.detectors
    out = torch.empty((len(dets), region.npy, region.npx), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    t_setup = time.perf_counter()
    basis.image(dets, region, out=out, recompute=True, stream=stream)   # coefficients + first pass
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for _ in range(args.warmup):
        basis.image(dets, region, out=out, recompute=True, stream=stream)
    torch.cuda.synchronize()

    clocks = ClockSampler(_gpu_id(torch))
    clocks.start()
    ctx.profile_enable(True)
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))                      # evict L2 between steps (outside the events)
        ev[k][0].record(stream)
        basis.image(dets, region, out=out, recompute=True, stream=stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if world > 1:
        import torch.distributed as dist
        total_ms = max_over_ranks(total_ms, world, dist)
    ms_per_step = total_ms / args.steps
    value = world * w.n_pixels / (ms_per_step / 1e3)
    img = out.cpu().numpy()

    # ---- other precisions on the same workload and step: the FP16 exit-wave store, and the
    # tensor-core form (split-FP16 32-point DFT stages on the tensor cores, complex64 store)
    def timed_precision(prec):
        wp = dataclasses.replace(w, basis=dataclasses.replace(w.basis, precision=prec))
        bp = lma.Basis(ctx, spec, wp.probe, wp.basis)
        out_p = torch.empty_like(out)
        for _ in range(1 + args.warmup):
            bp.image(dets, region, out=out_p, recompute=True, stream=stream)
        evp = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        torch.cuda.synchronize()
        barrier()
        ctx.profile_enable(True)
        for k in range(args.steps):
            flush.fill_(float(k))
            evp[k][0].record(stream)
            bp.image(dets, region, out=out_p, recompute=True, stream=stream)
            evp[k][1].record(stream)
        torch.cuda.synchronize()
        prp = ctx.profile_read()
        ctx.profile_enable(False)
        dist_mod = None
        if world > 1:
            import torch.distributed as dist_mod
        ms_p = max_over_ranks(sum(a.elapsed_time(b) for a, b in evp), world, dist_mod) / args.steps
        img_p = out_p.cpu().numpy()
        rel = np.abs(img_p - img) / np.abs(img)
        res = {"value": world * w.n_pixels / (ms_p / 1e3), "unit": UNIT, "ms_per_step": ms_p,
               "speedup_vs_c64": ms_per_step / ms_p,
               "max_rel_diff_vs_c64_all_pixels": float(rel.max()),
               "median_rel_diff_vs_c64": float(np.median(rel)),
               "slice_ms_per_launch": prp["slice"]["total_ms"] / max(1, prp["slice"]["launches"]),
               "exit_wave_GB": bp.info().exit_wave_bytes / 1e9}
        bp.close()
        return res

    mixed = timed_precision(WL.PREC_FP16_STORE)
    mixed["store"] = "exit waves as FP16 pairs with a per-wave power-of-two scale; FP32 propagation"
    tensor = timed_precision(WL.PREC_MIXED)
    tensor["form"] = ("32-point DFT stages of the slice step as split-FP16 (hi + lo) tcgen05 products, "
                      "FP32 accumulation in TMEM; pass B, transmission and propagator in FP32; complex64 store")
    sl_c64 = prof["slice"]["total_ms"] / max(1, prof["slice"]["launches"])
    tensor["slice_speedup_vs_fp32_kernel"] = sl_c64 / tensor["slice_ms_per_launch"]

    # ---- 3D and 4D STEM readouts of the same workload (Sec. 3.1): 20 rings of 5 mrad, and
    # the diffraction pattern on the 85 x 85 frequencies of the bandlimit's bounding square
    stem34 = None
    if args.stem34 and rank == 0:
        out_r = torch.empty((20, region.npy, region.npx), dtype=torch.float64, device="cuda")
        half = int(np.floor(w.basis.det_window / 3))     # |k| <= 42 at D = 128
        out_4 = torch.empty((region.npy, region.npx, 2 * half + 1, 2 * half + 1), dtype=torch.float32,
                            device="cuda")
        stem34 = {}
        for name, fn in (("rings_3d", lambda: basis.image_rings(0.005, 20, region, out=out_r, recompute=True,
                                                                  stream=stream)),
                         ("pattern_4d", lambda: basis.image_4d(half, half, region, out=out_4, recompute=True,
                                                                stream=stream))):
            fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(2):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 2
            stem34[name] = {"ms_per_image": ms, "pixels_per_s": w.n_pixels / (ms / 1e3),
                            "vs_2d_time": ms / ms_per_step}
        stem34["rings_3d"]["rings"] = "20 rings of 5 mrad from 0 (band ends at 86 mrad)"
        stem34["pattern_4d"]["pattern"] = f"{2 * half + 1} x {2 * half + 1} frequencies per probe, float32, " \
                                          f"{out_4.numel() * 4 / 1e9:.2f} GB per image"
        del out_r, out_4

    # ---- memory-bounded image (Sec. 4.2.4): 4096 resident exit waves per configuration
    # (0.54 GB instead of 2.15 GB), partition plans of the three strategies, and the plan
    # with the fewest Multislice runs timed on the same workload
    partition = None
    if args.partition and rank == 0:
        M = 4096
        plans = {}
        for name, strat in (("rows", lma.LMA_PART_ROWS), ("rectangles", lma.LMA_PART_RECTANGLES),
                            ("greedy", lma.LMA_PART_GREEDY)):
            t0 = time.perf_counter()
            _, n_parts, runs, peak = basis.partition(region, strat, M, start=0)
            plans[name] = {"parts": n_parts, "runs_per_configuration": runs, "peak_resident": peak,
                           "plan_s": time.perf_counter() - t0}
        codes = {"rows": lma.LMA_PART_ROWS, "rectangles": lma.LMA_PART_RECTANGLES, "greedy": lma.LMA_PART_GREEDY}
        best = min(plans, key=lambda k: plans[k]["runs_per_configuration"])
        out_p = torch.empty_like(out)
        basis.image_partitioned(dets, region, codes[best], M, out=out_p, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        basis.image_partitioned(dets, region, codes[best], M, out=out_p, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_p = e0.elapsed_time(e1)
        n_t = int(basis.info().n_translates)
        partition = {"max_resident": M, "store_GB": M * W * W * 8 / 1e9,
                     "unbounded_store_GB": n_t * W * W * 8 / 1e9,
                     "minimum_runs": n_t, "plans": plans,
                     "timed": {"strategy": best, "ms_per_image": ms_p, "pixels_per_s": w.n_pixels / (ms_p / 1e3),
                                          "vs_unbounded_time": ms_p / ms_per_step,
                                          "bitwise_equal_to_unbounded": bool(torch.equal(out_p, out))}}
        del out_p

    # ---- partial coherence: a focal series of 5 defocus values (Gaussian weights, 20 A
    # steps) from one set of exit waves, against 5 full images
    coherence = None
    if args.coherence and rank == 0:
        series = [(dz, 0.0, float(np.exp(-0.5 * (dz / 30.0) ** 2))) for dz in (-40.0, -20.0, 0.0, 20.0, 40.0)]
        out_c = torch.empty_like(out)
        basis.image_coherent(series, dets, region, out=out_c, recompute=True, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        basis.image_coherent(series, dets, region, out=out_c, recompute=True, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_c = e0.elapsed_time(e1)
        coherence = {"variants": len(series), "defocus_A": [v[0] for v in series],
                     "ms_per_image": ms_c, "pixels_per_s": w.n_pixels / (ms_c / 1e3),
                     "vs_one_image": ms_c / ms_per_step,
                     "speedup_vs_separate_images": len(series) * ms_per_step / ms_c}
        del out_c

    # ---- real-space propagation (Sec. 3.2): the propagation step as a K x K convolution,
    # one configuration of the workload, against the Fourier step; the cost model of
    # Sec. 3.2 predicts the ratio (1 + K^2) / (2 + 2 log2(W^2)) per slice
    realspace = None
    if args.realspace and rank == 0:
        w1 = w.with_phonons(1)
        spec1 = lma.Specimen(ctx, w1.grid, w1.potential, w1.phonons)
        b1 = lma.Basis(ctx, spec1, w1.probe, w1.basis)
        out1 = torch.empty_like(out)
        rows = []

        def timed_image(fn):
            fn()
            ctx.profile_enable(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            pr = ctx.profile_read()
            ctx.profile_enable(False)
            return e0.elapsed_time(e1), pr["slice"]["total_ms"]

        ms_f, sl_f = timed_image(lambda: b1.image(dets, region, out=out1, recompute=True, stream=stream))
        ref = out1.cpu().numpy()
        for K in (3, 5, 7, 9, 13, 25):
            ms_r, sl_r = timed_image(lambda: b1.image_realspace(K, K, dets, region, out=out1, stream=stream))
            img_r = out1.cpu().numpy()
            g_all, g_band = b1.realspace_gain(K, K)
            rows.append({"K": K, "ms_per_image": ms_r, "slice_ms": sl_r, "slice_vs_fourier": sl_r / sl_f,
                         "model_ratio": (1 + K * K) / (2 + 2 * 2 * np.log2(W)),
                         "per_slice_gain_max": g_all, "per_slice_gain_band": g_band,
                         "gain_over_slices": g_band ** w1.grid.n_slices,
                         "max_abs_diff_of_fourier_image_max": float(np.max(np.abs(img_r - ref)) / np.max(ref))})
        realspace = {"workload": w1.name, "fourier": {"ms_per_image": ms_f, "slice_ms": sl_f}, "kernels": rows}
        b1.close()
        spec1.close()
        del out1

    # ---- propagation windows W = 64, 128, 256 (detection window 128) on the serving specimen
    # (20 x 20 ABO3 cells, 1024^2, 100 slices, one configuration, 256 x 256 probes): image time
    # and the probe approximation error of each window (Sec. 4.2.1 option (ii), Sec. 4.2.3)
    windows = None
    if args.windows and rank == 0:
        ww = WL.serving_workload()
        wreg = WL.Region(0, 0, 256, 256, (4, 4))
        specw = lma.Specimen(ctx, ww.grid, ww.potential, ww.phonons)
        outw = torch.empty((len(dets), wreg.npy, wreg.npx), dtype=torch.float64, device="cuda")
        windows = {"workload": ww.name + " (window W, detection window 128)", "probes": wreg.npx * wreg.npy}
        for Wv in (64, 128, 256):
            bw = lma.Basis(ctx, specw, ww.probe, dataclasses.replace(ww.basis, window=Wv))
            bw.image(dets, wreg, out=outw, recompute=True, stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ctx.profile_enable(True)
            torch.cuda.synchronize()
            e0.record(stream)
            bw.image(dets, wreg, out=outw, recompute=True, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            prw = ctx.profile_read()
            ctx.profile_enable(False)
            ms_w = e0.elapsed_time(e1)
            err = bw.coefficients(0, 0)[3]
            windows[f"W{Wv}"] = {"ms_per_image": ms_w, "pixels_per_s": wreg.npx * wreg.npy / (ms_w / 1e3),
                                 "slice_ms": prw["slice"]["total_ms"], "synth_ms": prw["synth"]["total_ms"],
                                 "translate_slices": prw["slice"]["units"],
                                 "probe_err_l2": float(err[0]), "probe_err_sup": float(err[1]),
                                 "exit_wave_GB": bw.info().exit_wave_bytes / 1e9,
                                 "mean_haadf": float(outw.mean())}
            bw.close()
        specw.close()
        del outw

    # ---- end to end through the public API with host buffers
    host_out = np.empty((len(dets), region.npy, region.npx), dtype=np.float64)
    h2d = sum(a.x.nbytes + a.y.nbytes + a.species.nbytes + 4 * (w.grid.n_slices + 1) for a in w.phonons)
    e2e_steps = max(1, min(3, args.steps))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        spec.set_atoms(w.phonons)
        basis.image(dets, region, out=host_out, recompute=True)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_consistent = bool(np.array_equal(host_out, img))

    # ---- roofline of the dominant kernel (slice kernel, FP32 ALU bound)
    peaks = _peaks()
    sl = prof["slice"]
    slice_ms = sl["total_ms"] / max(1, sl["launches"])
    flops_per_launch = FLOPS_PER_TRANSLATE_SLICE * sl["units"] / max(1, sl["launches"])
    achieved = flops_per_launch / (slice_ms / 1e3) / 1e12
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sms = _sm_count(torch)
    peak = n_sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    cap = K_SLICE_TRAFFIC_CAPTURE
    traffic_current = cap["source_sha256"] == _kernel_source_sha()
    roofline = {"kernel": "k_slice", "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": (cap["bytes"] * (sl["units"] / max(1, sl["launches"])) / cap["translate_slices"])
                           if traffic_current else None,
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum of "
                                "the one-configuration launch, scaled by translate-slices); null when the "
                                "kernel source differs from the captured one",
                "peak_source": f"FP32 FMA: {n_sms} SMs (device query) x {FP32_LANES_PER_SM} lanes x 2 flop x "
                               f"{sm_max:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json); of measured clocks. "
                               f"An FMA-chain microbenchmark reached {FMA_MICROBENCH_TFLOPS} TFLOP/s on this GPU",
                "frac_of_fma_microbenchmark": achieved / FMA_MICROBENCH_TFLOPS,
                "algorithmic": f"{FLOPS_PER_TRANSLATE_SLICE} flop per translate-slice x "
                               f"{sl['units'] // max(1, sl['launches'])} translate-slices per launch",
                "share_of_step": sl["total_ms"] / max(1e-9, sum(v["total_ms"] for v in prof.values() if isinstance(v, dict))),
                "launch_ms": slice_ms}
    syn = prof["synth"]
    # the synthesis of one step: the grouped form is a group launch and a detection launch per
    # configuration, the gather one launch for all configurations
    synth_ms = syn["total_ms"] / args.steps
    u_bytes = basis.info().exit_wave_bytes
    n_translates = int(basis.info().n_translates)
    kernels = {k: {"launches_per_step": v["launches"] / args.steps,
                   "ms_per_launch": v["total_ms"] / max(1, v["launches"]),
                   "ms_per_step": v["total_ms"] / args.steps} for k, v in prof.items()
               if isinstance(v, dict)}
    # the synthesis of a step reads the exit-wave store of every configuration once
    kernels["synth"]["exit_wave_store_GBps"] = (u_bytes * len(w.phonons) / (synth_ms / 1e3) / 1e9
                                                if synth_ms else None)

    edits = None
    if rank == 0 and args.edits > 0:
        basis.close()                 # free the 8-configuration workload's exit waves first
        spec.close()
        torch.cuda.synchronize()
        edits = edit_latency(args.edits)
    serving = None
    if rank == 0 and args.serving > 0:
        torch.cuda.synchronize()
        serving = serving_measure(args.serving)

    batching = None
    if rank == 0 and args.batch_phonons > 0:
        torch.cuda.synchronize()
        # 32 configurations per specimen is about 19 s per pass: one timed pass per arm
        batching = batching_measure(args.batch_phonons, steps=1 if args.batch_phonons >= 16 else 2)

    cpu = None
    parity = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, sample = cpu_baseline(w, seed=5)
        parity = sample_parity(ctx, w, sample)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64",
            "data": "synthetic (seeded ABO3 slab, Gaussian frozen-phonon displacements)",
            "config": {"workload": w.name, "grid": [w.grid.nx, w.grid.ny], "slices": w.grid.n_slices,
                       "phonons": len(w.phonons), "probes": w.n_pixels,
                       "translates": n_translates, "L": w.basis.L, "W": W, "D": W,
                       "input_wave": "gaussian sigma=lambda/(2 alpha_max)", "precision": "complex64",
                       "detector_mrad": [1e3 * dets[0].r1, 1e3 * dets[0].r2],
                       "l2": "256 MiB buffer written between timed steps; per-step working set "
                             f"{u_bytes / 1e9:.2f} GB of exit waves > L2",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "parity": parity,
            "e2e": {"value": world * w.n_pixels / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(host_out.nbytes), "matches_device_run": e2e_consistent},
            "gpu_launches": int(sum(v["launches"] for v in prof.values() if isinstance(v, dict))),
            "allocations_timed": int(prof.get("allocations", 0)),
            "fp16_store": mixed,
            "tensor_core": tensor,
            "edit_latency": edits,
            "serving": serving,
            "batching": batching,
            "stem34": stem34,
            "partition": partition,
            "coherence": coherence,
            "realspace": realspace,
            "windows": windows,
            "clocks": clk,
            "kernels": kernels,
            "wall_s_timed_region": wall,
            "setup_s_first_call": t_setup,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
