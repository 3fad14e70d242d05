#!/usr/bin/env python
"""Benchmark: MOCCA iterations/s for 256x256 three-material spectral CT on GB300.

Workload (medium_256): 256 x 256 pixels of 0.5 mm, 512 views over 360 deg x 512
detector bins (flat detector, source 500 mm / detector 1000 mm), 4 overlapping
energy windows, 101 energy bins (20-120 keV), PMMA / Al / Gd basis, seeded
ellipse phantom with 4 Al and 6 Gd inserts, Poisson counts at 1e5 photons per
ray.  One step is one MOCCA iteration (forward projection + spectral model +
per-ray curvature and dual step, back-projection + block step-preconditioner +
primal step, D_TPL reduction) of one solve; a reconstruction is 500 steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

The GPU arm times K iterations with CUDA events (L2 flushed between steps),
reports per-kernel device time from events captured in the iteration graph,
the end-to-end rate through the host-buffer C-ABI call, the FP64 oracle on the
host cores as the CPU baseline, clocks sampled during the timed region, and
one JSON line on rank 0.  --impl reference times the FP64 oracle alone.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("MOCCA iters/sec & recon/s at 256² (served vs plain, 1 GB300) at 1e-4 rel L2; p50/p99")
WORKLOAD = "medium_256"
WORKLOAD_DESC = ("256x256 (0.5 mm), 512 views x 512 bins, 4 windows, 101 energies, 3 materials "
                 "(PMMA/Al/Gd), ellipse phantom 4 Al + 6 Gd, Poisson 1e5 photons/ray")
LAMBDA = 10.0 ** -7.5   # tuned with the oracle: tests/golden/lambda_sweeps.json
SOLVE_ITERS = 500
# the larger single solve, for profiling at a size whose working set exceeds L2 (--workload large_512)
LARGE = ("large_512", "512x512 (0.5 mm), 1024 views x 1024 bins, 4 windows, 101 energies, 3 materials "
         "(PMMA/Al/Gd), ellipse phantom 4 Al + 6 Gd, Poisson 1e6 photons/ray", 10.0 ** -8.5, 1000)
def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback (6.8 TB/s, earlier GB300 copy measurement)"


HBM_PEAK_GBPS, HBM_PEAK_SOURCE = _hbm_peak()


def _measured(key, default=None):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except (OSError, KeyError, ValueError, TypeError):
        return default


# Unit counts per SM of this GPU generation (the SM count and the clock come
# from the device at run time): 128 FP32 lanes (one FMA = 2 flop per clock
# each), 4 warp schedulers (one warp instruction issued per clock each),
# 128 bytes per clock from L1 to the register file, and one L1 data-pipe
# wavefront per clock (ncu's l1tex__data_pipe_lsu_wavefronts peak).
FP32_LANES_PER_SM, SCHEDULERS_PER_SM, L1_BYTES_PER_CLK_PER_SM, L1_WAVEFRONTS_PER_CLK_PER_SM = 128, 4, 128, 1
# Per launch of each per-iteration kernel, from one ncu --set full capture
# (cold cache) of the medium_256 workload: DRAM bytes (read + write), warp
# instructions executed and L1 data-pipe wavefronts (ncu's percentage of peak x
# elapsed SM cycles x the capturing GPU's SMs).  Valid only for that workload and for
# the kernel sources they were taken on (source_sha, see _source_sha).
NCU_WORKLOAD = "medium_256"
_SHA = "b6ce277f6d9a2514"
NCU_COUNTS = {
    "k_fp_proj": {"dram_bytes": 363276544 + 4203520, "warp_instructions": 41112016,
                  "l1_wavefronts": 16519622, "source_sha": _SHA},
    "k_mocca_ray": {"dram_bytes": 23119360 + 892672, "warp_instructions": 93367586,
                    "l1_wavefronts": 8975038, "source_sha": _SHA},
    # the back-projection's two launches: k_fpb_bp and k_fpb_finish
    "k_fpb_bp": {"dram_bytes": 436254720 + 4344320 + 19977984, "warp_instructions": 68896272 + 1998848,
                 "l1_wavefronts": 26924140 + 264357, "source_sha": _SHA},
}


def bp_view_groups(n_pixels, n_views):
    """View groups per pixel of the library's back-projection (the same rule as the
    library: enough threads to fill the GPU several times, at most 8, one view each)."""
    G = 8 if n_pixels <= 131072 else (4 if n_pixels <= 524288 else 2)
    while G > 1 and G > n_views:
        G >>= 1
    return G


def device_roofs(dev, sm_mhz):
    """Unit-count roofs of device `dev` at SM clock sm_mhz: FP32 TFLOP/s, warp
    instructions issued per second, L1-to-register TB/s; with how they were formed."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    ghz = sm_mhz / 1e3
    return {"sms": sms, "sm_mhz": sm_mhz,
            "fp32_tflops": sms * FP32_LANES_PER_SM * 2 * ghz / 1e3,
            "issue_per_s": sms * SCHEDULERS_PER_SM * ghz * 1e9,
            "l1_tbps": sms * L1_BYTES_PER_CLK_PER_SM * ghz / 1e3,
            "l1_wavefronts_per_s": sms * L1_WAVEFRONTS_PER_CLK_PER_SM * ghz * 1e9,
            "source": f"{sms} SMs (device) x per-SM unit counts x {sm_mhz:.0f} MHz (median SM clock sampled "
                      "during the timed steps)"}


KERNEL_SOURCES = ("mocca.cu", "osscir_internal.cuh", "osscir_launch.h")


def _source_sha() -> str:
    """Hash of the code of the per-iteration kernels (the traffic figures are tied to it):
    the sources with comments and blank lines removed, so that a comment edit keeps it,
    and the compiler flags."""
    from paper_1801_06263_gb300 import build as _b
    h = hashlib.sha256()
    h.update(" ".join(_b.FLAGS).encode())
    for f in KERNEL_SOURCES:
        text = open(os.path.join(ROOT, "paper_1801_06263_gb300", "csrc", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        lines = [ln.split("//", 1)[0].rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:16]


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        busy = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(ws, v):
    """Maximum of a per-rank value over all ranks (1 rank: the value itself)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws, units_per_rank, seconds_this_rank):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    t = _max_over_ranks(ws, seconds_this_rank)
    return ws * units_per_rank / t, t


# --------------------------------------------------------------------------- CPU oracle legs

def _oracle_problem(n_views=None):
    """The bench workload's counts for the oracle; with n_views, the same image,
    detector and spectra seen from n_views evenly spaced views of the full arc
    (every (512 / n_views)-th view of the workload)."""
    import numpy as np

    import oracle
    from paper_1801_06263_gb300 import inputs
    w = inputs.workload(WORKLOAD)
    if n_views is not None and n_views != w.geom.n_views:
        g = w.geom
        geom = inputs.make_geometry(g.n, g.pixel_mm, n_views, g.n_bins, bin_mm=g.bin_mm, sid_mm=g.sid_mm,
                                    sdd_mm=g.sdd_mm, arc_deg=g.arc_deg, start_deg=g.start_deg)
        w = inputs.Workload(w.name, geom, w.spectra, w.f_true, w.photons_per_ray, w.noise_seed, w.n_iters)
    cbar = oracle.counts(w.geom, w.spectra, w.f_true)
    c = inputs.poisson_counts(cbar, w.noise_seed)
    return w, np.ascontiguousarray(c)


def cpu_oracle_rate(n_iters: int, threads: int = 0):
    """FP64 oracle MOCCA iterations/s on the host cores for n_iters iterations
    (threads = 0: all cores)."""
    import oracle
    w, c = _oracle_problem()
    n_all = oracle.max_threads()
    if threads:
        oracle.set_threads(threads)
    try:
        used = oracle.max_threads()
        t0 = time.perf_counter()
        oracle.mocca(w.geom, w.spectra, c, n_iters, LAMBDA)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(n_all)
    return n_iters / dt, used, dt


REFERENCE_BUDGET_S = 150.0   # whole --impl reference run (warm-up and timed steps)


def run_reference(args):
    """The FP64 oracle on the host cores.  Each step is one MOCCA iteration on a
    bounded sample of the workload: the same image, detector and spectra seen
    from an evenly spaced subset of the 512 views, as many as keep all warm-up
    and timed steps within REFERENCE_BUDGET_S.  The work of an iteration is
    proportional to the number of rays, so the rate is reported as iterations/s
    of the full workload (sample rate x sample views / 512)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_1801_06263_gb300 import inputs
    full_views = inputs.workload(WORKLOAD).geom.n_views
    # calibrate on an 8-view sample, then take the largest power-of-two view count in budget
    w8, c8 = _oracle_problem(8)
    t0 = time.perf_counter()
    oracle.mocca(w8.geom, w8.spectra, c8, 1, LAMBDA)
    per_view = (time.perf_counter() - t0) / 8
    n_steps = max(1, args.steps + args.warmup)
    views = 8
    while views * 2 <= full_views and n_steps * per_view * views * 2 <= REFERENCE_BUDGET_S:
        views *= 2
    w, c = (w8, c8) if views == 8 else _oracle_problem(views)
    st = None
    for _ in range(args.warmup):
        st, _ = oracle.mocca(w.geom, w.spectra, c, 1, LAMBDA, st)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st, _ = oracle.mocca(w.geom, w.spectra, c, 1, LAMBDA, st)
    dt = time.perf_counter() - t0
    frac = views / full_views
    v = frac * args.steps / dt
    sample = (f"each step one MOCCA iteration of {WORKLOAD} from {views} of its {full_views} views "
              f"(one in every {full_views // views}), FP64 C oracle; rate scaled by {views}/{full_views}")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "iter/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps / frac,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": f"{WORKLOAD}: {WORKLOAD_DESC}", "lambda": LAMBDA},
        "cpu_baseline": {"value": v, "unit": "iter/s", "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm

def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    from paper_1801_06263_gb300 import Reconstructor, _lib, inputs, osscir_footprint_rays

    w = inputs.workload(WORKLOAD)
    R = Reconstructor(w.geom, w.spectra, LAMBDA)
    f4 = torch.zeros((w.geom.n_pixels, 4), dtype=torch.float32, device="cuda")
    f4[:, :3] = torch.tensor(w.f_true, dtype=torch.float32, device="cuda")
    chat = R.simulate(f4)
    c = _lib.osscir_poisson_noise(chat, w.noise_seed + (rank << 32))
    R.set_counts(c)
    # footprint size: number of (ray, pixel) pairs, the unit of the projector work
    cnt = torch.zeros(w.geom.n_rays, dtype=torch.int32, device="cuda")
    osscir_footprint_rays(R.handle, 0, w.geom.n_rays, 0, cnt, None, None)
    nnz = int(cnt.sum().item())

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for i in range(args.warmup):
        flush.fill_(i & 0xFF)
        R.step(1)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kms = []
    _barrier(ws)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.fill_((k + 1) & 0xFF)          # L2 flush between steps, outside the timed events
            ev[k][0].record(stream)
            R.step(1)
            ev[k][1].record(stream)
            kms.append(_lib.osscir_last_kernel_ms(R.handle))   # synchronises the stream
        torch.cuda.synchronize()
    _barrier(ws)
    step_ms = [s.elapsed_time(e) for s, e in ev]
    value, total_s = whole_job_rate(ws, args.steps, sum(step_ms) / 1e3)
    d_last = R.dtpl(1)

    # end to end: full reconstructions through the host-buffer C-ABI call
    e2e_steps = max(1, args.e2e)
    c_host = c.cpu().pin_memory()
    maps_host = torch.empty((w.geom.n_pixels, 4), dtype=torch.float32).pin_memory()
    _lib.osscir_reconstruct(R.handle, c_host, 5, maps_host)          # warm-up
    _barrier(ws)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        _lib.osscir_reconstruct(R.handle, c_host, SOLVE_ITERS, maps_host)
    e2e_rate, _ = whole_job_rate(ws, e2e_steps * SOLVE_ITERS, time.perf_counter() - t0)
    finite = bool(torch.isfinite(maps_host).all().item())

    nested = run_nested(args, w, c) if args.nested else None
    five = run_five_windows(args, w, f4, rank) if args.five_windows > 0 else None
    vsplit = run_view_split(args, w, c, 1e3 * total_s / args.steps) if args.split else None
    served = run_served(args, w, R, chat, rank) if args.served > 0 else None
    batched = run_batched(args, rank) if args.batch > 0 else None
    mixed = run_served_mixed(args, rank) if args.mixed > 0 else None

    if rank != 0:
        return 0
    L, nE, P = w.geom.n_rays, w.spectra.n_energies, w.geom.n_pixels
    mean = [statistics.mean(k[i] for k in kms) for i in range(3)]
    dev_bytes, table_bytes = _lib.osscir_memory(R.handle)
    G = bp_view_groups(P, w.geom.n_views)
    if table_bytes:
        # footprint tables: the projections stream them.  Algorithmic HBM bytes per
        # launch: forward 6 B per footprint pair (weight, 16-bit pixel step) + xbar read
        # (16 B per pixel) + g written and the pair count and first pixel read (24 B per
        # ray); back-projection 6 B per pair (weight, stage slot) + the view groups'
        # channel sums written and read (2 x 36 B per pixel and group) + x read and
        # written, xbar and its column-major copy written (64 B per pixel)
        names = ("k_fp_proj", "k_mocca_ray", "k_fpb_bp")
        alg = (6.0 * nnz + 16.0 * P + 24.0 * L, None, 6.0 * nnz + 72.0 * G * P + 64.0 * P)
    else:
        names = ("k_mocca_proj", "k_mocca_ray", "k_mocca_bp")
        alg = (None, None, None)
    kern = {
        # projection: 3 FMA per footprint pair (three materials)
        names[0]: {"ms": mean[0], "flop": 6.0 * nnz, "bytes": alg[0]},
        # per-ray step: 29 FMA per (ray, energy): p_i (3), D_w (4), alpha numerators (12),
        # beta_i (4) and sum_i beta_i mu_i mu_i^T (6); the per-ray 3x3 algebra is not counted
        names[1]: {"ms": mean[1], "flop": 58.0 * L * nE, "bytes": alg[1]},
        # back-projection: 9 FMA per footprint pair (K^T y' and the 6-channel block SPC)
        names[2]: {"ms": mean[2], "flop": 18.0 * nnz, "bytes": alg[2]},
    }
    dom = max(kern, key=lambda k: kern[k]["ms"])
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or _measured("sm_max_mhz", 2070.0)
    roofs = device_roofs(local, sm_mhz)
    sha = _source_sha()
    ncu = {k: (v if WORKLOAD == NCU_WORKLOAD and v.get("source_sha") == sha else None) for k, v in NCU_COUNTS.items()}
    kernels = {}
    for k, v in kern.items():
        sec = v["ms"] * 1e-3
        row = {"ms": v["ms"], "algorithmic_tflops": v["flop"] / sec / 1e12,
               "alu_frac": v["flop"] / sec / 1e12 / roofs["fp32_tflops"]}
        if v["bytes"]:
            row["algorithmic_GBps"] = v["bytes"] / sec / 1e9
            row["hbm_frac"] = v["bytes"] / sec / 1e9 / HBM_PEAK_GBPS
        if ncu.get(k):
            # issue: the warp instructions the kernel executed over the issue slots of its duration
            row["warp_instructions"] = ncu[k]["warp_instructions"]
            row["issue_frac"] = ncu[k]["warp_instructions"] / (sec * roofs["issue_per_s"])
            row["dram_bytes"] = ncu[k]["dram_bytes"]
            row["dram_frac"] = ncu[k]["dram_bytes"] / sec / 1e9 / HBM_PEAK_GBPS
            row["l1_wavefronts"] = ncu[k]["l1_wavefronts"]
            row["l1_frac"] = ncu[k]["l1_wavefronts"] / (sec * roofs["l1_wavefronts_per_s"])
            # the binding roof: the unit the kernel keeps busiest
            fr = {"hbm": row["dram_frac"], "instruction issue": row["issue_frac"], "L1 data pipe": row["l1_frac"]}
            row["binding"] = max(fr, key=fr.get)
        else:
            row["binding"] = "hbm" if v["bytes"] else "instruction issue"
        kernels[k] = row
    traffic = ncu[dom]["dram_bytes"] if ncu.get(dom) else None
    if kern[dom]["bytes"]:
        ach = kern[dom]["bytes"] / (kern[dom]["ms"] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": HBM_PEAK_GBPS, "unit": "GB/s",
                    "frac": ach / HBM_PEAK_GBPS, "traffic": traffic, "peak_source": HBM_PEAK_SOURCE,
                    "algorithmic_bytes": kern[dom]["bytes"]}
        if ncu.get(dom):
            ach_w = ncu[dom]["l1_wavefronts"] / (kern[dom]["ms"] * 1e-3)
            roofline["binding"] = {"unit": "L1 data-pipe wavefronts", "wavefronts": ncu[dom]["l1_wavefronts"],
                                   "achieved": ach_w / 1e12, "peak": roofs["l1_wavefronts_per_s"] / 1e12,
                                   "peak_unit": "T wavefronts/s", "frac": ach_w / roofs["l1_wavefronts_per_s"]}
    else:
        ach = kern[dom]["flop"] / (kern[dom]["ms"] * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": roofs["fp32_tflops"],
                    "unit": "TFLOP/s", "frac": ach / roofs["fp32_tflops"], "traffic": traffic,
                    "peak_source": roofs["source"] + "; 128 FP32 lanes x 2 flop per clock per SM"}
        if ncu.get(dom):
            ach_i = ncu[dom]["warp_instructions"] / (kern[dom]["ms"] * 1e-3)
            roofline["binding"] = {"unit": "instruction issue", "warp_instructions": ncu[dom]["warp_instructions"],
                                   "achieved": ach_i / 1e12, "peak": roofs["issue_per_s"] / 1e12,
                                   "peak_unit": "T warp-instr/s", "frac": ach_i / roofs["issue_per_s"]}
    cpu = None
    if ws == 1 and args.cpu_iters > 0:
        rate, cores, dt = cpu_oracle_rate(args.cpu_iters)
        cpu = {"value": rate, "unit": "iter/s", "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_iters} full MOCCA iterations of {WORKLOAD} (FP64 C oracle, {dt:.1f} s)"}
        if args.cpu_iters_1t > 0:
            r1, _, dt1 = cpu_oracle_rate(args.cpu_iters_1t, threads=1)
            cpu["one_thread"] = {"value": r1, "unit": "iter/s", "cores": 1,
                                 "sample": f"{args.cpu_iters_1t} full MOCCA iteration(s), one thread ({dt1:.1f} s)"}
    line = {
        "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: {WORKLOAD_DESC}", "solve_iterations": SOLVE_ITERS,
                   "lambda": LAMBDA, "l2": "flushed between steps (256 MB write)",
                   "parallelism": "independent solves per GPU" if ws > 1 else "single solve"},
        "recon_per_s": value / SOLVE_ITERS,
        "kernel_ms": {k: v["ms"] for k, v in kern.items()},
        "footprint_pairs": nnz,
        "intersections_per_s": 2.0 * nnz / (total_s / args.steps) * ws,
        "roofline": roofline,
        "kernels": kernels,
        "memory": {"context_bytes": dev_bytes, "footprint_table_bytes": table_bytes},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_rate, "unit": "iter/s", "h2d_bytes_per_step": int(c_host.numel() * 4),
                "d2h_bytes_per_step": int(maps_host.numel() * 4),
                "step": f"one {SOLVE_ITERS}-iteration reconstruction via osscir_reconstruct (pinned host buffers)",
                "recon_per_s": e2e_rate / SOLVE_ITERS},
        "plain_recon_per_s": e2e_rate / SOLVE_ITERS,
        "nested": nested,
        "view_split": vsplit,
        "five_windows": five,
        "served": served,
        "batched": batched,
        "served_mixed": mixed,
        "clocks": clocks,
        "gpu_launches": (5 if table_bytes else 4) * args.steps,   # proj, ray, reduction, bp (+ group sums)
        "dtpl_last": d_last,
        "maps_finite": finite,
    }
    print(json.dumps(line), flush=True)
    R.close()
    return 0


def run_nested(args, w, c):
    """Nested MOCCA (a new local model every k iterations; k = 1 is the single
    loop) on the headline workload: device time of the iterations and D_TPL at
    the maps x after 50, 100, 200 and SOLVE_ITERS iterations from zero."""
    import torch
    from paper_1801_06263_gb300 import Reconstructor

    marks = [m for m in (50, 100, 200) if m < SOLVE_ITERS] + [SOLVE_ITERS]
    stream = torch.cuda.current_stream()
    out = {}
    for k in args.nested:
        R = Reconstructor(w.geom, w.spectra, LAMBDA, inner=k)
        R.set_counts(c)
        R.step(2 * k)                                   # warm-up (both graphs)
        R.set_counts(c)
        done, ms, rows = 0, 0.0, []
        for m in marks:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            R.step(m - done)
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
            done = m
            rows.append({"iterations": m, "ms": ms, "dtpl_at_x": R.dtpl(0)})
        R.close()
        out[str(k)] = {"ms_per_iteration": ms / done, "trajectory": rows}
    return out


def run_view_split(args, w, c, serial_ms):
    """One solve split by views over N ranks (osscir_mocca_partial per rank's views,
    the channels summed, osscir_mocca_apply): the rank-local work measured on this
    one GPU.  Each rank's share and the sum with the primal step are captured as
    CUDA graphs (so host launch latency does not stand in for device time) and
    replayed in turn each iteration, so the solve follows the split iteration
    exactly; CUDA events around each replay.  The sum of the ranks' channels
    stands in for the all-reduce of 9 P floats, which N GPUs would add (not
    measured: one GPU here).  L2 is flushed before each iteration;
    vs_single_graph divides the headline's per-iteration time (also L2-flushed)
    by the largest rank share plus the primal step."""
    import statistics
    import torch
    from paper_1801_06263_gb300 import Reconstructor, _lib
    from paper_1801_06263_gb300.split import view_range

    stream = torch.cuda.current_stream()
    P, V = w.geom.n_pixels, w.geom.n_views
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for N in args.split:
        R = Reconstructor(w.geom, w.spectra, LAMBDA)
        R.set_counts(c)
        ranges = [view_range(V, r, N) for r in range(N)]
        chans = [torch.zeros((9, P), dtype=torch.float32, device="cuda") for _ in range(N)]
        total = torch.zeros((9, P), dtype=torch.float32, device="cuda")

        def share(r):
            _lib.osscir_mocca_partial(R.handle, ranges[r][0], ranges[r][1], chans[r])

        def combine():
            total.copy_(chans[0])
            for ch in chans[1:]:
                total.add_(ch)
            _lib.osscir_mocca_apply(R.handle, total)

        for _ in range(3):   # eager warm-up: builds the tables
            for r in range(N):
                share(r)
            combine()
        torch.cuda.synchronize()
        graphs = []
        for fn in [lambda r=r: share(r) for r in range(N)] + [combine]:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                fn()
            graphs.append(g)
        part_ms, apply_ms = [[] for _ in range(N)], []
        for it in range(2 + args.split_steps):
            flush.fill_(it & 0xFF)   # L2 flushed before each iteration, as for the headline steps
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(N + 1)]
            for k, g in enumerate(graphs):
                evs[k][0].record(stream)
                g.replay()
                evs[k][1].record(stream)
            torch.cuda.synchronize()
            if it >= 2:
                for r in range(N):
                    part_ms[r].append(evs[r][0].elapsed_time(evs[r][1]))
                apply_ms.append(evs[N][0].elapsed_time(evs[N][1]))
        per_rank = [statistics.mean(m) for m in part_ms]
        ap = statistics.mean(apply_ms)
        out[str(N)] = {"rank_views": [v1 - v0 for v0, v1 in ranges], "rank_ms": per_rank,
                       "sum_and_apply_ms": ap, "allreduce_bytes": 36 * P,
                       "rank_ms_per_iteration": max(per_rank) + ap,
                       "vs_single_graph": serial_ms / (max(per_rank) + ap),
                       "finite": bool(torch.isfinite(R.maps()).all().item())}
        del graphs
        R.close()
    return {"note": "rank-local work of an N-way view split measured on one GPU (every share run in turn "
                    "as a CUDA graph); N GPUs add one all-reduce of allreduce_bytes per iteration, not included",
            "split": out}


def run_five_windows(args, w, f4, rank):
    """The headline solve with five ideal windows (20-40-50-65-80-120 keV) in place
    of four: device time per iteration and per kernel, L2 flushed between steps."""
    import statistics as st
    import torch
    from paper_1801_06263_gb300 import Reconstructor, _lib, inputs

    sp = inputs.make_spectra(w.geom.n_bins, w.photons_per_ray, ideal_windows=True, n_windows=5)
    R = Reconstructor(w.geom, sp, LAMBDA)
    c = _lib.osscir_poisson_noise(R.simulate(f4), w.noise_seed + 5 + (rank << 32))
    R.set_counts(c)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    R.step(3)
    kms, ms = [], []
    for k in range(args.five_windows):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        R.step(1)
        b.record(stream)
        kms.append(_lib.osscir_last_kernel_ms(R.handle))
        ms.append(a.elapsed_time(b))
    d = R.dtpl(1)
    R.close()
    return {"ms_per_iteration": st.mean(ms), "kernel_ms": [st.mean(k[i] for k in kms) for i in range(3)],
            "iterations": args.five_windows, "dtpl_last": d, "windows": "20-40-50-65-80-120 keV, ideal",
            "counts_per_ray_bytes": 32}


def run_batched(args, rank):
    """64 independent reconstructions of uneven sizes (n in {128..512}, 90-720 views,
    1e4-1e6 photons per ray): one MOCCA iteration of all of them per step, (a) each
    solve's own iteration graph one after another (plain per-solve form), (b) the
    batched kernels with the default configuration, (c) after autotuning.  Inputs
    (maps, rays, tables, about 2 GB) exceed L2; nothing is flushed between steps."""
    import numpy as np
    import torch
    from paper_1801_06263_gb300 import Batch, Reconstructor, _lib, inputs

    ws = inputs.batch_workloads(args.batch)
    recs = []
    for i, w in enumerate(ws):
        R = Reconstructor(w.geom, w.spectra, inputs.step_ratio(w.geom.n, w.photons_per_ray))
        f4 = torch.zeros((w.geom.n_pixels, 4), dtype=torch.float32, device="cuda")
        f4[:, :3] = torch.tensor(w.f_true, dtype=torch.float32, device="cuda")
        R.set_counts(_lib.osscir_poisson_noise(R.simulate(f4), w.noise_seed + (rank << 32)))
        recs.append(R)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    K = max(1, args.batch_steps)

    def timed(step):
        for _ in range(2):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K

    def plain_step():
        for R in recs:
            R.step(1)

    plain_ms = timed(plain_step)
    B = Batch(recs)
    default_ms = timed(lambda: B.step(1))
    kms_default = _lib.osscir_batch_last_kernel_ms(B.handle)
    B.close()
    t0 = time.perf_counter()
    B = Batch(recs, autotune=True)
    tune_s = time.perf_counter() - t0
    tuned_ms = timed(lambda: B.step(1))
    kms_tuned = _lib.osscir_batch_last_kernel_ms(B.handle)
    cfg = B.config
    B.close()
    finite = sum(1 for R in recs if np.isfinite(R.dtpl(1)))
    P = sum(w.geom.n_pixels for w in ws)
    L = sum(w.geom.n_rays for w in ws)
    # per iteration: x_n, x_{n-1} read, x_{n+1} written; the per-ray fields; and the footprint
    # tables, which the batch streams once per iteration (about all of their bytes)
    table_bytes = sum(_lib.osscir_memory(R.handle)[1] for R in recs)
    alg_bytes = 48.0 * P + 124.0 * L + table_bytes
    best_ms = min(default_ms, tuned_ms)
    # per kernel of the default configuration (one branch: one launch per kernel for all
    # solves), the algorithmic bytes of the plain path's table kernels summed over the
    # solves: forward 6 B per footprint pair + 16 B per pixel + 24 B per ray; back-projection
    # 6 B per pair + 72 B per pixel and view group + 64 B per pixel
    from paper_1801_06263_gb300 import osscir_footprint_rays
    fwd_bytes = bp_bytes = 0.0
    for R, w in zip(recs, ws):
        cnt = torch.zeros(w.geom.n_rays, dtype=torch.int32, device="cuda")
        osscir_footprint_rays(R.handle, 0, w.geom.n_rays, 0, cnt, None, None)
        nnz = float(cnt.sum().item())
        Ps, Ls = w.geom.n_pixels, w.geom.n_rays
        fwd_bytes += 6.0 * nnz + 16.0 * Ps + 24.0 * Ls
        bp_bytes += 6.0 * nnz + 72.0 * bp_view_groups(Ps, w.geom.n_views) * Ps + 64.0 * Ps
    per_kernel = {}
    for name, ms, nbytes in (("proj", kms_default[0], fwd_bytes), ("bp", kms_default[2], bp_bytes)):
        gbps = nbytes / (ms * 1e-3) / 1e9
        per_kernel[name] = {"ms": ms, "algorithmic_bytes": nbytes, "achieved_GBps": gbps,
                            "hbm_frac": gbps / HBM_PEAK_GBPS}
    for R in recs:
        R.close()
    mix = {}
    for w in ws:
        mix[w.geom.n] = mix.get(w.geom.n, 0) + 1
    return {
        "solves": len(ws), "image_sizes": {str(k): v for k, v in sorted(mix.items())},
        "views": [min(w.geom.n_views for w in ws), max(w.geom.n_views for w in ws)],
        "pixels": P, "rays": L, "steps": K,
        "plain_ms_per_iteration": plain_ms, "batched_ms_per_iteration": default_ms,
        "tuned_ms_per_iteration": tuned_ms, "speedup_vs_plain": plain_ms / best_ms,
        "solve_iterations_per_s": len(ws) * 1e3 / best_ms,
        "kernel_ms_default": list(kms_default), "kernel_ms_tuned": list(kms_tuned),
        "tuned_config": cfg, "autotune_s": tune_s, "finite_solves": finite,
        "hbm": {"algorithmic_bytes_per_iteration": alg_bytes, "footprint_table_bytes": table_bytes,
                "achieved_GBps": alg_bytes / (best_ms * 1e-3) / 1e9,
                "peak_GBps": HBM_PEAK_GBPS, "frac": alg_bytes / (best_ms * 1e-3) / 1e9 / HBM_PEAK_GBPS,
                "peak_source": HBM_PEAK_SOURCE, "projector_kernels_default_config": per_kernel},
    }


def run_served(args, w, R, chat, rank):
    """Served form, 150 GB budget, args.slots slots, SOLVE_ITERS iterations per
    request, each request with its own seeded Poisson counts of the workload:
    (1) a burst of args.served requests submitted at once (saturated
    throughput), (2) args.served requests with seeded Poisson arrivals at
    args.rate requests/s (below capacity: p50 / p99 latency)."""
    import numpy as np
    import torch

    from paper_1801_06263_gb300 import _lib
    counts = []
    for k in range(args.served):
        counts.append(_lib.osscir_poisson_noise(chat, 3000 + k + (rank << 32)).cpu().numpy())
    sp = w.spectra

    def run(gaps):
        srv = _lib.osscir_server_create(150 << 30, args.slots)
        try:
            t = _lib.osscir_submit(srv, w.geom, sp.s, sp.N, sp.mu, LAMBDA, counts[0], 5)   # warm the cache
            _lib.osscir_poll(srv, t, -1)
            t0 = time.perf_counter()
            tickets = []
            for k in range(args.served):
                target = t0 + float(np.sum(gaps[:k]))
                while time.perf_counter() < target:
                    time.sleep(min(0.0005, max(0.0, target - time.perf_counter())))
                tickets.append(_lib.osscir_submit(srv, w.geom, sp.s, sp.N, sp.mu, LAMBDA, counts[k], SOLVE_ITERS))
            lat, ok = [], True
            for t in tickets:
                rc, st = _lib.osscir_poll(srv, t, -1)
                ok = ok and rc == 0
                lat.append(st.latency_ms)
            wall = time.perf_counter() - t0
        finally:
            _lib.osscir_server_destroy(srv)
        return wall, np.array(lat), ok

    wall_b, lat_b, ok_b = run(np.zeros(args.served))
    rng = np.random.default_rng(3000 + rank)
    wall_p, lat_p, ok_p = run(rng.exponential(1.0 / args.rate, size=args.served))
    return {"recon_per_s": args.served / wall_b, "iters_per_s": args.served * SOLVE_ITERS / wall_b,
            "burst_p50_ms": float(np.percentile(lat_b, 50)), "burst_p99_ms": float(np.percentile(lat_b, 99)),
            "poisson_rate_per_s": args.rate, "p50_ms": float(np.percentile(lat_p, 50)),
            "p99_ms": float(np.percentile(lat_p, 99)), "poisson_recon_per_s": args.served / wall_p,
            "requests": args.served, "slots": args.slots, "all_ok": bool(ok_b and ok_p),
            "note": "burst of requests for throughput; seeded Poisson arrivals below capacity for latency; "
                    "150 GB budget; admitted requests batched in up to 4 groups, one stream each"}


def run_served_mixed(args, rank):
    """Mixed requests (128^2-512^2, 90-1024 views, 200-500 iterations, 1e4-1e6
    photons per ray) at seeded Poisson arrival rates, through a fresh server
    (150 GB budget, args.slots slots, no cached contexts) per rate, beside the
    plain per-solve form (create, load, iterate, read back, release, one request
    after another) on the same requests."""
    import numpy as np
    import torch

    from paper_1801_06263_gb300 import Reconstructor, _lib, inputs
    reqs = inputs.served_requests(args.mixed, seed=3000 + rank)
    counts = []
    for w in reqs:
        lam = inputs.step_ratio(w.geom.n, w.photons_per_ray)
        R = Reconstructor(w.geom, w.spectra, lam)
        f4 = torch.zeros((w.geom.n_pixels, 4), dtype=torch.float32, device="cuda")
        f4[:, :3] = torch.tensor(w.f_true, dtype=torch.float32, device="cuda")
        counts.append(_lib.osscir_poisson_noise(R.simulate(f4), w.noise_seed + (rank << 32)).cpu().numpy())
        R.close()
    lams = [inputs.step_ratio(w.geom.n, w.photons_per_ray) for w in reqs]
    total_iters = sum(w.n_iters for w in reqs)

    # plain per-solve form, one request after another
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for w, c, lam in zip(reqs, counts, lams):
        R = Reconstructor(w.geom, w.spectra, lam)
        c_host = torch.from_numpy(c).pin_memory()
        out = torch.empty((w.geom.n_pixels, 4), dtype=torch.float32).pin_memory()
        _lib.osscir_reconstruct(R.handle, c_host, w.n_iters, out)
        R.close()
    plain_s = time.perf_counter() - t0

    rates = {}
    for rate in args.mixed_rates:
        gaps = np.random.default_rng(4000 + rank + int(rate)).exponential(1.0 / rate, size=len(reqs))
        srv = _lib.osscir_server_create(150 << 30, args.slots)
        try:
            t0 = time.perf_counter()
            tickets = []
            for k, (w, c, lam) in enumerate(zip(reqs, counts, lams)):
                target = t0 + float(np.sum(gaps[:k]))
                while time.perf_counter() < target:
                    time.sleep(min(0.0005, max(0.0, target - time.perf_counter())))
                sp = w.spectra
                tickets.append(_lib.osscir_submit(srv, w.geom, sp.s, sp.N, sp.mu, lam, c, w.n_iters))
            lat, ok = [], True
            for t in tickets:
                rc, st = _lib.osscir_poll(srv, t, -1)
                ok = ok and rc == 0
                lat.append(st.latency_ms)
            wall = time.perf_counter() - t0
        finally:
            _lib.osscir_server_destroy(srv)
        lat = np.array(lat)
        rates[str(rate)] = {"recon_per_s": len(reqs) / wall, "iters_per_s": total_iters / wall,
                            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                            "all_ok": bool(ok)}
    mix = {}
    for w in reqs:
        mix[w.geom.n] = mix.get(w.geom.n, 0) + 1
    return {"requests": len(reqs), "image_sizes": {str(k): v for k, v in sorted(mix.items())},
            "views": [min(w.geom.n_views for w in reqs), max(w.geom.n_views for w in reqs)],
            "iterations": total_iters, "slots": args.slots, "budget_GB": 150,
            "plain_recon_per_s": len(reqs) / plain_s, "plain_iters_per_s": total_iters / plain_s,
            "served_by_rate": rates,
            "note": "wall-clock from first submit to last result; context creation included on both sides"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="medium_256", choices=["medium_256", "large_512"],
                    help="the 256x256 headline workload, or the 512x512 solve for profiling")
    ap.add_argument("--e2e", type=int, default=3, help="full reconstructions for the end-to-end rate")
    ap.add_argument("--cpu-iters", type=int, default=3, help="oracle iterations for the CPU baseline")
    ap.add_argument("--cpu-iters-1t", type=int, default=1, help="oracle iterations on one thread (0: skip)")
    ap.add_argument("--served", type=int, default=16, help="requests for the served measurement (0: skip)")
    ap.add_argument("--slots", type=int, default=4, help="server slots")
    ap.add_argument("--batch", type=int, default=64, help="solves in the batched measurement (0: skip)")
    ap.add_argument("--mixed", type=int, default=16, help="mixed requests in the served sweep (0: skip)")
    ap.add_argument("--mixed-rates", type=float, nargs="+", default=[2.0, 5.0, 10.0, 20.0, 50.0],
                    help="Poisson arrival rates of the mixed served sweep, requests/s")
    ap.add_argument("--batch-steps", type=int, default=5, help="timed iterations of the batched measurement")
    ap.add_argument("--rate", type=float, default=1.5, help="Poisson request arrival rate, requests/s")
    ap.add_argument("--five-windows", type=int, default=20,
                    help="timed iterations of the five-window solve (0: skip)")
    ap.add_argument("--split", type=int, nargs="*", default=[2, 4, 8],
                    help="view-split rank counts whose rank-local work is measured (none: skip)")
    ap.add_argument("--split-steps", type=int, default=10, help="timed iterations per split")
    ap.add_argument("--nested", type=int, nargs="*", default=[1, 2, 4, 8],
                    help="iterations per local model for the nested MOCCA leg (none: skip)")
    args = ap.parse_args()
    if args.workload == "large_512":
        global WORKLOAD, WORKLOAD_DESC, LAMBDA, SOLVE_ITERS
        WORKLOAD, WORKLOAD_DESC, LAMBDA, SOLVE_ITERS = LARGE
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
