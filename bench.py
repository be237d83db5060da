"""Benchmark of the fused stream-collide path on the 4096 x 4096 Kolmogorov flow
(D2Q9, SMRT tau_2 = 0.6, tau_3 = tau_4 = 1, FP32 storage of deviations,
g_x = 1e-5 sin(2 pi y / 4096), initial u = that profile plus seeded 1e-4
Gaussian noise).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

One step = one lattice time step over the whole domain (pull-stream, collide,
store) with the FP64 check (mass, momentum, K-step residual) every
--check-every steps inside the timed region.  Prints one JSON line (rank 0).

N > 1 (torchrun) runs one independent replica per GPU (weak scaling); ranks
share nothing but a barrier and a max-reduction of their times.

--impl reference times the FP64 CPU oracle (the reference arm of this
project) on a bounded strip of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lbm_workloads as W  # noqa: E402

METRIC = "MLUPS and % of HBM roofline per lattice"
UNIT = "MLUPS"
WORKLOAD = "kolmogorov_d2q9_smrt_f32_4096x4096"
PROFILE_TRAFFIC = {c: os.path.join(ROOT, "profiles", f"k_step_d2q9_{c.lower()}_f32_traffic.json")
                   for c in ("SMRT", "SMRT_FNEQ", "MRT_RAW")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--n", type=int, default=4096, help="domain edge (4096 = the benchmark workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--min-seconds", type=float, default=2.0,
                    help="kolmogorov: repeat the timed region of --steps steps until about this much device time")
    ap.add_argument("--max-repeats", type=int, default=1000)
    ap.add_argument("--repeats", type=int, default=0, help="kolmogorov: fixed number of timed regions (0: from --min-seconds)")
    ap.add_argument("--workload", default="kolmogorov",
                    choices=["kolmogorov", "tgv", "batch", "surrogate", "precision", "unet", "womersley", "peaks"],
                    help="kolmogorov: the 4096^2 MLUPS line (default); batch: 512 channels to steady "
                         "state; surrogate: learned warm start of obstacle channels vs cold start; "
                         "precision: every storage mode on the Kolmogorov and TGV workloads vs FP64")
    ap.add_argument("--lattice", default="D2Q9", choices=["D2Q9", "D3Q19", "D3Q27"],
                    help="tgv: the 3-D lattice (D2Q9 selects D3Q27)")
    ap.add_argument("--storage", default="F32", choices=["F64", "F32", "F16", "BF16"],
                    help="kolmogorov: storage of the populations (F32 is the benchmark configuration)")
    ap.add_argument("--collision", default="SMRT", choices=["SMRT", "SMRT_FNEQ", "MRT_RAW"],
                    help="kolmogorov: SMRT (the benchmark configuration), SMRT with the force's "
                         "non-equilibrium terms (Eq. Frc, third and fourth), or the appendix's raw-moment MRT")
    ap.add_argument("--tau-bulk", type=float, default=0.0,
                    help="kolmogorov: relaxation time of the trace (bulk) part of the second order (0: tau_2)")
    ap.add_argument("--channels", type=int, default=512, help="batch: number of channels (512: the benchmark)")
    ap.add_argument("--tune-only", action="store_true",
                    help="batch: autotune the tiles, print the chosen shape and stop (a short run for profilers)")
    ap.add_argument("--tgv-n", type=int, default=256)
    ap.add_argument("--tgv-steps", type=int, default=5000)
    ap.add_argument("--kol-steps", type=int, default=10000)
    ap.add_argument("--train-cases", type=int, default=2000)
    ap.add_argument("--held-cases", type=int, default=200)
    ap.add_argument("--train-seconds", type=float, default=180.0)
    ap.add_argument("--tol-train", type=float, default=1e-8)
    ap.add_argument("--plain-stride", type=int, default=16, help="batch: every n-th channel runs the plain solver")
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--max-steps", type=int, default=50_000_000, help="batch: step budget per channel")
    ap.add_argument("--K", type=int, default=1000)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, dist, device) -> float:
    """Max of x over the ranks (x itself with no process group)."""
    if not dist:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank runs the same workload)."""
    return ws * units_per_rank / seconds


# the sources that define the D2Q9 stream-collide kernel and its launch
STEP_SOURCES = ("lbm_device.cuh", "lbm_kernels.cuh", "lbm_internal.h", "lbm_f32x2.cuh", "lbm_inst_d2q9.cu",
                "lbm_step_vec.cuh", "lbm_vec_d2q9_f32.cu")


def kernel_sources_sha():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2212_07494_gb300", "csrc")
    for fn in STEP_SOURCES:
        h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._th = threading.Thread(target=self._read, daemon=True)
            self._th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        if which == 0:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for t, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            rows.append((t, parts))
        mine = [r for r in rows if r[1][1] == str(self.index)]
        if mine:
            rows = mine
        inside = [r for r in rows if self.t0 and self.t1 and self.t0 - 0.15 <= r[0] <= self.t1 + 0.15]
        use = inside if inside else rows
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(p[2]) for _, p in use if p[2].replace(".", "").isdigit()]
        smax = [float(p[3]) for _, p in use if p[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, p in use:
            for k, n in enumerate(names):
                if p[6 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(use), "in_window": bool(inside)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_per_launch(n_nodes, collision="SMRT"):
    """DRAM bytes per launch of the stream-collide kernel from the committed ncu
    summary, scaled to this launch by node count; None when the summary is
    missing or the kernel sources changed since it was taken."""
    path = PROFILE_TRAFFIC.get(collision)
    if path is None or not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("kernel_sources_sha") != kernel_sources_sha():
        return None
    return float(d["dram_bytes_per_node"]) * n_nodes


# ------------------------------------------------------------------ oracle arm
def oracle_strip(n, rows, seed=2212074940, collision="SMRT"):
    """Rows [0, rows) of the n x n Kolmogorov workload as an n x rows periodic
    strip (same per-node work; the oracle cannot hold the full run)."""
    import oracle as O
    wl = W.kolmogorov(n=n, seed=seed) if n <= 1024 else None
    if wl is None:
        # draw only what the strip needs: same profile and noise recipe
        rng = W.SplitMix64(seed)
        y = np.arange(rows, dtype=np.float64)
        prof = 1e-5 * np.sin(2 * np.pi * y / n)
        u0 = rng.normal(2 * rows * n).reshape(2, 1, rows, n) * 1e-4
        u0[0, 0] += prof[:, None]
        g = np.zeros((rows, 2))
        g[:, 0] = prof
        tau = (1.0, 1.0, 0.6, 1.0, 1.0)
    else:
        u0 = wl.u0[:, :, :rows]
        g = wl.g[:rows]
        tau = wl.tau
    coll = getattr(O, collision)
    return O.Sim(O.D2Q9, coll, (n, rows, 1), (1, 1, 1), tau, g=g, force_kind="rows",
                 u0=np.ascontiguousarray(u0))


def cpu_baseline(n, seconds, collision="SMRT"):
    import oracle as O
    cores = O.set_threads(os.cpu_count() or 1)
    rows = max(8, min(n, 256))
    sim = oracle_strip(n, rows, collision=collision)
    sim.step(1)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds and steps < 50:
        sim.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    mlups = n * rows * steps / dt / 1e6
    return {"value": mlups, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} steps of the FP64 oracle on a {n} x {rows} periodic strip of the "
                      f"{n} x {n} Kolmogorov workload ({n * rows * steps} node updates, {dt:.1f} s)"}


def run_reference(args, ws, rank):
    """Reference arm: the FP64 oracle timed on the host cores."""
    if rank != 0:
        return
    import oracle as O
    cores = O.set_threads(os.cpu_count() or 1)
    n = args.n
    # size the strip so that warmup + steps take about two minutes
    probe = oracle_strip(n, 8)
    t0 = time.perf_counter()
    probe.step(2)
    per_row = (time.perf_counter() - t0) / 2 / 8
    total = max(1, args.steps + args.warmup)
    rows = int(max(1, min(n, 120.0 / (total * per_row))))
    sim = oracle_strip(n, rows)
    sim.step(args.warmup)
    t0 = time.perf_counter()
    sim.step(args.steps)
    dt = time.perf_counter() - t0
    mlups = n * rows * args.steps / dt / 1e6
    sample = f"each step: one FP64 oracle time step on a {n} x {rows} periodic strip of the {n} x {n} workload"
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": "D2Q9", "collision": "SMRT", "storage": "F64 (oracle)",
                       "nx": n, "ny": n, "tau": [1.0, 1.0, 0.6, 1.0, 1.0]},
            "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- GPU arm
def workload_spec(args):
    """The workload of the MLUPS line: the 4096^2 Kolmogorov flow on D2Q9
    (configuration 2), or --workload tgv: the 256^3 Taylor-Green vortex at
    Re 1600 plus g_x = 1e-6 on --lattice D3Q27 or D3Q19 (configuration 3)."""
    if args.workload == "tgv":
        lat = args.lattice if args.lattice != "D2Q9" else "D3Q27"
        wl = W.taylor_green_3d(n=args.tgv_n, steps=args.tgv_steps, lattice=lat)
        n = args.tgv_n
        return wl, {"lattice": lat, "shape": (n, n, n), "N": n ** 3, "kind": "uniform",
                    "name": f"tgv3d_{lat.lower()}_{{coll}}_{{st}}_{n}x{n}x{n}",
                    "config": {"nx": n, "ny": n, "nz": n, "Re": 1600, "U0": 0.05, "tau": list(wl.tau),
                               "force": "uniform g_x = 1e-6", "length": "N / 2 pi"}}
    n = args.n
    wl = W.kolmogorov(n=n)
    return wl, {"lattice": "D2Q9", "shape": (n, n, 1), "N": n * n, "kind": "rows",
                "name": "kolmogorov_d2q9_{coll}_{st}_" + f"{n}x{n}",
                "config": {"nx": n, "ny": n, "tau": list(wl.tau), "force": "rows g_x = 1e-5 sin(2 pi y / n)"}}


def make_lattice(P, wl, spec, st, coll, tau_bulk=0.0, torch_stream=None, host_inputs=None):
    g, u0, rho0 = (wl.g, wl.u0, wl.rho0) if host_inputs is None else host_inputs
    return P.Lattice(spec["lattice"], coll, spec["shape"], wl.tau, st, (1, 1, 1), g=g, force_kind=spec["kind"],
                     rho0=rho0, u0=u0, torch_stream=torch_stream, tau_bulk=tau_bulk)


def run_gpu(args, ws, rank, local):
    import torch

    import paper_2212_07494_gb300 as P

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream(device=local)
    st = args.storage
    coll = args.collision
    wl, spec = workload_spec(args)
    n = args.n
    N = spec["N"]
    lat = make_lattice(P, wl, spec, st, coll, args.tau_bulk, torch_stream=stream)
    D, Q, _, bytes_per_node = lat.info()
    steps = max(1, args.steps)
    C = max(1, args.check_every)
    warm = torch.zeros(7, dtype=torch.float64, device=f"cuda:{local}")
    # warm-up: graphs captured, clocks up; its time sizes the repeats
    wsteps = max(args.warmup, 3)
    w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        lat.step(wsteps)
        lat.check_device(warm.data_ptr())
        w0.record(stream)
        lat.step(wsteps)
        w1.record(stream)
    torch.cuda.synchronize()
    est_ms = w0.elapsed_time(w1) / wsteps * steps
    # The timed region (exactly `steps` steps) is repeated until about
    # --min-seconds of device work has run, so that the clock sampler sees the
    # GPU under load.  The FP64 check keeps the workload's cadence (every
    # check_every steps counted over all regions), so the regions together
    # are a run of repeats * steps steps with its checks.
    repeats = int(max(1, min(args.max_repeats, math.ceil(args.min_seconds * 1e3 / max(est_ms, 1e-3)))))
    if args.repeats:
        repeats = args.repeats
    n_checks = repeats * steps // C
    checks = torch.zeros((max(1, n_checks), 7), dtype=torch.float64, device=f"cuda:{local}")
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(repeats)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(repeats)]
    chunk_ev = []          # (start, end, steps) of every run of step launches
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    done = 0               # steps since the timed work began
    k = 0
    for r in range(repeats):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if r == 0:
            sampler.mark(0)
        with torch.cuda.stream(stream):
            e0[r].record(stream)
            left = steps
            while left > 0:
                n_run = min(left, C - done % C)
                es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                es.record(stream)
                lat.step(n_run)
                ee.record(stream)
                chunk_ev.append((es, ee, n_run))
                done += n_run
                left -= n_run
                if done % C == 0:
                    lat.check_device(checks[k].data_ptr())
                    k += 1
            e1[r].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    sampler.mark(1)
    sampler.stop()
    region_ms = [reduce_max(e0[r].elapsed_time(e1[r]), dist, f"cuda:{local}") for r in range(repeats)]
    total_ms = sum(region_ms)
    kern_ms = sum(es.elapsed_time(ee) for es, ee, _ in chunk_ev) / sum(n for _, _, n in chunk_ev)
    bx, npt, layout = lat.launch()
    u_stall = lat.force_resolution()
    ck = checks[:max(1, k)].cpu().numpy()
    finite = bool(np.all(ck[:, 6] == 0)) and bool(np.all(np.isfinite(ck)))
    res = float(math.sqrt(ck[-1, 4]) / (C * math.sqrt(ck[-1, 5]))) if k > 1 and ck[-1, 5] > 0 else None
    mass_drift = float(abs(ck[-1, 0] - ck[0, 0]) / ck[0, 0]) if k > 0 else None
    lat.close()

    all_steps = steps * repeats
    value = job_rate(ws, N * all_steps, total_ms * 1e-3) / 1e6
    peak, peak_kind = measured_peaks()
    algo_bytes = bytes_per_node * N
    achieved = algo_bytes / (kern_ms * 1e-3) / 1e9
    traffic = (traffic_per_launch(N, coll) if st == "F32" and not args.tau_bulk and spec["lattice"] == "D2Q9"
               else None)
    clocks = sampler.summary()
    launches = all_steps + 2 * k   # step kernels, and the moments and finalize kernels per check

    e2e = None
    if not args.no_e2e:
        # the configuration's whole job (its full step count), through the
        # public API from host buffers: creation and the final read-back are
        # part of every real run, so they are timed, not amortised away
        e2e_steps = max(args.kol_steps if spec["lattice"] == "D2Q9" else args.tgv_steps, steps)
        e2e = run_e2e(P, torch, wl, spec, e2e_steps, min(args.check_every, e2e_steps), local, ws, dist, st, coll,
                      args.tau_bulk)

    L = spec["lattice"]
    kname = "SMRT_TRIM" if coll == "SMRT" else coll
    q_bytes = N * Q * {"F64": 8, "F32": 4}.get(st, 2)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": steps,
            "warmup": args.warmup, "ms_per_step": total_ms / all_steps, "higher_is_better": True,
            "repeats": repeats,
            "timing": f"{repeats} timed regions of exactly {steps} steps each, each bracketed by a barrier and a "
                      f"device synchronisation; value and ms_per_step over all of them (per region: median "
                      f"{statistics.median(region_ms) / steps:.5f}, min {min(region_ms) / steps:.5f}, max "
                      f"{max(region_ms) / steps:.5f} ms per step)",
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if st == "F32" else (f"{st.lower()} storage, f32 arithmetic" if st != "F64" else "f64"),
            "data": "synthetic",
            "config": dict({"workload": spec["name"].format(coll=coll.lower(), st=st.lower()) +
                                        (f"_bulk{args.tau_bulk:g}" if args.tau_bulk else ""),
                            "lattice": L, "collision": coll, "storage": st, "tau_bulk": args.tau_bulk or None},
                           **spec["config"],
                           **{"check_every": C, "checks_timed": k,
                              "l2": (f"inputs larger than L2 (two {q_bytes / 1e6:.0f} MB population buffers)"
                                     if q_bytes > 129e6 else
                                     f"two {q_bytes / 1e6:.0f} MB population buffers fit in L2: "
                                     "a small case for profilers, not a bench line"),
                              "replicas": ws}),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": (f"k_step_vec<{L},{kname},{st},{npt}>" if layout
                                    else f"k_step<{L},{kname},{st},{npt}>"),
                         "launch": {"block_x": bx, "nodes_per_thread": npt, "layout": "vector" if layout else "strided"},
                         "bytes_per_launch": algo_bytes,
                         "avg_launch_ms": kern_ms, "peak_source": f"{peak_kind} hbm_gbs (copy)"},
            "gpu_launches": launches, "clocks": clocks,
            "check": {"finite": finite, "mass_drift": mass_drift, "residual_K": res},
            "storage_resolution": {"u_stall": u_stall,
                                   "what": "speed above which one step of the body force rounds away in this "
                                           "storage (lbm_force_resolution)"}}
    if e2e:
        line["e2e"] = e2e
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = (cpu_baseline(n, args.cpu_seconds, coll) if L == "D2Q9"
                                else cpu_baseline_3d(wl, L, args.tgv_n))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_e2e(P, torch, wl, spec, steps, C, local, ws, dist, storage="F32", collision="SMRT", tau_bulk=0.0):
    """Whole job through the public API from pinned host memory: create (H2D of
    the initial fields and the force), run with a host-read residual every C
    steps, read rho and u back (D2H)."""
    pin = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    u0, g, rho0 = pin(wl.u0), pin(wl.g), pin(wl.rho0)
    N = spec["N"]
    D = 2 if spec["lattice"] == "D2Q9" else 3
    rho = torch.empty(N, dtype=torch.float64).pin_memory()
    u = torch.empty(D * N, dtype=torch.float64).pin_memory()
    tot = np.empty(4)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat = make_lattice(P, wl, spec, storage, collision, tau_bulk,
                       host_inputs=(g.numpy(), u0.numpy(), None if rho0 is None else rho0.numpy()))
    r = None
    for _ in range(steps // C):
        r = lat.residual(C)
    P.lbm_moments(lat.h, rho.numpy(), u.numpy(), tot)
    dt = time.perf_counter() - t0
    lat.close()
    dt = reduce_max(dt, dist, f"cuda:{local}")
    h2d = sum(a.numel() * 8 for a in (u0, g, rho0) if a is not None)
    d2h = (rho.numel() + u.numel()) * 8 + (steps // C) * 7 * 8
    return {"value": job_rate(ws, N * steps, dt) / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h / steps, "residual_last": r, "steps": steps,
            "what": f"the whole {steps}-step job: lbm_create from host initial fields and force, lbm_residual "
                    f"every {C} steps, lbm_moments to host"}


def cpu_baseline_3d(wl, lattice, n, steps=3):
    """The FP64 oracle on the host cores: `steps` steps of an n x n x 4
    periodic slab of the Taylor-Green vortex."""
    import oracle as O
    cores = O.set_threads(os.cpu_count() or 1)
    sl = (slice(0, 4), slice(None), slice(None))
    orc = O.Sim(getattr(O, lattice), O.SMRT, (n, n, 4), (1, 1, 1), wl.tau, g=wl.g,
                rho0=np.ascontiguousarray(wl.rho0[sl]), u0=np.ascontiguousarray(wl.u0[(slice(None),) + sl]))
    t0 = time.perf_counter()
    orc.step(steps)
    dt = time.perf_counter() - t0
    return {"value": n * n * 4 * steps / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} FP64 oracle steps on a {n} x {n} x 4 periodic slab of the {n}^3 vortex ({dt:.1f} s)"}


def run_batch(args, ws, rank, local):
    """512 independent force-driven channels (periodic x, walls in y; seeded
    sizes, tau_2 and g_x) run to the K-step residual tol: one persistent
    launch for all channels vs the plain solver (one lattice at a time,
    lbm_residual every K steps) on every plain-stride-th channel, its time
    scaled to all channels.  Equal error: both stop at the same r_K <= tol;
    the final fields of the two are compared channel by channel."""
    import torch

    import paper_2212_07494_gb300 as P

    torch.cuda.set_device(local)
    chans = W.batch_channels(n=args.channels)
    spec = [{"shape": (c.nx, c.ny, 1), "tau": (1.0, 1.0, c.tau2, 1.0, 1.0), "periodic": (1, 0, 1),
             "g": [c.gx, 0.0]} for c in chans]
    b = P.Batch(spec, "SMRT", "F32")
    block, tile, ms_tune = b.autotune(200)
    if args.tune_only:
        b.close()
        if rank == 0:
            print(json.dumps({"metric": "batch tile autotune", "value": ms_tune, "unit": "ms per step",
                              "higher_is_better": False, "config": {"workload": f"batched_channels_{len(spec)}",
                                                                     "block": block, "tile_nodes": tile}}))
        return
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    sampler.mark(0)
    t0 = time.perf_counter()
    status, steps, st, r = b.run_to_steady(args.tol, args.K, max_steps=args.max_steps)
    t_batch = time.perf_counter() - t0
    print(f"batch: {t_batch:.1f} s, status {status}, steps max {int(steps.max())}", file=sys.stderr, flush=True)
    sampler.mark(1)
    sampler.stop()
    clocks = sampler.summary()
    nodes = np.array([c.nx * c.ny for c in chans], np.float64)
    updates = float((steps * nodes).sum())
    idx = list(range(0, len(chans), max(1, args.plain_stride)))
    t_plain = 0.0
    errs, plain_steps = [], []
    for i in idx:
        sp = spec[i]
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        lat = P.Lattice("D2Q9", "SMRT", sp["shape"], sp["tau"], "F32", sp["periodic"], g=sp["g"])
        n = 0
        while True:
            rr = lat.residual(args.K)
            n += args.K
            if rr <= args.tol or n >= args.max_steps:
                break
        _, u_plain, _ = lat.moments()
        t_plain += time.perf_counter() - t1
        print(f"plain channel {i}: {n} steps, r {rr:.3g}, {time.perf_counter() - t1:.1f} s", file=sys.stderr, flush=True)
        lat.close()
        plain_steps.append(n)
        _, u_b = b.moments(i)
        errs.append(float(np.linalg.norm(u_b - u_plain) / np.linalg.norm(u_plain)))
    scale = len(chans) / len(idx)
    t_plain_est = t_plain * scale
    # distance of each steady profile from the no-slip Poiseuille parabola
    # (mean over x), an accuracy statement independent of both solvers
    para = []
    for i, c in enumerate(chans):
        _, u = b.moments(i)
        nu = (c.tau2 - 0.5) / 3.0
        y = np.arange(c.ny) + 0.5
        ua = c.gx / (2 * nu) * (y * (c.ny - y))
        para.append(float(np.linalg.norm(u[0, 0].mean(axis=1) - ua) / np.linalg.norm(ua)))
    b.close()
    peak, peak_kind = measured_peaks()
    line = {"metric": "wall time to steady state vs plain at equal error", "value": t_batch, "unit": "s",
            "n_gpus": 1, "steps": int(steps.max()), "warmup": 0, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched_channels_d2q9_smrt_f32_512", "channels": len(chans),
                       "nx": "U[32,512]", "ny": "U[16,256]", "tau2": "U[0.55,1.5]", "tau3": 1.0, "tau4": 1.0,
                       "gx": "log-U[1e-7,1e-5]", "redraws": int(sum(c.redraws for c in chans)),
                       "seed": 2212074941, "tol": args.tol, "K": args.K, "tiles": {"block": block, "tile_nodes": tile}},
            "batch": {"seconds": t_batch, "node_updates": updates, "mlups": updates / t_batch / 1e6,
                      "hbm_gbs": updates * 72 / t_batch / 1e9, "hbm_frac": updates * 72 / t_batch / 1e9 / peak,
                      "converged": int((st == 0).sum()), "not_converged": int((st == 1).sum()),
                      "unstable": int((st == -4).sum()), "status": int(status),
                      "steps_min": int(steps.min()), "steps_median": float(np.median(steps)),
                      "steps_max": int(steps.max())},
            "plain": {"seconds_measured": t_plain, "channels_measured": len(idx), "seconds_extrapolated": t_plain_est,
                      "how": f"every {args.plain_stride}th channel run alone (lbm_create, lbm_residual every K), "
                             f"time x {scale:g}"},
            "speedup_vs_plain": t_plain_est / t_batch, "clocks": clocks,
            "equal_error": {"max_rel_l2_batch_vs_plain": max(errs), "plain_vs_batch_steps_diff_max":
                            int(max(abs(int(steps[i]) - 1 - p) for i, p in zip(idx, plain_steps))),
                            "rel_l2_vs_noslip_parabola_median": float(np.median(para)),
                            "rel_l2_vs_noslip_parabola_max": float(max(para))}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def obstacle_cases(seed, n, nx=256, ny=128):
    """n seeded obstacle channels (per-case seeds drawn from one stream)."""
    rng = W.SplitMix64(seed)
    return [W.obstacle_channel(int(rng.next_u64(1)[0] & 0x7FFFFFFFFFFF), nx=nx, ny=ny) for _ in range(n)]


def run_surrogate(args, ws, rank, local):
    """256 x 128 channels with 1-4 seeded circular obstacles: 2000 steady
    fields from the batched solver train the U-Net; on 200 held-out cases the
    predicted (rho, u) start runs to r_K <= tol, against cold starts of the
    same cases (both batched), and a plain sequential cold solver on every
    10th held-out case (scaled to all)."""
    import torch

    import paper_2212_07494_gb300 as P
    import paper_2212_07494_gb300.surrogate as S

    torch.cuda.set_device(local)
    H, Wd = 128, 256
    tol, K, max_steps = args.tol, args.K, 5_000_000
    train = obstacle_cases(2212074942, args.train_cases)
    held = obstacle_cases(2212074943, args.held_cases)
    t0 = time.perf_counter()
    secs_d, steps_d, st_d, r_d, b = S.solve(train, args.tol_train, K, max_steps)
    ok = np.where(st_d == 0)[0]
    X = np.stack([S.features(train[k][0], train[k][1], train[k][2]) for k in ok])
    steady = [b.moments(int(k)) for k in ok]
    alpha = S.prior_scale([train[k] for k in ok], steady)
    Y = np.stack([S.targets(*steady[j], train[k][1], train[k][2], train[k][0], alpha) for j, k in enumerate(ok)])
    del steady
    M = np.stack([1.0 - train[k][0][0] for k in ok]).astype(np.float32)
    b.close()
    Xf, Yf, Mf = S.mirror(X, Y, M)
    X, Y, M = np.concatenate([X, Xf]), np.concatenate([Y, Yf]), np.concatenate([M, Mf])
    del Xf, Yf, Mf
    t_data = time.perf_counter() - t0
    sur = S.Surrogate(H, Wd, batch=8, alpha=alpha)
    losses, t_train, nsteps = sur.train(X, Y, M, epochs=1000, lr=1e-3, seconds=args.train_seconds)
    flops = S.train_flops_per_sample(H, Wd) * 8 * nsteps
    # held-out: cold (batched), warm (batched, inference included)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    sampler.mark(0)
    secs_c, steps_c, st_c, r_c, bc = S.solve(held, tol, K, max_steps)
    cold = S.final_fields(bc, len(held))
    bc.close()
    Xh = np.stack([S.features(s, t2, g) for s, t2, g in held])
    Yh = sur.predict(Xh)
    pred_err = [float(np.linalg.norm(S.fields(Yh[k], *held[k], alpha=alpha)[1] - cold[k][1]) /
                      np.linalg.norm(cold[k][1])) for k in range(len(held))]
    lub_err = [float(np.linalg.norm(S.fields(0 * Yh[k], *held[k], alpha=alpha)[1] - cold[k][1]) /
                     np.linalg.norm(cold[k][1])) for k in range(len(held))]
    # the fit on training cases, for comparison with the held-out error
    tr = [int(k) for k in ok[:50]]
    Yt = sur.predict(np.stack([S.features(*train[k]) for k in tr]))
    train_err = []
    for j, k in enumerate(tr):
        ut = S.fields(Y[j], *train[k], alpha=alpha)[1]
        train_err.append(float(np.linalg.norm(S.fields(Yt[j], *train[k], alpha=alpha)[1] - ut) / np.linalg.norm(ut)))
    secs_l, steps_l, st_l, _, _, fallbacks_l = S.warm_start(None, held, tol, K, max_steps)
    secs_w, steps_w, st_w, warm, t_inf, fallbacks = S.warm_start(sur, held, tol, K, max_steps)
    sampler.mark(1)
    sampler.stop()
    clocks = sampler.summary()
    diff = [float(np.linalg.norm(warm[k][1] - cold[k][1]) / np.linalg.norm(cold[k][1])) for k in range(len(held))]
    # plain sequential cold start on a subset
    t_plain, n_plain = 0.0, 0
    for k in range(0, len(held), 10):
        s_, t2, g = held[k]
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        lat = P.Lattice("D2Q9", "SMRT", (Wd, H, 1), (1, 1, t2, 1, 1), "F32", (1, 0, 1), g=[g, 0.0], solid=s_)
        n = 0
        while n < max_steps:
            n += K
            if lat.residual(K) <= tol:
                break
        lat.close()
        t_plain += time.perf_counter() - t1
        n_plain += 1
    t_plain_est = t_plain * len(held) / max(1, n_plain)
    sur.close()
    peak_tf = 1698.0
    try:
        peak_tf = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops_sustained"])
    except Exception:
        pass
    line = {"metric": "wall time to steady state, surrogate warm start vs cold start at equal error",
            "value": secs_w, "unit": "s", "n_gpus": 1, "steps": int(np.max(steps_w)), "warmup": 0,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (solver), bf16 (network)",
            "data": "synthetic",
            "config": {"workload": "obstacle_channels_d2q9_smrt_f32_256x128_unet_bf16", "H": H, "W": Wd,
                       "train_cases": int(len(ok)), "held_out": len(held), "tol": tol, "tol_train": args.tol_train,
                       "K": K, "seeds": [2212074942, 2212074943],
                       "unet": "4 levels, widths 32/64/128/256, periodic in x, 5 inputs incl. a lubrication estimate",
                       "augmentation": "mirror y -> H - 1 - y", "lubrication_scale": list(alpha)},
            "cold": {"seconds": secs_c, "steps_mean": float(np.mean(steps_c)), "steps_max": int(np.max(steps_c)),
                     "converged": int((st_c == 0).sum())},
            "warm": {"seconds_incl_inference": secs_w, "inference_seconds": t_inf,
                     "steps_mean": float(np.mean(steps_w)), "steps_max": int(np.max(steps_w)),
                     "converged": int((st_w == 0).sum()),
                     "fallbacks_to_cold": int(fallbacks)},
            "lubrication_only": {"seconds": secs_l, "steps_mean": float(np.mean(steps_l)),
                                 "converged": int((st_l == 0).sum()), "fallbacks_to_cold": int(fallbacks_l),
                                 "what": "warm start from the lubrication estimate the network corrects"},
            "speedup_vs_cold_batched": secs_c / secs_w, "clocks": clocks,
            "plain_cold": {"seconds_extrapolated": t_plain_est, "cases_measured": n_plain,
                           "how": "every 10th held-out case alone (lbm_create, lbm_residual every K), time scaled"},
            "speedup_vs_plain_cold": t_plain_est / secs_w,
            "steps_saved_frac_mean": float(1.0 - np.mean(steps_w) / np.mean(steps_c)),
            "steps_saved_frac_median_per_case": float(np.median(1.0 - steps_w / steps_c)),
            "equal_error": {"rel_l2_warm_vs_cold_median": float(np.median(diff)), "rel_l2_warm_vs_cold_max": max(diff),
                            "prediction_rel_l2_u_median": float(np.median(pred_err)),
                            "lubrication_rel_l2_u_median": float(np.median(lub_err)),
                            "train_fit_rel_l2_u_median": float(np.median(train_err)),
                            "steps_ratio_warm_over_cold_quantiles": [float(q) for q in
                                                                     np.quantile(steps_w / steps_c, [0.1, 0.5, 0.9])]},
            "training": {"data_seconds": t_data, "train_seconds": t_train, "steps": nsteps, "batch": 8,
                         "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1], "epochs": len(losses),
                         "tflops": flops / t_train / 1e12, "frac_of_bf16_sustained": flops / t_train / 1e12 / peak_tf,
                         "flops_per_sample": S.train_flops_per_sample(H, Wd)}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_unet(args, ws, rank, local):
    """Training steps of the surrogate network alone (the warm start's 128 x 256
    channels, batch 8, eight input channels, periodic along x): forward, loss,
    backward and Adam, all in the library's kernels, on seeded synthetic
    tensors; TFLOP/s against the measured sustained BF16 peak."""
    import torch

    import paper_2212_07494_gb300 as P
    import paper_2212_07494_gb300.surrogate as S

    torch.cuda.set_device(local)
    H, Wd, B = 128, 256, 8
    stream = torch.cuda.Stream(device=local)
    g = torch.Generator(device=f"cuda:{local}")
    g.manual_seed(2212074945)
    with torch.cuda.stream(stream):
        net = P.UNet(H, Wd, B, stream.cuda_stream, cin=S.NF, periodic_x=True)
        net.set_params(S.init_params(S.ARCH, 2212074946))
        x = torch.randn(B, H, Wd, S.NF, device=f"cuda:{local}", generator=g)
        t = torch.randn(B, H, Wd, 3, device=f"cuda:{local}", generator=g)
        m = torch.ones(B, H, Wd, device=f"cuda:{local}")
        ld = torch.zeros(1, dtype=torch.float64, device=f"cuda:{local}")
        scale = 1.0 / (3 * B * H * Wd)
        for _ in range(max(args.warmup, 3)):
            net.train_step(x.data_ptr(), t.data_ptr(), m.data_ptr(), B, scale, 1e-4, ld.data_ptr())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.4)
        sampler.mark(0)
        e0.record(stream)
        for _ in range(args.steps):
            net.train_step(x.data_ptr(), t.data_ptr(), m.data_ptr(), B, scale, 1e-4, ld.data_ptr())
        e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark(1)
    sampler.stop()
    net.params()   # a synchronising call: reports a tensor-core wait that expired
    ms = e0.elapsed_time(e1) / args.steps
    flops = S.train_flops_per_sample(H, Wd) * B
    tf = flops / (ms * 1e-3) / 1e12
    peak = 1695.8
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops_sustained"])
    except Exception:
        pass
    net.close()
    line = {"metric": "surrogate training throughput", "value": tf, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
            "config": {"workload": "unet_train_step_128x256_batch8", "H": H, "W": Wd, "batch": B, "cin": S.NF,
                       "flops_per_step": flops},
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                         "traffic": None, "peak_source": "measured bf16_tflops_sustained"},
            "clocks": sampler.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_precision(args, ws, rank, local):
    """Storage precision: the 4096^2 Kolmogorov flow (D2Q9 SMRT, 10000 steps)
    and the 256^3 Taylor-Green vortex (D3Q27 and D3Q19 SMRT, Re 1600, 5000 steps) in
    FP64, FP32, FP16 and BF16 storage.  Errors are relative L2 of u against
    the FP64 run (the GPU FP64 path, which matches the FP64 oracle to 1e-12 in
    the parity tests; the oracle itself cannot run these sizes)."""
    import torch

    import paper_2212_07494_gb300 as P

    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(device=local)
    peak, _ = measured_peaks()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    sampler.mark(0)

    def run(label, make, steps):
        out, ref = {}, None
        for st in ["F64", "F32", "F16", "BF16"]:
            lat = make(st)
            with torch.cuda.stream(stream):
                bx, npt, _ = lat.autotune(5)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                lat.step(steps)
                e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            D, Q, _, bpn = lat.info()
            rho, u, tot = lat.moments()
            N = rho.size
            ach = N * bpn / ms / 1e6
            rec = {"mlups": N / ms / 1e3, "gbs": ach, "hbm_frac": ach / peak,
                   "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                "traffic": None},
                   "ms_per_step": ms, "launch": list(lat.launch()), "finite": bool(np.all(np.isfinite(u))),
                   "u_stall": lat.force_resolution(), "u_max": float(np.abs(u).max())}
            if ref is None:
                ref = u
            else:
                rec["rel_l2_u_vs_f64"] = float(np.linalg.norm(u - ref) / np.linalg.norm(ref))
            out[st] = rec
            lat.close()
        return out

    wl = W.kolmogorov(n=args.n, steps=args.kol_steps)
    kol = run("kolmogorov", lambda st: P.Lattice("D2Q9", "SMRT", wl.shape, wl.tau, st, wl.periodic, g=wl.g,
                                                 force_kind="rows", u0=wl.u0, torch_stream=stream), wl.steps)
    del wl
    tg = W.taylor_green_3d(n=args.tgv_n, steps=args.tgv_steps)
    tgv = run("tgv", lambda st: P.Lattice("D3Q27", "SMRT", tg.shape, tg.tau, st, tg.periodic, g=tg.g,
                                          rho0=tg.rho0, u0=tg.u0, torch_stream=stream), tg.steps)
    tgv19 = run("tgv19", lambda st: P.Lattice("D3Q19", "SMRT", tg.shape, tg.tau, st, tg.periodic, g=tg.g,
                                              rho0=tg.rho0, u0=tg.u0, torch_stream=stream), tg.steps)
    sampler.mark(1)
    sampler.stop()
    clocks = sampler.summary()
    # the FP64 oracle on the host cores, as a baseline per 3-D lattice: 3 steps on
    # a 256 x 256 x 4 periodic slab of the same vortex
    import oracle as O
    cores = O.set_threads(os.cpu_count() or 1)
    cpu = {}
    for name, lat in (("D3Q27", O.D3Q27), ("D3Q19", O.D3Q19)):
        sl = (slice(0, 4), slice(None), slice(None))
        orc = O.Sim(lat, O.SMRT, (args.tgv_n, args.tgv_n, 4), (1, 1, 1), tg.tau, g=tg.g,
                    rho0=np.ascontiguousarray(tg.rho0[sl]), u0=np.ascontiguousarray(tg.u0[(slice(None),) + sl]))
        t0 = time.perf_counter()
        orc.step(3)
        dt = time.perf_counter() - t0
        cpu[name] = {"value": args.tgv_n * args.tgv_n * 4 * 3 / dt / 1e6, "unit": "MLUPS", "cores": cores,
                     "kind": "oracle", "sample": f"3 FP64 oracle steps on a {args.tgv_n} x {args.tgv_n} x 4 periodic slab"}
    line = {"metric": "MLUPS and % of HBM roofline per lattice, with velocity error vs FP64 per storage mode",
            "value": tgv["F16"]["mlups"], "unit": "MLUPS", "n_gpus": 1, "steps": args.tgv_steps, "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 arithmetic",
            "data": "synthetic",
            "config": {"workload": "precision_modes", "kolmogorov": {"n": args.n, "steps": args.kol_steps},
                       "tgv3d": {"n": args.tgv_n, "steps": args.tgv_steps, "Re": 1600, "U0": 0.05,
                                 "tau2": tg.tau[2], "lattice": "D3Q27"}},
            "kolmogorov_d2q9_smrt": kol, "tgv_d3q27_smrt": tgv, "tgv_d3q19_smrt": tgv19, "peak_gbs": peak,
            "clocks": clocks,
            "cpu_baseline_3d": cpu}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_peaks(args, ws, rank, local):
    """The CUDA-core FMA peaks (FP32, FP64) of this GPU with sampled clocks:
    the ceilings of the 2-byte and FP64 step kernels (lbm_alu_peak)."""
    import torch

    import paper_2212_07494_gb300 as P

    torch.cuda.set_device(local)
    out = {}
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    sampler.mark(0)
    for prec, iters in (("F32", 1 << 21), ("F64", 1 << 15)):
        runs = [P.lbm_alu_peak(prec, iters) for _ in range(5)]
        best = max(r[0] for r in runs)
        out[prec] = {"tflops": best, "tflops_median": statistics.median(r[0] for r in runs),
                     "ms_per_launch": statistics.median(r[1] for r in runs), "launches": len(runs),
                     "fmas_per_launch": 8 * iters * 256 * 8 * torch.cuda.get_device_properties(local).multi_processor_count}
    sampler.mark(1)
    sampler.stop()
    clocks = sampler.summary()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clocks.get("sm_mhz") or 2070.0
    nominal32 = sms * 128 * 2 * mhz * 1e6 / 1e12
    line = {"metric": "CUDA-core FMA peak", "value": out["F32"]["tflops"], "unit": "TFLOP/s", "n_gpus": 1,
            "steps": 5, "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 and f64", "data": "synthetic",
            "config": {"workload": "fma_chains", "chains_per_thread": 8, "threads": f"{sms} SMs x 8 x 256"},
            "fp32": out["F32"], "fp64": out["F64"], "clocks": clocks, "sms": sms,
            "fp32_nominal_at_clock": nominal32,
            "issue_rate_warp_instr_per_s": out["F32"]["tflops"] * 1e12 / 2 / 32,
            "what": "FP32 FMAs per second / 32 = warp instructions issued per second at one FFMA per lane"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def womersley_analytic(y, t, A, om, nu, Lh, nmax=200):
    """Sec. III.B: the periodic Womersley profile plus the start-up transient
    of the diffusion equation from rest (even no-slip modes)."""
    k = (1 + 1j) * math.sqrt(om / (2 * nu))

    def periodic(yy, tt):
        return np.real(1j * A / om * (1 - np.cosh(k * yy) / np.cosh(k * Lh)) * np.exp(1j * om * tt))

    yq = np.linspace(-Lh, Lh, 40001)
    u0 = -periodic(yq, 0.0)
    out = periodic(y, t)
    for m in range(nmax):
        km = (2 * m + 1) * math.pi / (2 * Lh)
        bm = np.trapezoid(u0 * np.cos(km * yq), yq) / Lh
        out = out + bm * np.cos(km * y) * math.exp(-nu * km * km * t)
    return out


def run_womersley(args, ws, rank, local):
    """Sec. III.B, the Womersley channel: 50 x 200 nodes, periodic x,
    plates in y, T = 1200 steps, nu = 0.1, A_p = 1e-4, 20 periods, D2Q9 SMRT
    FP32.  The oscillating force comes from the device-side schedule inside
    the 64-step graphs; the same run with a host lbm_set_force before every
    step (public API) is timed beside it."""
    import torch

    import paper_2212_07494_gb300 as P

    torch.cuda.set_device(local)
    nx, ny, T, nu, A, periods = 50, 200, 1200, 0.1, 1e-4, 20
    tau = (1.0, 1.0, 3 * nu + 0.5, 1.0, 1.0)
    om = 2 * math.pi / T
    tab = np.stack([-A * np.cos(om * np.arange(T)), np.zeros(T)], axis=1)
    stream = torch.cuda.Stream(device=local)
    # created with g(0), as the per-step run is: the initial state carries -F/2 (C-8)
    lat = P.Lattice("D2Q9", "SMRT", (nx, ny, 1), tau, "F32", (1, 0, 1), g=tab[0], torch_stream=stream)
    lat.set_force_schedule(tab)
    with torch.cuda.stream(stream):
        lat.step(T)                                   # warm-up: one period, graphs captured
    torch.cuda.synchronize()
    steps = periods * T
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    torch.cuda.synchronize()
    sampler.mark(0)
    with torch.cuda.stream(stream):
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark(1)
    sampler.stop()
    ms = e0.elapsed_time(e1)
    t_end = T + steps
    u = lat.moments()[1]
    y = np.arange(ny) + 0.5 - ny / 2
    ua = womersley_analytic(y, t_end, A, om, nu, ny / 2)
    err = float(np.abs(u[0, 0, :, 0] - ua).max() / (A / om))
    f_sched = lat.populations()
    lat.close()
    # the same steps with a host call per step
    ref = P.Lattice("D2Q9", "SMRT", (nx, ny, 1), tau, "F32", (1, 0, 1), g=tab[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for t in range(t_end):
        ref.set_force(tab[t % T])
        ref.step(1)
    torch.cuda.synchronize()
    host_s = time.perf_counter() - t0
    same = bool(np.array_equal(ref.populations(), f_sched))
    ref.close()
    N = nx * ny
    peak, peak_kind = measured_peaks()
    achieved = 72 * N * steps / (ms * 1e-3) / 1e9
    line = {"metric": "Womersley channel MLUPS with the force schedule in step graphs", "value": N * steps / (ms * 1e-3) / 1e6,
            "unit": "MLUPS", "n_gpus": 1, "steps": steps, "warmup": T, "ms_per_step": ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "womersley_d2q9_smrt_f32_50x200", "nx": nx, "ny": ny, "T": T, "nu": nu, "A_p": A,
                       "periods": periods, "walls": "halfway bounce-back in y", "l2": "L2-resident (1.4 MB of populations)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "note": "10,000 nodes per step: launch latency bounds it, not HBM",
                         "peak_source": f"{peak_kind} hbm_gbs (copy)"},
            "gpu_launches": 2 * steps + steps // 64,   # k_step and the force update per step, a counter advance per 64
            "clocks": sampler.summary(),
            "per_step_set_force": {"seconds": host_s, "steps": t_end, "mlups": N * t_end / host_s / 1e6,
                                   "us_per_step": host_s / t_end * 1e6},
            "speedup_vs_per_step_set_force": (host_s / t_end) / (ms * 1e-3 / steps),
            "schedule_equals_per_step_bitwise": same,
            "max_err_vs_analytic_over_amplitude": err}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.gpus != ws and ws != 1:
        print(f"warning: --gpus {args.gpus} but WORLD_SIZE {ws}", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "batch":
        run_batch(args, ws, rank, local)
    elif args.workload == "surrogate":
        run_surrogate(args, ws, rank, local)
    elif args.workload == "precision":
        run_precision(args, ws, rank, local)
    elif args.workload == "unet":
        run_unet(args, ws, rank, local)
    elif args.workload == "womersley":
        run_womersley(args, ws, rank, local)
    elif args.workload == "peaks":
        run_peaks(args, ws, rank, local)
    else:
        run_gpu(args, ws, rank, local)


if __name__ == "__main__":
    main()
