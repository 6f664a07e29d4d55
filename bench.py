#!/usr/bin/env python3
"""Throughput of the fused PML + characteristic-BC lattice Boltzmann step on GB300.

Workload (one step = one pass of the whole hot path over the grid): 2048^2 bulk + 32-node PML
(cubic sigma, sigma_max 0.1) + characteristic outer BC (east CBC relax with beta 0.3, the other
edges PNR-LODI), D2Q37, tau 0.55, isentropic vortex (R 20, Mach 0.05) in a Mach 0.3 mean flow.
Synthetic seeded inputs; populations resident in HBM (1.33 GB FP32 / 2.65 GB FP64 working set,
larger than the 129 MB L2, so no flush between steps).

value   = million fluid-node updates per second (MLUPS, F = (2048 + 64)^2 nodes per step), summed
          over ranks, FP32-deviation storage (the throughput path), device time from CUDA events
          on the launching stream, max over ranks.
e2e     = the same metric through the C ABI with host buffers: lbm_init from pinned host fields,
          K steps, lbm_moments back to host, wall-clock.
Multi-GPU: every rank runs an independent replica (instances do not exchange data), so
scaling is weak and there is no data-path collective.

--impl reference times the CPU oracle (numpy, FP64) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "vortex2048_w32_nrbc_d2q37"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="CPU-baseline budget of the oracle sample (0 skips it)")
    ap.add_argument("--window", type=int, default=150,
                    help="steps per fresh solve; the printed PML stays finite on this workload "
                         "for about 300 steps (tau 0.55) and the FP32 path within 1e-5 of the "
                         "FP64 path for about 150, so timed steps run in windows of 150")
    ap.add_argument("--long", type=int, default=1,
                    help="also measure how many steps the workload survives with the printed "
                         "and the link-integrated PML gradient (1) or not (0)")
    ap.add_argument("--variants", type=int, default=1,
                    help="also time the other stencils and PML / boundary variants (1) or not (0)")
    ap.add_argument("--serving", type=int, default=1,
                    help="also run the batched sweep and the serving stream (0 skips)")
    ap.add_argument("--size", type=int, default=2048,
                    help="bulk edge (2048 = the workload; smaller sizes for profiler captures)")
    ap.add_argument("--pml-grad", default="central", choices=("central", "link"),
                    help="PML gradient of the headline workload: the printed differences (the "
                         "workload as stated) or the link-integrated option (its kernels' "
                         "timings and profiles)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("lbm_device.cuh", "ops.cuh", "stencils.cuh"):
        with open(os.path.join(ROOT, "paper_2504_20169_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(name):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on this source."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip().strip("-* ")] = v.strip()
        if kv.get("kernel_source_sha256") != kernel_source_sha():
            return None
        return float(kv["dram_bytes_per_launch"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.rows, self.proc = [], None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def wait_first(self, timeout=15.0):
        """Block until the sampler has printed its first row (nvidia-smi start-up can stall
        the driver for seconds; that must not land inside the timed region)."""
        t0 = time.time()
        while self.proc and not self.rows and time.time() - t0 < timeout:
            time.sleep(0.05)
        time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        if not sm:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in self.rows if len(r) > 8 for n, v in zip(names, r[5:9])
                          if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(self.rows[0][2]),
                "samples": len(sm), "reasons": reasons}


def max_over_ranks(x, dist=None, device=None):
    """Max of a per-rank float over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample(seconds, n_bulk=512, steps=None):
    """The oracle as it stands on a bounded sample of the workload: the same physics and BC mix
    on an n_bulk^2 bulk (PML 32), stepped `steps` times (at most, when `seconds` > 0 also bounds
    the time) or, without `steps`, until about `seconds` have passed."""
    import workloads as wl
    from oracle import OracleLBM
    c = wl.vortex_2048(n=n_bulk, W=32)
    o = OracleLBM(c.nx, c.ny, c.W, c.tau, c.sigma_max, c.sigma_power, c.bc,
                  nrbc_edges=c.nrbc_edges, beta=c.beta, mean=c.mean)
    o.init(*c.fields())
    t0 = time.perf_counter()
    n = 0
    while True:
        if steps is not None:
            if n >= steps or (seconds > 0 and n >= 1 and time.perf_counter() - t0 >= seconds):
                break
        elif n >= 2 and time.perf_counter() - t0 >= seconds:
            break
        o.step(1)
        n += 1
    dt = time.perf_counter() - t0
    sites = (c.nx + 2 * c.W) * (c.ny + 2 * c.W)
    return {"value": sites * n / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"numpy FP64 oracle, {n_bulk}^2 bulk + PML 32, same BC/physics, {n} steps, "
                      f"{dt:.1f} s, single thread"}


def _config1_oracle(_):
    """Config 1 in full with the oracle (64^2 bulk + PML 8, ZG, pulse, 200 steps): seconds."""
    import workloads as wl
    from oracle import OracleLBM
    c = wl.pulse_64()
    o = OracleLBM(c.nx, c.ny, c.W, c.tau, c.sigma_max, c.sigma_power, c.bc)
    o.init(*c.fields())
    t0 = time.perf_counter()
    o.step(c.steps)
    return time.perf_counter() - t0


def config1_cpu():
    """The oracle on config 1 in full, single-threaded and as one process per host core
    (spawned, so no CUDA state is inherited)."""
    import multiprocessing as mp
    import platform
    n = os.cpu_count() or 1
    nodes = (64 + 16) ** 2 * 200
    one = _config1_oracle(0)
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(n) as pool:
        pool.map(_config1_oracle, range(n))
    wall = time.perf_counter() - t0
    model = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"workload": "pulse64_w8_zg (64^2 bulk + PML 8, ZG, 200 steps, FP64)",
            "single_thread_mlups": round(nodes / one / 1e6, 3), "single_thread_s": round(one, 2),
            "all_cores_mlups": round(n * nodes / wall / 1e6, 3), "all_cores_wall_s": round(wall, 2),
            "cores": n, "cpu": model,
            "note": "one oracle process per core (process start-up included in the wall time)"}


def run_reference(args, ws, rank):
    """The oracle as the reference arm: one warm-up step, then up to K steps of the oracle on a
    128^2-bulk sample of the workload (PML 32, same BC and physics), bounded to about 90 s so any
    K ends within a few minutes; the rate is nodes x steps done / time."""
    if rank != 0:
        return
    oracle_sample(0, n_bulk=128, steps=1)
    base = oracle_sample(90.0, n_bulk=128, steps=max(1, args.steps))
    line = {"metric": "MLUPS", "value": base["value"], "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": {"workload": WORKLOAD, "sample": base["sample"]},
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_run(Solver, c, fields, precision, steps, warmup, dev, window, prof_steps=0):
    """Headline region: `steps` steps as repeated fresh solves of at most `window` steps (the
    state is re-initialized, untimed, between windows), each step a CUDA-graph replay with one
    event pair on the launching stream. Then a profiled window launched directly with CUDA
    events around every kernel class (the interior kernel's live duration)."""
    import torch
    s = Solver(c.nx, c.ny, c.W, c.tau, c.sigma_max, c.sigma_power, c.bc, 37, c.nrbc_edges,
               c.beta, c.mean, precision=precision, pml_grad=c.pml_grad)
    s.init(*fields)
    s.step(warmup)
    s.sync()
    st = torch.cuda.current_stream()
    per, total, done = [], 0.0, 0
    torch.cuda.synchronize()
    clocks = Clocks(dev)
    clocks.wait_first()
    while done < steps:
        n = min(window, steps - done)
        s.init(*fields)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
        ev[0].record(st)
        for k in range(n):
            s.step(1)
            ev[k + 1].record(st)
        torch.cuda.synchronize()
        per += [ev[k].elapsed_time(ev[k + 1]) for k in range(n)]
        total += ev[0].elapsed_time(ev[n])
        done += n
    ck = clocks.stop()
    prof = None
    if prof_steps:
        s.init(*fields)
        s.profile_enable(prof_steps)
        s.step(prof_steps)
        prof = s.profile_read()
    tot = s.reduce()
    s.close()
    return total, per, prof, ck, tot


def variant_runs(size, window, warmup):
    """Step time of the largest single-GPU case (8192^2 + PML 64) and of the other built
    variants on the 2048^2-class grid (FP32 deviation storage, one CUDA-graph replay per step,
    CUDA events around the window): the D2Q17 / D2Q9 stencils, an
    outlet-heavy per-edge PML (W 8 / 32 / 8 / 8), the split sigma_x != sigma_y form, the
    Appendix PML source (terms I + II + III) and a periodic y axis with open x edges."""
    import torch
    import workloads as wl
    from paper_2504_20169_gb300 import Solver
    c = wl.vortex_2048(n=size)
    base = dict(sigma_max=c.sigma_max, sigma_power=c.sigma_power, bc=c.bc, q=37,
                nrbc_edges=c.nrbc_edges, beta=c.beta, mean=c.mean)
    runs = {
        "D2Q17": dict(base, q=17),
        "D2Q9": dict(base, q=9),
        "per_edge_8_32_8_8": dict(base, pml_widths=(8, 32, 8, 8)),
        "split_sigma": dict(base, sigma_split=True),
        "pml_source_I_II_III": dict(base, pml_source=7),
        "periodic_y_W32_x": dict(base, periodic_y=True, nrbc_edges=(0, 1, 0, 0)),
    }
    out = {}
    # the largest single-GPU case: 8192^2 + PML 64 (about 20 GB of FP32 populations)
    cs = wl.stress_8192()
    with Solver(cs.nx, cs.ny, cs.W, cs.tau, cs.sigma_max, cs.sigma_power, cs.bc, 37,
                cs.nrbc_edges, cs.beta, cs.mean, precision="fp32dev") as s:
        fields = cs.fields()
        s.init(*fields)
        s.step(warmup)
        s.init(*fields)
        del fields
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        nst = 50
        ev[0].record(torch.cuda.current_stream())
        s.step(nst)
        ev[1].record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / nst
        nodes = s.Lx * s.Ly
        # algorithmic bytes: interior 2 x 37 x 4 B, frame (PML + inner ring) 4 x 37 x 4 B,
        # boundary layers outside F 37 x 4 B
        fd = cs.W + 1
        frame = 2 * fd * s.Lx + 2 * (s.Ly - 2 * fd) * fd
        band = 2 * 3 * (s.Lx + 6) + 2 * 3 * s.Ly
        alg = (nodes - frame) * 296 + frame * 592 + band * 148
        out["stress8192_w64"] = finite_or_unmeasured({
            "ms_per_step": round(ms, 4), "mlups": round(nodes / (ms * 1e-3) / 1e6, 1),
            "nodes": nodes, "finite": bool(s.reduce()[6] == 0), "alg_bytes_per_step": alg,
            "step_hbm_frac": round(alg / (ms * 1e-3) / 1e9 / measured_peaks()[0]["hbm_gbs"], 4)})
    for name, kw in runs.items():
        W = c.W
        widths = kw.get("pml_widths")
        py = kw.get("periodic_y", False)
        fw = widths if widths is not None else (W, W, 0, 0) if py else W
        fields = wl.isentropic_vortex(size, size, fw, R=20.0, Mv=0.05, mean_u=(0.3, 0.0))
        s = Solver(size, size, W, c.tau, kw["sigma_max"], kw["sigma_power"], kw["bc"], kw["q"],
                   kw["nrbc_edges"], kw["beta"], kw["mean"], precision="fp32dev",
                   pml_widths=widths, periodic_y=py, sigma_split=kw.get("sigma_split", False),
                   pml_source=kw.get("pml_source", 0))
        s.init(*fields)
        s.step(warmup)
        s.init(*fields)
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(st)
        s.step(window)
        ev[1].record(st)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / window
        nodes = s.Lx * s.Ly
        out[name] = finite_or_unmeasured({
            "ms_per_step": round(ms, 4), "mlups": round(nodes / (ms * 1e-3) / 1e6, 1),
            "nodes": nodes, "finite": bool(s.reduce()[6] == 0)})
        s.close()
    return out


def finite_or_unmeasured(rec):
    """A timing taken on a run that produced non-finite or non-positive fields is not a
    measurement of the method: drop its rates."""
    if not rec["finite"]:
        for k in ("ms_per_step", "mlups", "step_hbm_frac"):
            rec.pop(k, None)
        rec["unmeasured"] = "the run went unphysical inside the window"
    return rec


def long_runs(size, warmup, limit=20000):
    """How many steps the workload survives (FP32, checked every 250 steps through the
    library's unphysical-state flag): with the printed PML gradient, and with the
    link-integrated gradient under the workload's boundary condition (east CBC relax) and with
    PNR-LODI on every edge; wall-clock rate of the surviving steps."""
    import torch
    import workloads as wl
    from paper_2504_20169_gb300 import LBMError, Solver
    c = wl.vortex_2048(n=size)
    fields = c.fields()
    out = {}
    for name, grad, edges, lim in (("printed_gradient", "central", c.nrbc_edges, 2000),
                                   ("link_gradient", "link", c.nrbc_edges, limit),
                                   ("link_gradient_pnr_edges", "link", (0, 0, 0, 0), limit)):
        with Solver(c.nx, c.ny, c.W, c.tau, c.sigma_max, c.sigma_power, c.bc, 37, edges,
                    c.beta, c.mean, precision="fp32dev", pml_grad=grad) as s:
            s.init(*fields)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            done, chunk, status = 0, 250, "finite"
            try:
                while done < lim:
                    s.step(chunk)
                    s.sync()
                    done += chunk
            except LBMError:
                status = "flagged unphysical"
            dt = time.perf_counter() - t0
            rec = {"pml_gradient": grad, "edges_WESN": list(edges), "limit": lim,
                   "steps_finite": done, "status": status,
                   "mlups": round(s.Lx * s.Ly * done / dt / 1e6, 1) if done else None}
            if status == "finite":
                r = s.moments("bulk")[0]
                rec["bulk_rho_range"] = [float(r.min()), float(r.max())]
            out[name] = rec
    return out


def fp64_flops_per_node():
    """Algorithmic FP64 operations of one interior node update, D2Q37 (FMA = 2), counted from
    the interior kernel's arithmetic: moments 125 (74 column / row sums, 28 for the first and
    second moments, 23 for rho, u, u^2, T); equilibrium coefficients 27; BGK with the +/- pair
    form 476 (8 shells x 14 shell constants, 18 pairs x 20, 4 for the rest velocity)."""
    return 125 + 27 + 476


def _served_error(reqs, ids, precision_ref="fp64"):
    """Field error of served FP32 results against the same requests run alone in FP64 (bulk:
    relative L2 of rho and T, velocity L2 over max(||u_ref||, c_s sqrt(N) / 10)); max over the
    sampled requests that finished."""
    import numpy as np
    from paper_2504_20169_gb300 import Solver
    worst = {"rho": 0.0, "ux": 0.0, "uy": 0.0, "T": 0.0}
    n = 0
    for r in reqs:
        if r.rid not in ids or r.status != "done" or r.result is None:
            continue
        c = r.case
        with Solver(c.nx, c.ny, c.W, c.tau, c.sigma_max, c.sigma_power, c.bc, 37, c.nrbc_edges,
                    c.beta, c.mean, precision=precision_ref,
                    pml_grad=getattr(c, "pml_grad", "central")) as s:
            s.init(*c.fields())
            s.step(r.steps)
            ref = s.moments(region="bulk")
        n += 1
        for k, name in enumerate(("rho", "ux", "uy", "T")):
            a, b = r.result[k], ref[k]
            den = np.sqrt(np.sum(b * b))
            if name in ("ux", "uy"):
                den = max(den, 0.1 * np.sqrt(b.size))
            worst[name] = max(worst[name], float(np.sqrt(np.sum((a - b) ** 2)) / den))
    return {"samples": n, "max_rel_l2_vs_fp64": {k: float(f"{v:.3e}") for k, v in worst.items()}}


def serving_runs(args):
    """The batched sweep at its stated size (256 seeded uneven instances, admitted at t = 0,
    1000 steps) and the Poisson request stream at its stated size (500 requests at 50/s, bulk
    64..2048, PML 8..64) with the request lengths scaled from 1k..20k to 100..2000 steps, then
    the same stream at a sustainable 5/s (150 requests). Both use the link-integrated PML
    gradient and PNR-LODI on every characteristic edge: the printed gradient and CBC relax do
    not survive such lengths (long-run entry). FP32 deviation storage through the
    continuous-batching loop. Each section samples its smallest finished requests and reruns
    them alone in FP64."""
    import workloads as wl
    from paper_2504_20169_gb300.serving import Engine, Request, summarize
    sweep = wl.batched_sweep(count=256, seed=0, steps=1000, pml_grad="link",
                             nrbc_edges=(0, 0, 0, 0))
    reqs = [Request(k, 0.0, c, c.steps) for k, c in enumerate(sweep)]
    sample = {r.rid for r in sorted(reqs, key=lambda r: r.case.nx)[:4]}
    eng = Engine(budget_bytes=200e9, precision="fp32dev", chunk=250, keep_ids=sample,
                 lookahead=len(reqs))
    eng.run(reqs)
    eng.close()
    b = summarize(reqs, eng.wall, eng.sites_steps, eng.step_seconds)
    b["error"] = _served_error(reqs, sample)
    b["what"] = "256 instances of the seeded batched sweep (N 128..1024, W 4..64, sigma_max " \
                "0.01..0.5, ZG / PNR-LODI, pulse / vortex Mach 0.1..0.5), link PML gradient, " \
                "1000 steps each (the stated 5000 are out of reach, see the long-run entry), " \
                "one launch per kernel class over all instances, chunks of 250 steps; wall " \
                "clock includes admission (host IC + upload) and retirement"
    out = [b]
    for rate, count in ((50.0, 500), (5.0, 150)):
        stream = wl.request_stream(count, rate=rate, seed=0, nmax=2048, smin=100, smax=2000,
                                   pml_grad="link", nrbc_edges=(0, 0, 0, 0))
        reqs = [Request(k, t, c, c.steps) for k, (t, c) in enumerate(stream)]
        sample = {r.rid for r in sorted(reqs, key=lambda r: r.case.nx * r.steps)[:4]}
        eng = Engine(budget_bytes=100e9, precision="fp32dev", chunk=100, keep_ids=sample)
        eng.run(reqs)
        eng.close()
        sv = summarize(reqs, eng.wall, eng.sites_steps, eng.step_seconds)
        sv["error"] = _served_error(reqs, sample)
        sv["what"] = f"Poisson stream {rate:g}/s, {count} requests, bulk log-uniform 64..2048, " \
                     "PML 8..64, 100..2000 steps (config lengths / 10), link PML gradient, " \
                     "PNR-LODI on every edge of the NRBC requests, " \
                     "100 GB admission budget, chunks of 100 steps; latency from arrival to " \
                     "fields on the host"
        out.append(sv)
    return out


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import numpy as np
    import torch
    import workloads as wl
    from paper_2504_20169_gb300 import Solver
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    c = wl.vortex_2048(n=args.size)
    if args.pml_grad != c.pml_grad:
        c = dataclasses.replace(c, pml_grad=args.pml_grad)
    fields = c.fields()
    Lx = c.nx + 2 * c.W
    sites = Lx * Lx
    Wf = c.W + 1
    interior = (Lx - 2 * Wf) ** 2

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    total, per, prof, ck, tot = timed_run(Solver, c, fields, "fp32dev", args.steps, args.warmup,
                                          local, args.window,
                                          prof_steps=min(args.steps, args.window))
    barrier()
    t_max = max_over_ranks(total, dist, "cuda")
    ms_step = t_max / args.steps
    value = ws * sites / (ms_step * 1e-3) / 1e6

    # dominant kernel: the interior BGK kernel (D2Q37 FP32: 37 loads + 37 stores of 4 B)
    peaks, peak_kind = measured_peaks()
    interior_ms = prof[0]["interior"] / max(1, prof[1])
    alg_bytes = interior * 2 * 37 * 4
    achieved = alg_bytes / (interior_ms * 1e-3) / 1e9
    traffic = profiled_traffic("k_bulk_fp32_vortex2048.md")
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
            "traffic": traffic, "kernel": "k_bulk<D2Q37,float,dev>",
            "alg_bytes_per_launch": alg_bytes, "peak_source": peak_kind,
            "frac_vs_nominal_7900": round(achieved / 7900.0, 4),
            "kernel_ms": round(interior_ms, 4),
            "kernel_share": {k: round(v / max(1e-9, sum(prof[0].values())), 4)
                             for k, v in prof[0].items()}}
    step_bytes = sites * 2 * 37 * 4
    # algorithmic bytes of one whole step (FP32): interior nodes 2 x 37 x 4 B; frame nodes
    # (PML + inner ring) also read and write the accumulator: 4 x 37 x 4 B; boundary layers
    # outside F are written once: 37 x 4 B
    frame_nodes = 2 * Wf * Lx + 2 * (Lx - 2 * Wf) * Wf
    band_nodes = 2 * 3 * (Lx + 6) + 2 * 3 * Lx
    alg_step = interior * 296 + frame_nodes * 592 + band_nodes * 148
    step_roof = {"alg_bytes_per_step": alg_step,
                 "achieved": round(alg_step / (ms_step * 1e-3) / 1e9, 1),
                 "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "frac": round(alg_step / (ms_step * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)}
    fp64 = None
    if not args.no_fp64:
        k64 = max(20, args.steps // 8)
        total64, per64, prof64, ck64, _ = timed_run(Solver, c, fields, "fp64", k64,
                                                     args.warmup, local, args.window,
                                                     prof_steps=min(k64, 100))
        ms64 = total64 / k64
        int64_ms = prof64[0]["interior"] / max(1, prof64[1])
        fp64 = {"value": round(sites / (ms64 * 1e-3) / 1e6, 1), "unit": "MLUPS",
                "ms_per_step": round(ms64, 4), "steps": k64,
                "interior_kernel_gbs": round(interior * 2 * 37 * 8 / (int64_ms * 1e-3) / 1e9, 1),
                "hbm_frac": round(interior * 2 * 37 * 8 / (int64_ms * 1e-3) / 1e9 /
                                  peaks["hbm_gbs"], 4),
                "bound": "alu (FP64 pipe)"}
        from paper_2504_20169_gb300 import peak_fma
        peak64, _ = peak_fma("fp64")
        peak32, _ = peak_fma("fp32dev")
        fl = fp64_flops_per_node()
        ach = fl * interior / (int64_ms * 1e-3) / 1e12
        fp64["alu_roofline"] = {
            "bound": "alu", "achieved": round(ach, 4), "peak": round(peak64, 4),
            "unit": "TFLOP/s", "frac": round(ach / peak64, 4),
            "flops_per_node": fl, "peak_source": "measured (lbm_peak_fma, FP64 FMA chains)",
            "fp32_fma_peak_tflops": round(peak32, 2)}
        # accuracy of the FP32 deviation storage against the FP64 path on the same solve
        res = {}
        for prec in ("fp32dev", "fp64"):
            with Solver(c.nx, c.ny, c.W, c.tau, c.sigma_max, c.sigma_power, c.bc, 37,
                        c.nrbc_edges, c.beta, c.mean, precision=prec, pml_grad=c.pml_grad) as s:
                s.init(*fields)
                s.step(args.window)
                res[prec] = (s.moments(region="F", device=True),
                             s.moments(region="bulk", device=True))
        for reg, key in ((0, "fp32_vs_fp64_rel_l2"), (1, "fp32_vs_fp64_rel_l2_bulk")):
            err = {}
            for name, a, b in zip(("rho", "ux", "uy", "T"), res["fp32dev"][reg], res["fp64"][reg]):
                den = torch.linalg.vector_norm(b) if name in ("rho", "T") else \
                    torch.clamp(torch.linalg.vector_norm(b), min=0.1 * math.sqrt(b.numel()))
                err[name] = float(f"{float(torch.linalg.vector_norm(a - b) / den):.3e}")
            fp64[key] = err
        fp64["fp32_vs_fp64_after_steps"] = args.window

    # end to end through the C ABI with host buffers
    pin = [torch.from_numpy(np.ascontiguousarray(f)).pin_memory() for f in fields]
    outs = [torch.empty((Lx, Lx), dtype=torch.float64).pin_memory() for _ in range(4)]
    s = Solver(c.nx, c.ny, c.W, c.tau, c.sigma_max, c.sigma_power, c.bc, 37, c.nrbc_edges,
               c.beta, c.mean, precision="fp32dev", pml_grad=c.pml_grad)
    import ctypes as C
    from paper_2504_20169_gb300 import _lib as L
    barrier()
    nrep = max(1, args.steps // args.window)
    t0 = time.perf_counter()
    for _ in range(nrep):
        st = L.lib().lbm_init(s.ctx, *[C.c_void_p(p.data_ptr()) for p in pin], 0)
        assert st == 0
        s.step(args.window)
        st = L.lib().lbm_moments(s.ctx, *[C.c_void_p(o.data_ptr()) for o in outs], 1, 0)
        assert st == 0
    e2e_s = time.perf_counter() - t0
    barrier()
    s.close()
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    field_bytes = 4 * sites * 8
    e2e = {"value": round(ws * sites * nrep * args.window / e2e_s / 1e6, 1), "unit": "MLUPS",
           "h2d_bytes_per_step": field_bytes / args.window,
           "d2h_bytes_per_step": field_bytes / args.window,
           "what": f"{nrep} solves through the C ABI: lbm_init from pinned host fields, "
                   f"{args.window} steps, lbm_moments to pinned host; wall clock"}

    # informational sections (single-GPU measurements): rank 0 only, after the timed work
    batched = serving = serving_sustainable = variants = None
    if rank == 0 and args.serving:
        batched, serving, serving_sustainable = serving_runs(args)
    if rank == 0 and args.variants:
        variants = variant_runs(args.size, args.window, args.warmup)
    longrun = long_runs(args.size, args.warmup) if rank == 0 and args.long else None

    if rank == 0:
        cpu = oracle_sample(args.cpu_seconds) if args.cpu_seconds > 0 else None
        if cpu is not None:
            cpu["config1_full"] = config1_cpu()
        per_sorted = sorted(per)
        line = {
            "metric": "MLUPS", "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": (WORKLOAD if args.size == 2048 else f"vortex{args.size}_w32_nrbc_d2q37")
                       + ("" if c.pml_grad == "central" else "_link_gradient"),
                       "bulk": [c.nx, c.ny], "pml_width": c.W, "pml_gradient": c.pml_grad,
                       "sigma": "cubic, sigma_max 0.1", "bc": "E: CBC relax beta 0.3; W,S,N: PNR-LODI",
                       "tau": c.tau, "stencil": "D2Q37", "storage": "FP32 deviation from rest weights",
                       "fluid_nodes_per_step": sites, "working_set_bytes": step_bytes,
                       "l2": f"working set {step_bytes / 1e9:.2f} GB > 129 MB L2; no flush"
                             if step_bytes > 129e6 else "working set below L2 size",
                       "parallelism":
                       f"replicas x{ws}"},
            "latency_ms": {"p50": round(statistics.median(per), 5),
                           "p99": round(per_sorted[min(len(per) - 1, int(math.ceil(0.99 * len(per))) - 1)], 5)},
            "roofline": roof, "step_roofline": step_roof, "fp64": fp64, "batched_fp32": batched, "serving": serving,
            "serving_sustainable": serving_sustainable,
            "variants_fp32": variants, "long_run_fp32": longrun,
            "e2e": e2e, "cpu_baseline": cpu,
            # per step: k_nrbc_rk4, k_pml_fused, k_gamma, k_bulk (one CUDA-graph replay); the
            # link gradient runs the frame as two kernels
            "gpu_launches": args.steps * ((4 if c.bc == "nrbc" else 3) + (c.pml_grad == "link")),
            "clocks": ck,
            "also": {"mlups_bulk_only": round(value * c.nx * c.ny / sites, 1),
                     "mlups_over_G": round(value * (Lx + 6) * (Lx + 6) / sites, 1),
                     "note": "bulk-only counts the PML as overhead (the paper's view); over G "
                             "adds the 3 boundary layers outside F"},
            "timing": f"headline: fresh solves of {args.window} steps (untimed re-init between), "
                      "CUDA-graph replay, events per step on the launching stream; roofline: "
                      "interior kernel events in a separate window where each kernel class "
                      "runs alone; step_roofline: whole-step algorithmic bytes / ms_per_step",
            "totals_check": {"mass": float(tot[0]), "bad_nodes": float(tot[6])},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
