"""The boundary studies of Sec. 5, run on the GPU through the public API.

Density step (Sec. 5.1, `run_density_step`): 200 x 20 bulk, periodic y axis, Mach 0.05 mean
flow along x, the tanh density step (workloads.density_step), D2Q9 / D2Q17 / D2Q37. Cases per
stencil: ZG and PNR-LODI without PML, and with PML W = 10 / 20 / 40 on the two x edges with
the sigma_max of Table 1 (quadratic ramp). Errors e_rho, e_ux against a periodic reference on
an x-padded grid, sampled every `sample` steps; C_Z and C_t relative to ZG without PML, as below.

Thermal vortex (Sec. 5.2, `run`):

D2Q17 (third-order equilibrium), 300 x 300 bulk, every edge open, Mach 0.1 mean flow, the
vortex of Sec. 5.2 (workloads.paper_vortex). Cases, as in Figs. 8-9:
  ZG      zero gradient, without PML and with PML W = 10 / 20 / 40
          (sigma_max 0.02 / 0.01 / 0.003, quadratic ramp of Eq. PML_ramp)
  CBC(A)  outlet (east) CBC relax with beta = Ma, other edges PNR-LODI, without PML and with
          PML W = 10 / 20 / 40 (sigma_max 0.007 / 0.002 / 0.001)
  CBC(B)  outlet with zero incoming amplitudes (CBC relax with beta = 1), W = 20
Errors: e_Z of Sec. 5 for Z = rho, u_x, T against a fully periodic reference run on a grid
padded so that no signal wraps back into the bulk within the run, sampled every `sample`
steps; e_bar_Z = mean over the samples; C_Z = e_bar_Z / e_bar_Z of ZG without PML.
Cost: C_t = t_BC / t_ZG (Sec. 5, "Computational Cost") with t_BC the GPU time of the kernels
that handle the boundary: the PML frame (its stream-collide and PML terms), the
characteristic targets and the boundary band; t_ZG the band time of ZG without PML. Each
kernel class is timed alone with CUDA events (lbm_profile_*).
The paper leaves tau and the vortex's b, r*, K open; tau = 0.8, b = 0.2, r* = 0.5, K = 180.

Run: python -m paper_2504_20169_gb300.study [--case vortex|step|all]   (one JSON line per case
and a table)
"""
from __future__ import annotations

import json
import math
import os
import sys


def cases(Ma):
    zg = {10: 0.02, 20: 0.01, 40: 0.003}
    cbc = {10: 0.007, 20: 0.002, 40: 0.001}
    out = [("ZG", "zg", 0, 0.0, (0, 0, 0, 0), 0.0)]
    out += [("ZG", "zg", W, s, (0, 0, 0, 0), 0.0) for W, s in zg.items()]
    out += [("CBC(A)", "nrbc", 0, 0.0, (0, 1, 0, 0), Ma)]
    out += [("CBC(A)", "nrbc", W, s, (0, 1, 0, 0), Ma) for W, s in cbc.items()]
    out += [("CBC(B)", "nrbc", 20, cbc[20], (0, 1, 0, 0), 1.0)]
    return out


def run(L=300, steps=1500, sample=50, tau=0.8, Ma=0.1, q=17, precision="fp64", prof_steps=100):
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads as wl
    from . import Solver, lattice_info
    _, _, r = lattice_info(q)
    speed = (math.sqrt(2.0) + Ma) / r                  # fastest signal, nodes per step
    pad = int(speed * steps * 1.05) + 8
    # reference: fully periodic, padded grid; keep the bulk window at every sample
    big = L + 2 * pad
    refs = []
    with Solver(big, big, 0, tau, bc="periodic", q=q, precision=precision) as ref:
        ref.init(*wl.paper_vortex(L, L, 0, Ma=Ma, pad=pad))
        for k in range(steps // sample):
            ref.step(sample)
            f = ref.moments(region="F", device=True)
            refs.append([t[pad:pad + L, pad:pad + L].contiguous() for t in f])
    results = []
    for label, bc, W, sig, edges, beta in cases(Ma):
        s = Solver(L, L, W, tau, sig, 2, bc, q, edges, beta, (1.0, Ma, 0.0, 1.0),
                   precision=precision)
        s.init(*wl.paper_vortex(L, L, W, Ma=Ma))
        e = {"rho": [], "ux": [], "T": []}
        status = "ok"
        try:
            for k in range(steps // sample):
                s.step(sample)
                sums = s.error_sums(refs[k])
                e["rho"].append(math.sqrt(sums[2]))
                e["ux"].append(math.sqrt(sums[5]))
                e["T"].append(math.sqrt(sums[11]))
        except Exception as ex:  # the library reports LBM_EUNSTABLE for a diverged run
            status = str(ex).split(":")[0]
        s.init(*wl.paper_vortex(L, L, W, Ma=Ma))
        s.profile_enable(prof_steps)
        s.step(prof_steps)
        ms, n = s.profile_read()
        s.close()
        t_bc = (ms["frame1"] + ms["frame2"] if W > 0 else 0.0) + ms["targets"] + ms["band"]
        results.append({"bc": label, "W": W, "sigma_max": sig, "status": status,
                        "ebar": {k: (sum(v) / len(v) if v and status == "ok" else None)
                                 for k, v in e.items()},
                        "t_bc_us": 1e3 * t_bc / n})
    base = results[0]
    for r_ in results:
        r_["C_Z"] = {k: (r_["ebar"][k] / base["ebar"][k]
                         if r_["ebar"][k] and base["ebar"][k] else None) for k in r_["ebar"]}
        r_["C_t"] = r_["t_bc_us"] / base["t_bc_us"]
    meta = {"L": L, "steps": steps, "sample": sample, "tau": tau, "Ma": Ma, "q": q,
            "precision": precision, "reference_grid": big}
    return meta, results


# Table 1: sigma_max of the density-step runs per stencil, boundary condition and width
STEP_SIGMA = {
    9: {"ZG": {10: 0.17, 20: 0.10, 40: 0.07}, "LODI": {10: 0.001, 20: 0.04, 40: 0.04}},
    17: {"ZG": {10: 0.33, 20: 0.14, 40: 0.09}, "LODI": {10: 0.001, 20: 0.08, 40: 0.04}},
    37: {"ZG": {10: 0.35, 20: 0.175, 40: 0.10}, "LODI": {10: 0.001, 20: 0.10, 40: 0.06}},
}


def step_cases(q):
    """(label, bc, W, sigma_max, Appendix source bitmask). The last ones are the Appendix
    comparison (Fig. A.1 setting: LODI, W = 10, sigma_max = 0.001) with the PML source terms
    I, II, III of Eq. (NSF-CHAR-PML) added to the LODI targets, with the sign of the collision
    term and (suffix "+sign") with the printed sign."""
    out = [("ZG", "zg", 0, 0.0, 0), ("LODI", "nrbc", 0, 0.0, 0)]
    for W in (10, 20, 40):
        out += [("ZG", "zg", W, STEP_SIGMA[q]["ZG"][W], 0),
                ("LODI", "nrbc", W, STEP_SIGMA[q]["LODI"][W], 0)]
    for src, name in ((1, "I"), (2, "II"), (4, "III"), (3, "I+II"), (7, "I+II+III")):
        out.append((f"LODI+{name}", "nrbc", 10, 0.001, src))
        out.append((f"LODI+{name} +sign", "nrbc", 10, 0.001, src + 8))
    return out


def run_density_step(q=37, Lx=200, Ly=20, steps=2000, sample=20, tau=0.8, Ma=0.05,
                     precision="fp64", prof_steps=100, cases=None, pml_grad="central"):
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads as wl
    from . import Solver, lattice_info
    _, _, r = lattice_info(q)
    speed = (math.sqrt(2.0) + Ma) / r
    pad = int(speed * steps * 1.05) + 8
    refs = []
    # reference: periodic in x and y on an x-padded grid; the formula continues into the pad
    with Solver(Lx + 2 * pad, Ly, 0, tau, bc="periodic", q=q, precision=precision) as ref:
        fr = wl.density_step(Lx, Ly, Ma=Ma, W=(pad, pad, 0, 0))
        ref.init(*fr)
        for k in range(steps // sample):
            ref.step(sample)
            f = ref.moments(region="F", device=True)
            refs.append([t[:, pad:pad + Lx].contiguous() for t in f])
    results = []
    mean = (1.0, Ma, 0.0, 1.0)
    for label, bc, W, sig, src in (cases if cases is not None else step_cases(q)):
        s = Solver(Lx, Ly, W, tau, sig, 2, bc, q, (0, 0, 0, 0), 0.0, mean,
                   precision=precision, periodic_y=True, pml_source=src, pml_grad=pml_grad)
        fields = wl.density_step(Lx, Ly, Ma=Ma, W=W, Wy=0)
        s.init(*fields)
        e = {"rho": [], "ux": []}
        status = "ok"
        try:
            for k in range(steps // sample):
                s.step(sample)
                sums = s.error_sums(refs[k])
                e["rho"].append(math.sqrt(sums[2]))
                e["ux"].append(math.sqrt(sums[5]))
        except Exception as ex:
            status = str(ex).split(":")[0] + f" after <= {(len(e['rho']) + 1) * sample} steps"
        s.init(*fields)
        s.profile_enable(prof_steps)
        s.step(prof_steps)
        ms, n = s.profile_read()
        s.close()
        t_bc = (ms["frame1"] + ms["frame2"] if W > 0 else 0.0) + ms["targets"] + ms["band"]
        results.append({"q": q, "bc": label, "W": W, "sigma_max": sig, "status": status,
                        "ebar": {k: (sum(v) / len(v) if v and status == "ok" else None)
                                 for k, v in e.items()},
                        "emax": {k: (max(v) if v and status == "ok" else None)
                                 for k, v in e.items()},
                        "t_bc_us": 1e3 * t_bc / n})
    base = results[0]
    for r_ in results:
        r_["C_Z"] = {k: (r_["ebar"][k] / base["ebar"][k]
                         if r_["ebar"][k] and base["ebar"][k] else None) for k in r_["ebar"]}
        r_["C_t"] = r_["t_bc_us"] / base["t_bc_us"]
    meta = {"case": "density_step", "Lx": Lx, "Ly": Ly, "steps": steps, "sample": sample,
            "tau": tau, "Ma": Ma, "q": q, "precision": precision, "pml_grad": pml_grad,
            "reference_grid": [Lx + 2 * pad, Ly]}
    return meta, results


def run_bench_workload(steps=200, sample=20, precision="fp32dev", n=2048, W=32):
    """e_Z of the benchmark workload itself (2048^2 + PML 32 cubic 0.1, characteristic BC with
    CBC relax on the east edge, D2Q37, tau 0.55, isentropic vortex in a Mach 0.3 flow) against a
    periodic reference on a grid padded by the distance the fastest signal covers; also ZG
    without PML, ZG with the same PML and the characteristic BC without PML, for C_Z. The
    window stays below the step count at which the PML modes of the printed scheme grow."""
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads as wl
    from . import Solver, lattice_info
    _, _, r = lattice_info(37)
    pad = int((math.sqrt(2.0) + 0.35) / r * steps * 1.05) + 8
    tau, vort = 0.55, dict(R=20.0, Mv=0.05, mean_u=(0.3, 0.0))
    refs = []
    with Solver(n + 2 * pad, n + 2 * pad, 0, tau, bc="periodic", q=37, precision=precision) as ref:
        ref.init(*wl.isentropic_vortex(n + 2 * pad, n + 2 * pad, 0, **vort))
        for k in range(steps // sample):
            ref.step(sample)
            f = ref.moments(region="F", device=True)
            refs.append([t[pad:pad + n, pad:pad + n].contiguous() for t in f])
    mean = (1.0, 0.3, 0.0, 1.0)
    cases = [("ZG", "zg", 0, (0, 0, 0, 0), "central"),
             ("ZG + PML", "zg", W, (0, 0, 0, 0), "central"),
             ("ZG + PML (link gradient)", "zg", W, (0, 0, 0, 0), "link"),
             ("CBC(A)", "nrbc", 0, (0, 1, 0, 0), "central"),
             ("CBC(A) + PML (benchmark)", "nrbc", W, (0, 1, 0, 0), "central"),
             ("CBC(A) + PML (link gradient)", "nrbc", W, (0, 1, 0, 0), "link"),
             ("PNR + PML (link gradient)", "nrbc", W, (0, 0, 0, 0), "link")]
    results = []
    for label, bc, w, edges, grad in cases:
        with Solver(n, n, w, tau, 0.1 if w else 0.0, 3, bc, 37, edges, 0.3, mean,
                    precision=precision, pml_grad=grad) as s:
            s.init(*wl.isentropic_vortex(n, n, w, **vort))
            e = {"rho": [], "ux": [], "T": []}
            status = "ok"
            try:
                for k in range(steps // sample):
                    s.step(sample)
                    sums = s.error_sums(refs[k])
                    e["rho"].append(math.sqrt(sums[2]))
                    e["ux"].append(math.sqrt(sums[5]))
                    e["T"].append(math.sqrt(sums[11]))
            except Exception as ex:
                status = str(ex).split(":")[0]
        results.append({"bc": label, "W": w, "status": status,
                        "ebar": {k: (sum(v) / len(v) if v else None) for k, v in e.items()},
                        "e_last": {k: (v[-1] if v else None) for k, v in e.items()}})
    for r_ in results:
        r_["C_Z"] = {k: (r_["ebar"][k] / results[0]["ebar"][k]
                         if r_["ebar"][k] and results[0]["ebar"][k] else None) for k in r_["ebar"]}
    meta = {"case": "bench_workload", "n": n, "W": W, "steps": steps, "sample": sample,
            "precision": precision, "reference_grid": n + 2 * pad}
    return meta, results


def run_stability_map(N=256, steps=10000, chunk=500, precision="fp64"):
    """How long each boundary treatment survives (section "long runs" of the design notes):
    isentropic vortex R 20, Mv 0.05 on an N^2 bulk, PML W 32 with cubic sigma_max 0.1 where a
    PML is used, D2Q37 and D2Q17, tau 0.55 / 0.8, mean flow Mach 0 / 0.3; periodic, ZG,
    PNR-LODI and east CBC relax without PML, and ZG / PNR / east CBC relax with the printed
    and with the link-integrated PML gradient. Each run is checked every `chunk` steps through
    the library's unphysical-state flag."""
    import workloads as wl
    from . import LBMError, Solver
    out = []
    for q in (37, 17):
        for tau in (0.55, 0.8):
            for Ma in (0.0, 0.3):
                runs = [(0, "periodic", (0, 0, 0, 0), "central")]
                for W in (0, 32):
                    for bc, edges in (("zg", (0, 0, 0, 0)), ("nrbc", (0, 0, 0, 0)),
                                      ("nrbc", (0, 1, 0, 0))):
                        for grad in (("central",) if W == 0 else ("central", "link")):
                            runs.append((W, bc, edges, grad))
                for W, bc, edges, grad in runs:
                    f = wl.isentropic_vortex(N, N, W, R=20.0, Mv=0.05, mean_u=(Ma, 0.0))
                    s = Solver(N, N, W, tau, 0.1 if W else 0.0, 3, bc, q, edges, Ma,
                               (1.0, Ma, 0.0, 1.0), precision=precision, pml_grad=grad)
                    s.init(*f)
                    done, status = 0, "ok"
                    try:
                        while done < steps:
                            s.step(chunk)
                            s.sync()
                            done += chunk
                    except LBMError:
                        status = f"div. {done + chunk}"
                    s.close()
                    out.append(dict(q=q, tau=tau, Ma=Ma, W=W, bc=bc, edges=list(edges),
                                    grad=grad, status=status))
    return out


def _fmt(v):
    return "n/a" if v is None else f"{v:.3g}"


def main():
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="all", choices=("vortex", "step", "scan", "bench", "stability", "all"))
    ap.add_argument("--tau", type=float, default=0.8)
    ap.add_argument("--grad", default="central", choices=("central", "link"),
                    help="PML gradient of the density-step cases: the printed central "
                         "differences or the link-integrated option")
    ap.add_argument("--steps", type=int, default=None)
    a = ap.parse_args()
    if a.case in ("bench", "all"):
        # e_Z is a sum over the 2048^2 bulk (no 1/N); the rms relative error is e_Z / 2048
        print("| precision | BC | W | e_bar rho | e_bar u_x | e_bar T | rms rel. error rho at end |")
        print("|---|---|---|---|---|---|---|")
        for prec in ("fp32dev", "fp64"):
            st = a.steps or 200
            meta, results = run_bench_workload(steps=st, precision=prec,
                                               sample=20 if st <= 400 else 50)
            print(json.dumps(meta))
            for r in results:
                eb = r["ebar"]
                rms = None if r["e_last"]["rho"] is None else r["e_last"]["rho"] / meta["n"]
                print(f"| {prec} | {r['bc']} | {r['W']} | {_fmt(eb['rho'])} | {_fmt(eb['ux'])} | "
                      f"{_fmt(eb['T'])} | {_fmt(rms)} |" + ("" if r["status"] == "ok" else f" {r['status']}"))
    if a.case in ("scan", "all"):
        # Figs. 3-4: the sigma_max scan of the density step with ZG beyond a W = 20 PML (and
        # PNR-LODI for comparison); the first row of each block is ZG without PML (C_Z = 1)
        print("| q | BC | W | sigma_max | e_bar rho | e_bar u_x | max e rho | C_rho | C_ux | status |")
        print("|---|---|---|---|---|---|---|---|---|---|")
        sig = (0.01, 0.03, 0.06, 0.10, 0.14, 0.2, 0.3, 0.6)
        for q in (9, 17, 37):
            cases = [("ZG", "zg", 0, 0.0, 0)] + [("ZG", "zg", 20, v, 0) for v in sig] + \
                    [("LODI", "nrbc", 20, v, 0) for v in sig]
            meta, results = run_density_step(q=q, steps=a.steps or 2000, tau=a.tau, cases=cases,
                                             pml_grad=a.grad)
            print(json.dumps(meta))
            for r in results:
                eb, cz = r["ebar"], r["C_Z"]
                print(f"| {q} | {r['bc']} | {r['W']} | {r['sigma_max']} | {_fmt(eb['rho'])} | "
                      f"{_fmt(eb['ux'])} | {_fmt(r['emax']['rho'])} | {_fmt(cz['rho'])} | "
                      f"{_fmt(cz['ux'])} | {r['status']} |")
    if a.case in ("step", "all"):
        print("| q | BC | W | sigma_max | e_bar rho | e_bar u_x | max e rho | C_rho | C_ux | C_t |")
        print("|---|---|---|---|---|---|---|---|---|---|")
        for q in (9, 17, 37):
            meta, results = run_density_step(q=q, steps=a.steps or 2000, tau=a.tau,
                                             pml_grad=a.grad)
            print(json.dumps(meta))
            for r in results:
                print(json.dumps(r))
            for r in results:
                eb, cz = r["ebar"], r["C_Z"]
                print(f"| {q} | {r['bc']} | {r['W']} | {r['sigma_max']} | {_fmt(eb['rho'])} | "
                      f"{_fmt(eb['ux'])} | {_fmt(r['emax']['rho'])} | {_fmt(cz['rho'])} | "
                      f"{_fmt(cz['ux'])} | {r['C_t']:.1f} |"
                      + ("" if r["status"] == "ok" else f" {r['status']}"))
    if a.case == "stability":
        for r in run_stability_map(steps=a.steps or 10000):
            print(json.dumps(r))
    if a.case in ("vortex", "all"):
        meta, results = run(steps=a.steps or 1500, tau=a.tau)
        print(json.dumps(meta))
        for r in results:
            print(json.dumps(r))
        print("| BC | W | sigma_max | e_bar rho | e_bar u_x | e_bar T | C_rho | C_ux | C_T | C_t |")
        print("|---|---|---|---|---|---|---|---|---|---|")
        for r in results:
            eb, cz = r["ebar"], r["C_Z"]
            print(f"| {r['bc']} | {r['W']} | {r['sigma_max']} | {_fmt(eb['rho'])} | "
                  f"{_fmt(eb['ux'])} | {_fmt(eb['T'])} | {_fmt(cz['rho'])} | {_fmt(cz['ux'])} | "
                  f"{_fmt(cz['T'])} | {r['C_t']:.1f} |"
                  + ("" if r["status"] == "ok" else f" {r['status']}"))


if __name__ == "__main__":
    main()
