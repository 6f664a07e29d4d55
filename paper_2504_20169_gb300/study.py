"""The thermal-vortex boundary study of Sec. 5.2, run on the GPU through the public API.

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

Run: python -m paper_2504_20169_gb300.study   (prints one JSON line per case and a table)
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


def main():
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--tau", type=float, default=0.8)
    ap.add_argument("--steps", type=int, default=1500)
    a = ap.parse_args()
    meta, results = run(steps=a.steps, tau=a.tau)
    print(json.dumps(meta))
    for r in results:
        print(json.dumps(r))
    print("| BC | W | sigma_max | e_bar rho | e_bar u_x | e_bar T | C_rho | C_ux | C_T | C_t |")
    print("|---|---|---|---|---|---|---|---|---|---|")
    for r in results:
        eb, cz = r["ebar"], r["C_Z"]
        f = lambda v: "n/a" if v is None else f"{v:.3g}"
        print(f"| {r['bc']} | {r['W']} | {r['sigma_max']} | {f(eb['rho'])} | {f(eb['ux'])} | "
              f"{f(eb['T'])} | {f(cz['rho'])} | {f(cz['ux'])} | {f(cz['T'])} | {r['C_t']:.1f} |"
              + ("" if r["status"] == "ok" else f" {r['status']}"))


if __name__ == "__main__":
    main()
