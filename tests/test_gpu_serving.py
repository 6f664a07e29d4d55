"""Batched execution and the continuous-batching loop: every instance computes the same
result alone and in the mix (bit for bit), including instances admitted while others run and
a mix from which an unstable member is retired."""
import numpy as np
import pytest

import workloads as wl
from parity_helpers import case_kwargs, make_solver

pytestmark = pytest.mark.gpu

CASES = [
    case_kwargs(nx=64, ny=48, W=6, tau=0.7, sigma_max=0.1, bc="zg"),
    case_kwargs(nx=40, ny=40, W=0, tau=0.6, sigma_max=0.0, bc="nrbc", nrbc_edges=(1, 0, 0, 1),
                beta=0.2, mean=(1.0, 0.1, 0.0, 1.0)),
    case_kwargs(nx=96, ny=80, W=12, tau=0.8, sigma_max=0.05, bc="nrbc", nrbc_edges=(0, 1, 0, 0),
                beta=0.3, mean=(1.0, 0.2, 0.0, 1.0)),
    # periodic y axis, CBC relax on the x edges, Appendix PML source
    case_kwargs(nx=60, ny=12, W=8, tau=0.8, sigma_max=0.05, sigma_power=2, bc="nrbc",
                nrbc_edges=(1, 1, 0, 0), beta=0.2, mean=(1.0, 0.05, 0.0, 1.0), periodic_y=True,
                pml_source=3),
    # per-edge widths with the split sigma form
    case_kwargs(nx=40, ny=30, W=0, tau=0.75, sigma_max=0.15, sigma_power=2, bc="zg",
                widths=(3, 10, 0, 5), split=True),
]


def fields_of(k, kw):
    if k == 0:
        return wl.pressure_pulse(kw["nx"], kw["ny"], kw["W"], amp=1e-3, halfwidth=4.0)
    if k == 1:
        return wl.pressure_pulse(kw["nx"], kw["ny"], kw["W"], amp=2e-3, halfwidth=3.0,
                                 u0=(0.1, 0.0))
    if k == 2:
        return wl.isentropic_vortex(kw["nx"], kw["ny"], kw["W"], R=8.0, mean_u=(0.2, 0.0))
    if k == 3:
        return wl.density_step(kw["nx"], kw["ny"], Ma=0.05, W=kw["W"], Wy=0)
    return wl.random_smooth_state(kw["nx"], kw["ny"], kw["widths"], seed=4, du=0.03)


def alone(k, steps, precision):
    kw = CASES[k]
    with make_solver(kw, precision) as s:
        s.init(*fields_of(k, kw))
        s.step(steps)
        return s.moments()


@pytest.mark.parametrize("precision", ["fp64", "fp32dev"])
def test_batch_results_equal_alone_with_midrun_admission(precision):
    from paper_2504_20169_gb300.serving import Batch
    solvers = [make_solver(kw, precision) for kw in CASES]
    for k, s in enumerate(solvers):
        s.init(*fields_of(k, CASES[k]))
    b = Batch()
    b.set(solvers[:2])                 # instances 2.. arrive later
    assert b.step(20)
    b.set(solvers)                     # admitted while the others are resident
    assert b.step(25)
    b.set([solvers[0]] + solvers[2:])  # instance 1 retires after 45 steps
    assert b.step(15)
    got = [s.moments() for s in solvers]
    b.close()
    for s in solvers:
        s.close()
    steps = [60, 45] + [40] * (len(CASES) - 2)
    for k in range(len(CASES)):
        ref = alone(k, steps[k], precision)
        for g, r in zip(got[k], ref):
            assert np.array_equal(g, r), k


def test_unstable_member_is_retired_without_touching_others():
    import torch
    from paper_2504_20169_gb300.serving import Engine, Request
    eng = Engine(budget_bytes=4e9, precision="fp64", chunk=10)
    reqs = [Request(k, 0.0, wl.Case(f"c{k}", kw["nx"], kw["ny"], kw["W"], kw["tau"],
                                    kw["sigma_max"], kw["sigma_power"], kw["bc"], 30, "uniform",
                                    dict(zip(("rho", "ux", "uy", "T"), kw["mean"])),
                                    nrbc_edges=kw["nrbc_edges"], beta=kw["beta"],
                                    mean=kw["mean"]), 30)
            for k, kw in enumerate(CASES[:3])]
    # poison instance 1 right after it is admitted
    orig = eng._start

    def start(r, now):
        orig(r, now)
        if r.rid == 1:
            P = r.solver.export_populations()
            P[:, 8, 8] = np.nan
            r.solver.import_populations(P)
            r.solver.step(1)
            torch.cuda.synchronize()
            r.remaining -= 1
    eng._start = start
    eng.run(reqs)
    eng.close()
    assert [r.status for r in reqs] == ["done", "unstable", "done"]
    for k in (0, 2):
        kw = CASES[k]
        with make_solver(kw) as s:
            s.init(*wl.uniform(kw["nx"], kw["ny"], kw["W"], *kw["mean"]))
            s.step(30)
            ref = s.moments(region="bulk")
        for g, r in zip(reqs[k].result, ref):
            assert np.array_equal(g, r)


def test_engine_serves_a_poisson_stream():
    from paper_2504_20169_gb300.serving import Engine, Request, summarize
    stream = wl.request_stream(12, rate=200.0, seed=1, nmax=256, smin=20, smax=60)
    reqs = [Request(k, t, c, c.steps) for k, (t, c) in enumerate(stream)]
    eng = Engine(budget_bytes=2e9, precision="fp32dev", chunk=16)
    eng.run(reqs)
    eng.close()
    s = summarize(reqs, eng.wall, eng.sites_steps)
    assert s["done"] + s["unstable"] == 12 and s["rejected"] == 0
    assert s["latency_p99_s"] >= s["latency_p50_s"] > 0


MIX = [  # one group per (stencil, precision, gradient mode) with ragged members
    (case_kwargs(nx=64, ny=48, W=6, tau=0.7, sigma_max=0.1, bc="zg"), "fp32dev"),
    (case_kwargs(nx=96, ny=80, W=12, tau=0.8, sigma_max=0.05, bc="nrbc", nrbc_edges=(0, 1, 0, 0),
                 beta=0.3, mean=(1.0, 0.2, 0.0, 1.0)), "fp32dev"),
    (case_kwargs(nx=50, ny=70, W=5, tau=0.75, sigma_max=0.2, sigma_power=2, bc="zg",
                 pml_grad="link"), "fp32dev"),
    (case_kwargs(nx=40, ny=40, W=0, tau=0.6, sigma_max=0.0, bc="nrbc", nrbc_edges=(1, 0, 0, 1),
                 beta=0.2, mean=(1.0, 0.1, 0.0, 1.0)), "fp32dev"),
    (case_kwargs(nx=60, ny=12, W=8, tau=0.8, sigma_max=0.05, sigma_power=2, bc="nrbc",
                 mean=(1.0, 0.05, 0.0, 1.0), periodic_y=True, pml_grad="link"), "fp64"),
    (case_kwargs(nx=36, ny=44, W=4, tau=0.7, sigma_max=0.1, bc="zg", q=17), "fp32dev"),
]


def _mix_fields(kw):
    if kw["periodic_y"]:
        return wl.density_step(kw["nx"], kw["ny"], Ma=0.05, W=kw["W"], Wy=0)
    return wl.random_smooth_state(kw["nx"], kw["ny"], kw["W"], seed=kw["nx"], du=0.03,
                                  mean_u=(kw["mean"][1], 0.0))


def _alone(kw, prec, steps):
    with make_solver(kw, prec) as s:
        s.init(*_mix_fields(kw))
        s.step(steps)
        return s.moments()


@pytest.mark.parametrize("tile", [(32, 4), (128, 1), (64, 2), (32, 8)])
def test_batched_groups_equal_alone_for_every_tile_shape(tile):
    """Mixed stencils, precisions and gradient modes in one batch (four groups); the interior
    block shape never changes a bit; a member stepped on its own between batch steps makes the
    batch rebuild its plans."""
    from paper_2504_20169_gb300.serving import Batch
    solvers = [make_solver(kw, prec) for kw, prec in MIX]
    for (kw, prec), s in zip(MIX, solvers):
        s.init(*_mix_fields(kw))
    b = Batch()
    b.tile(*tile)
    b.set(solvers)
    assert b.step(13)
    solvers[2].step(3)                  # out-of-band step of one member
    assert b.step(10)
    got = [s.moments() for s in solvers]
    b.close()
    for s in solvers:
        s.close()
    for k, (kw, prec) in enumerate(MIX):
        ref = _alone(kw, prec, 26 if k == 2 else 23)
        for g, r in zip(got[k], ref):
            assert np.array_equal(g, r), (k, tile)


def test_autotune_picks_a_shape_and_changes_nothing():
    from paper_2504_20169_gb300.serving import Batch
    solvers = [make_solver(kw, prec) for kw, prec in MIX[:3]]
    for (kw, prec), s in zip(MIX[:3], solvers):
        s.init(*_mix_fields(kw))
    b = Batch()
    b.set(solvers)
    tx, by = b.autotune(steps=2)
    assert tx in (32, 64, 128, 256) and by >= 1 and tx * by <= 256
    assert b.step(5)
    got = [s.moments() for s in solvers]
    steps = [s.steps for s in solvers]
    b.close()
    for s in solvers:
        s.close()
    assert steps == [8 * 3 + 5] * 3
    for k, (kw, prec) in enumerate(MIX[:3]):
        ref = _alone(kw, prec, steps[k])
        for g, r in zip(got[k], ref):
            assert np.array_equal(g, r), k
