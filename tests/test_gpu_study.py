"""The Sec. 5 study drivers run end to end on short windows (structure and sanity of the
reported errors and cost ratios; the full runs are in the study module's main)."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_density_step_study_short():
    from paper_2504_20169_gb300 import study
    cases = [("ZG", "zg", 0, 0.0, 0), ("LODI", "nrbc", 0, 0.0, 0), ("ZG", "zg", 10, 0.33, 0),
             ("LODI+I", "nrbc", 10, 0.001, 1)]
    meta, res = study.run_density_step(q=17, steps=60, sample=20, prof_steps=10, cases=cases)
    assert meta["q"] == 17 and len(res) == 4
    assert res[0]["C_Z"]["rho"] == pytest.approx(1.0) and res[0]["C_t"] == pytest.approx(1.0)
    for r in res:
        assert r["status"] == "ok"
        assert all(math.isfinite(v) and v >= 0 for v in r["ebar"].values())
        assert r["t_bc_us"] > 0
    # the PML adds the frame kernel to the boundary cost
    assert res[2]["C_t"] > 1.0


def test_vortex_study_short():
    from paper_2504_20169_gb300 import study
    meta, res = study.run(L=64, steps=40, sample=20, prof_steps=10)
    assert meta["L"] == 64 and res[0]["bc"] == "ZG" and res[0]["W"] == 0
    labels = {r["bc"] for r in res}
    assert {"ZG", "CBC(A)", "CBC(B)"} <= labels
    for r in res:
        assert r["t_bc_us"] > 0
        if r["status"] == "ok":
            assert all(math.isfinite(v) for v in r["ebar"].values())
