"""Host-side logic of the serving loop: HBM-budget admission with FIFO order and backfill."""
from paper_2504_20169_gb300.serving import Request, Scheduler, summarize


class R:
    def __init__(self, rid, nbytes):
        self.rid, self.nbytes = rid, nbytes


def test_admission_respects_budget_fifo_and_backfill():
    s = Scheduler(100, lookahead=4)
    q = [R(0, 60), R(1, 50), R(2, 30), R(3, 10), R(4, 5)]
    got = [r.rid for r in s.pick(q)]
    assert got == [0, 2, 3]          # 1 does not fit after 0; 2 and 3 backfill; 4 beyond look-ahead
    assert s.used == 100
    s.release(q[0])
    q2 = [q[1], q[4]]
    assert [r.rid for r in s.pick(q2)] == [1, 4]
    assert s.used == 95


def test_request_that_can_never_fit_is_skipped():
    s = Scheduler(10)
    assert s.pick([R(0, 11), R(1, 5)])[0].rid == 1


def test_summary_percentiles():
    reqs = []
    for k in range(100):
        r = Request(k, 0.0, None, 1)
        r.status, r.finished = "done", float(k + 1)
        reqs.append(r)
    out = summarize(reqs, 10.0, 5e7)
    assert out["done"] == 100 and abs(out["latency_p50_s"] - 50.5) < 1e-9
    assert out["latency_p99_s"] > 99 and out["aggregate_mlups"] == 5.0
