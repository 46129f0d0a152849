"""Host logic of the serving loop and the autotuner, on the CPU with a fake
batch (no GPU): admission order and refusal, slot reuse after retirement,
requests arriving while others run sharing launches, latency bookkeeping,
and the tuner's choice and cache."""
import json

import numpy as np

from paper_2012_11075_gb300 import autotune, serve


class FakeParams:
    def __init__(self, nx, ny):
        self.nx, self.ny = nx, ny


class FakeBatch:
    """Holds at most `slots` cases; a case stops after `need` launches."""

    def __init__(self, slots, precision=1, scheme=1):
        self.slots = slots
        self.precision, self.scheme = precision, scheme
        self.cases = {}
        self.next = 0
        self.admit_log = []
        self.launch_log = []
        self.cfg = (128, 32, 4)

    def admit(self, params, rho, tol, max_steps):
        if len(self.cases) >= self.slots:
            return None
        cid = self.next
        self.next += 1
        self.cases[cid] = {"need": int(rho), "done": 0, "steps": 0, "reported": False}
        self.admit_log.append(cid)
        return cid

    def get_config(self):
        return self.cfg

    def set_config(self, *cfg):
        self.cfg = tuple(cfg)

    def advance(self, n):
        for _ in range(n):
            running = [c for c, v in self.cases.items() if v["done"] < v["need"]]
            self.launch_log.append(tuple(running))
            for c in running:
                self.cases[c]["done"] += 1
                self.cases[c]["steps"] += self.cfg[2]

    def poll(self):
        out = []
        for c, v in self.cases.items():
            if v["done"] >= v["need"] and not v["reported"]:
                v["reported"] = True
                out.append(c)
        return out

    def info(self, cid):
        v = self.cases[cid]
        return {"state": v.get("state", 1), "steps": v["steps"]}

    def retire(self, cid):
        del self.cases[cid]

    def counts(self):
        return {"running": sum(1 for v in self.cases.values() if v["done"] < v["need"])}


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001
        return self.t


def _req(rid, arrival, need):
    return serve.Request(rid, arrival, FakeParams(10, 10), need, 1e-6, 1000)


def test_fifo_admission_refusal_and_slot_reuse():
    b = FakeBatch(slots=2)
    srv = serve.Server(b, clock=FakeClock())
    for k, need in enumerate([3, 1, 2, 1]):
        srv.submit(_req(k, 0.0, need))
    srv.admit_waiting()
    assert b.admit_log == [0, 1] and len(srv.queue) == 2      # 3rd refused, kept queued
    srv.step()                                                # case 1 finishes
    assert [r.rid for r in srv.report.completed] == [1]
    srv.admit_waiting()
    assert b.admit_log == [0, 1, 2]                           # freed slot reused, FIFO
    while srv.resident or srv.queue:
        srv.step()
        srv.admit_waiting()
    assert sorted(r.rid for r in srv.report.completed) == [0, 1, 2, 3]
    assert all(r.finished >= r.admitted >= r.arrival for r in srv.report.completed)


def test_late_arrivals_share_launches_with_running_cases():
    b = FakeBatch(slots=8)
    clock = FakeClock()
    srv = serve.Server(b, clock=clock)
    reqs = [_req(0, 0.0, 50), _req(1, 0.01, 5), _req(2, 0.02, 5)]
    rep = srv.run(reqs, duration=0.0, drain=True)
    assert sorted(r.rid for r in rep.completed) == [0, 1, 2]
    # some launch advanced the first case together with a later arrival
    assert any(0 in l and (1 in l or 2 in l) for l in b.launch_log)
    s = rep.summary()
    assert s["completed"] == 3 and s["backlog_at_end"] == 0
    assert s["p50_latency_s"] > 0 and s["p99_latency_s"] >= s["p50_latency_s"]
    assert s["mlups"] > 0


def test_poisson_arrivals_rate_and_order():
    t = serve.poisson_arrivals(rate=200.0, duration=20.0, seed=5)
    assert abs(len(t) / 20.0 - 200.0) < 200.0 * 0.1
    assert np.all(np.diff(t) > 0) and t[-1] < 20.0


def test_autotune_picks_fastest_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("WBLBE_TUNE_CACHE", str(tmp_path / "tune.json"))

    class TimedBatch(FakeBatch):
        def advance(self, n):
            import time
            # candidate (128, 32, 8) is the fastest per lattice update
            cost = {(128, 32, 8): 0.001}.get(tuple(self.cfg), 0.004)
            time.sleep(cost * n)
            super().advance(n)

    b = TimedBatch(slots=4)
    for k in range(3):
        b.admit(None, 10 ** 6, 0, 0)
    shapes = [(64, 64), (128, 96), (300, 200)]
    cands = [(64, 16, 8), (128, 32, 8), (256, 64, 8)]
    out = autotune.tune(b, shapes, "FakeGPU", candidates=cands, launches=2)
    assert out["config"] == [128, 32, 8] and not out["cached"]
    assert b.cfg == (128, 32, 8)
    stored = json.loads((tmp_path / "tune.json").read_text())
    assert list(stored.values())[0]["config"] == [128, 32, 8]
    b.set_config(64, 16, 1)
    again = autotune.tune(b, shapes, "FakeGPU", candidates=cands, launches=2)
    assert again["cached"] and b.cfg == (128, 32, 8)
    assert autotune.size_class(shapes) == autotune.size_class(list(reversed(shapes)))


class BoundedBatch(FakeBatch):
    """Refuses any case whose `need` exceeds `limit`, even when empty."""

    def __init__(self, slots, limit):
        super().__init__(slots)
        self.limit = limit

    def admit(self, params, rho, tol, max_steps):
        if int(rho) > self.limit:
            return None
        return super().admit(params, rho, tol, max_steps)


def test_request_that_never_fits_is_rejected_not_blocking():
    b = BoundedBatch(slots=1, limit=10)
    srv = serve.Server(b, clock=FakeClock())
    reqs = [_req(0, 0.0, 3), _req(1, 0.0, 50), _req(2, 0.0, 2)]
    rep = srv.run(reqs, duration=0.0, drain=True)
    assert sorted(r.rid for r in rep.completed) == [0, 2]
    assert [r.rid for r in rep.rejected] == [1] and rep.rejected[0].state == serve.REJECTED
    s = rep.summary()
    assert s["rejected"] == 1 and s["backlog_at_end"] == 0


def test_autotune_with_cases_that_stop_at_once(tmp_path, monkeypatch):
    """Every resident case stops during the first warm-up launch: nothing can
    be timed, the first candidate is kept and nothing is cached."""
    monkeypatch.setenv("WBLBE_TUNE_CACHE", str(tmp_path / "tune.json"))
    b = FakeBatch(slots=2)
    b.admit(None, 1, 0, 0)
    cands = [(64, 16, 8), (128, 32, 8)]
    out = autotune.tune(b, [(64, 64)], "FakeGPU", candidates=cands, launches=2)
    assert out["config"] == [64, 16, 8] and out["mlups"] is None and not out["cached"]
    assert b.cfg == (64, 16, 8) and not (tmp_path / "tune.json").exists()


class OutcomeBatch(FakeBatch):
    """Case k's outcome state is outcomes[k % len(outcomes)]."""

    def __init__(self, slots, outcomes):
        super().__init__(slots)
        self.outcomes = outcomes

    def admit(self, params, rho, tol, max_steps):
        cid = super().admit(params, rho, tol, max_steps)
        if cid is not None:
            self.cases[cid]["state"] = self.outcomes[cid % len(self.outcomes)]
        return cid


def test_latency_is_split_by_outcome_and_stop_after():
    """Converged, budget-exhausted and unstable requests are counted and
    timed separately; converged step counts are reported; stop_after ends
    the run once that many requests have completed."""
    b = OutcomeBatch(slots=16, outcomes=[serve.CONVERGED, serve.UNSTABLE, serve.CONVERGED,
                                         serve.BUDGET])
    srv = serve.Server(b, clock=FakeClock())
    reqs = [_req(k, 0.0, 1 + k) for k in range(12)]
    rep = srv.run(reqs, duration=1e9, stop_after=8)
    s = rep.summary()
    assert s["completed"] >= 8 and s["completed"] < 12
    n = {name: s[f"{name}_count"] for name in serve.OUTCOMES.values()}
    assert sum(n.values()) == s["completed"]
    assert n["converged"] == sum(1 for r in rep.completed if r.state == serve.CONVERGED) > 0
    assert n["unstable"] > 0 and n["budget"] > 0
    conv = rep.latencies(serve.CONVERGED)
    assert s["converged_p50_latency_s"] == float(np.percentile(conv, 50))
    steps = [r.steps for r in rep.completed if r.state == serve.CONVERGED]
    assert s["converged_p99_steps"] == float(np.percentile(steps, 99))


def test_time_cap_ends_a_drain():
    """A drain stops at the time cap, leaving the unfinished requests
    resident (reported as running at the end)."""
    b = FakeBatch(slots=4)
    clock = FakeClock()
    srv = serve.Server(b, clock=clock)
    reqs = [_req(k, 0.0, 10 ** 6 if k == 0 else 2) for k in range(3)]
    rep = srv.run(reqs, duration=0.0, drain=True, time_cap=0.5)
    s = rep.summary()
    assert s["completed"] == 2 and s["running_at_end"] == 1
    assert rep.elapsed >= 0.5
