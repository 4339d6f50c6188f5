"""Host logic of the serving loop and the batch runner, on CPU, against a fake
instance (no GPU): first-come-first-served admission by footprint, the budget,
rejection of requests that can never fit, phase order (drag, relax, ...) and
the per-request accounting."""
import numpy as np
import pytest

from paper_2105_10576_gb300 import batch, serve


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3      # every look at the clock costs 1 ms of fake time
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


class FakeSim:
    log = []
    live = 0
    clock = None

    def __init__(self, params, solid, alpha0, stream=0):
        self.p = params
        self.pending = None
        self.ready_at = 0.0
        self.closed = False
        FakeSim.live += 1
        FakeSim.log.append(("create", params["rid"]))

    def stats(self):
        assert self.pending is None, "a pending handle accepts only wait"
        return {"n_fluid": self.p["n_fluid"], "device_bytes": self.p["fake_bytes"]}

    def _launch(self, kind):
        assert self.pending is None
        self.pending = kind
        self.ready_at = FakeSim.clock.t + self.p["dur"]
        FakeSim.log.append((kind, self.p["rid"]))
        return 0

    def drag_step_async(self, dt):
        return self._launch("drag")

    def relax_async(self, dt, N):
        return self._launch("relax")

    def query(self):
        assert self.pending is not None
        return FakeSim.clock.t >= self.ready_at

    def wait(self, strict=True):
        assert self.pending is not None
        kind, self.pending = self.pending, None
        return 0, (self.p["kf"] if kind == "relax" else 1), 0.0

    def field(self, which):
        return np.full(4, float(self.p["rid"]))

    def close(self):
        assert not self.closed
        self.closed = True
        FakeSim.live -= 1


@pytest.fixture
def fake(monkeypatch):
    clk = Clock()
    FakeSim.log, FakeSim.live, FakeSim.clock = [], 0, clk
    monkeypatch.setattr(serve.ox, "Oscar", FakeSim)
    monkeypatch.setattr(serve.ox, "oscar_footprint", lambda p: p["fake_bytes"])
    monkeypatch.setattr(serve.time, "sleep", clk.sleep)
    return clk


def req(rid, arrival, nbytes, steps=2, kf=3, dur=0.01, n_fluid=100):
    p = {"rid": rid, "fake_bytes": nbytes, "kf": kf, "dur": dur, "n_fluid": n_fluid}
    return serve.Request(rid, arrival, p, None, None, 1e-6, 1e-7, 5, steps)


def test_fifo_admission_within_budget(fake):
    reqs = [req(0, 0.0, 60), req(1, 0.0, 50), req(2, 0.0, 30), req(3, 0.005, 40)]
    srv = serve.Server(budget_bytes=100, clock=fake)
    recs = srv.run(reqs, keep_alpha=True)
    assert srv.max_used <= 100 and FakeSim.live == 0
    creates = [rid for op, rid in FakeSim.log if op == "create"]
    assert creates == [0, 1, 2, 3]          # first come, first served (request 2 waits behind 1)
    for rec in recs:
        assert rec.status == 0 and rec.k_f == [3, 3]
        assert rec.cell_updates == 100 * 2 * (1 + 3)
        assert rec.done >= rec.admitted >= rec.arrival
        assert rec.alpha[0] == rec.rid
    # each instance alternates drag and relax
    for rid in range(4):
        ops = [op for op, r in FakeSim.log if r == rid and op != "create"]
        assert ops == ["drag", "relax", "drag", "relax"]


def test_request_larger_than_budget_is_rejected(fake):
    reqs = [req(0, 0.0, 500), req(1, 0.0, 40)]
    recs = serve.Server(budget_bytes=100, clock=fake).run(reqs)
    assert recs[0].status == -1 and recs[0].done < 0
    assert recs[1].status == 0 and recs[1].k_f == [3, 3]


def test_batch_steps_every_instance(fake):
    sims = [FakeSim({"rid": q, "fake_bytes": 1, "kf": q + 1, "dur": 0.0, "n_fluid": 1}, None, None)
            for q in range(3)]
    b = batch.Batch(sims)
    assert b.step([1e-6] * 3, [1e-7] * 3, [5] * 3) == [1, 2, 3]
    b.close()
    assert FakeSim.live == 0
