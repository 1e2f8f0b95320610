"""Host logic of the continuous-batching service, without a GPU: the library
calls are replaced by fakes that record what the service asks of them.
Requests are admitted first come, first served while their footprint (with
the margin) fits the budget; a request waits, and holds back the ones behind
it, until retirements free enough memory; every request advances one step per
tick until its own step count; a request larger than the whole budget is
refused before anything runs; latencies and throughput are summarised from
what the ticks recorded."""
import numpy as np
import pytest

from paper_1302_3663_gb300 import bfibm, serve, workloads


class FakeCtx:
    dim = 3

    def __init__(self, inst):
        self.inst = inst
        self.closed = False
        self.steps = 0

    def set_option(self, option, value):
        pass

    def get_velocity(self, d):
        return np.zeros(2)

    def get_pressure(self):
        return np.zeros(2)

    def get_nodes(self):
        return np.zeros((1, 3))

    def get_broken(self):
        return []

    def close(self):
        self.closed = True


class FakeBatch:
    """Records the slots stepped at each tick and the memory they hold."""

    def __init__(self, persistent=False, tune=True):
        self.slots = {}
        self.next = 0
        self.ticks = []

    def add(self, ctx):
        slot = self.next
        self.next += 1
        self.slots[slot] = ctx
        return slot

    def remove(self, slot):
        del self.slots[slot]

    def step(self):
        self.ticks.append(sorted(self.slots))
        for ctx in self.slots.values():
            ctx.steps += 1

    def wait(self):
        return bfibm.OK

    def slot_ms(self, slot):
        return 2.0 + slot

    def close(self):
        self.slots.clear()


@pytest.fixture
def fakes(monkeypatch):
    made = []

    def load_instance(inst):
        c = FakeCtx(inst)
        made.append(c)
        return c

    monkeypatch.setattr(bfibm, "load_instance", load_instance)
    monkeypatch.setattr(bfibm, "Batch", FakeBatch)
    monkeypatch.setattr(bfibm, "footprint", lambda prm, eta, m: prm["fp"])
    monkeypatch.setattr(workloads, "cells", lambda prm: prm["cells"])
    return made


def request(rid, fp, steps, arrival=0.0, cells=1000):
    inst = {"params": {"fp": fp, "cells": cells}, "X": np.zeros((5, 3)), "ab": np.zeros((4, 2))}
    return serve.Request(rid, inst, steps, arrival)


def test_first_come_first_served_within_the_budget(fakes):
    # budget 100 with a 5 % margin: 40 + 40 fit (84), the third (42) waits for
    # a retirement, and the fourth (small) waits behind it although it fits
    reqs = [request(0, 40, 3), request(1, 40, 5), request(2, 40, 2), request(3, 5, 2)]
    srv = serve.Server(100)
    done = srv.run(reqs)
    assert sorted(r.rid for r in done) == [0, 1, 2, 3]
    ticks = srv.batch.ticks
    assert ticks[0] == [0, 1]
    # request 0 retires after its 3 steps: 2 and 3 join on the next tick
    assert ticks[3] == [1, 2, 3]
    for r in reqs:
        assert r.done == r.steps and len(r.step_ms) == r.steps
        assert r.admitted is not None and r.finished >= r.admitted
    # every context was closed, the memory given back, nothing left active
    assert all(c.closed for c in fakes)
    assert srv.used == 0 and not srv.active
    # at no tick did the admitted footprints exceed the budget
    fp = {r.rid: int(r.footprint * srv.margin) for r in reqs}
    assert all(sum(fp[s] for s in t) <= 100 for t in ticks)
    srv.close()


def test_a_request_larger_than_the_budget_is_refused(fakes):
    srv = serve.Server(100)
    with pytest.raises(ValueError):
        srv.run([request(0, 10, 1), request(1, 99, 1)])   # 99 * 1.05 > 100
    assert not fakes   # nothing was admitted
    srv.close()


def test_later_arrivals_wait_for_their_time(fakes):
    reqs = [request(0, 10, 2, arrival=0.0), request(1, 10, 2, arrival=0.15)]
    srv = serve.Server(1000)
    done = srv.run(reqs)
    assert [r.rid for r in done] == [0, 1]
    assert reqs[1].admitted >= 0.15
    srv.close()


def test_results_are_kept_and_summarised(fakes):
    reqs = [request(0, 10, 3, cells=100), request(1, 10, 1, cells=50)]
    srv = serve.Server(1000)
    done = srv.run(reqs)
    assert all(r.result is not None and set(r.result) == {"u", "p", "X", "broken"}
               for r in done)
    out = serve.summarize(done, 2.0, busy=1.0)
    assert out["requests"] == 2
    assert out["cell_steps"] == 3 * 100 + 1 * 50
    assert out["cell_steps_per_s"] == pytest.approx(350 / 2.0)
    assert out["cell_steps_per_busy_s"] == pytest.approx(350.0)
    lat = np.array(reqs[0].step_ms + reqs[1].step_ms)
    assert out["step_ms_p50"] == pytest.approx(np.percentile(lat, 50))
    assert out["step_ms_p99"] == pytest.approx(np.percentile(lat, 99))
    srv.close()


def test_max_ticks_stops_the_loop(fakes):
    srv = serve.Server(1000, keep_results=False)
    done = srv.run([request(0, 10, 50)], max_ticks=4)
    assert not done and srv.ticks == 4
    srv.close()
    assert all(c.closed for c in fakes)
