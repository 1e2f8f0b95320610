"""Continuous-batching service for independent biofilm simulations.

Requests (a parameter set, nodes and springs, and a number of time steps)
arrive over time. A request is admitted as soon as its device footprint fits
the memory budget (first come, first served); it then keeps its grids and
node state on the device and advances one time step per tick together with
every other admitted simulation (one ``bfibm_batch_step`` per tick: each
simulation replaying its step graph on its own stream, or, with
``persistent``, all of them in lock step, each multigrid level of their
solves one launch over all of them). Finished simulations
hand back their results and free their memory, which admits waiting
requests. Per-request step latencies come from CUDA events around each
simulation's step.
"""
import collections
import time

import numpy as np

from . import bfibm, workloads


class Request:
    def __init__(self, rid, inst, steps, arrival):
        self.rid = rid
        self.inst = inst
        self.steps = steps
        self.arrival = arrival
        self.footprint = bfibm.footprint(inst["params"], inst["X"].shape[0], inst["ab"].shape[0])
        self.cells = workloads.cells(inst["params"])
        self.admitted = None
        self.finished = None
        self.done = 0
        self.step_ms = []
        self.result = None


class Server:
    """Admission by device-memory footprint, continuous batching of steps."""

    def __init__(self, budget_bytes, keep_results=True, margin=1.05, persistent=False):
        self.budget = int(budget_bytes)
        self.margin = margin
        self.keep_results = keep_results
        # the persistent plan is rebuilt whenever a request joins or leaves, so
        # its sweep shapes keep the built-in choice instead of being timed
        self.batch = bfibm.Batch(persistent=persistent, tune=False)
        self.used = 0
        self.active = {}          # slot -> (request, context)
        self.ticks = 0
        self.busy = 0.0           # seconds from each tick's launch to its completion

    def _admit(self, req, now):
        ctx = bfibm.load_instance(req.inst)
        ctx.set_option(bfibm.OPT_STATS, 0)
        slot = self.batch.add(ctx)
        self.active[slot] = (req, ctx)
        self.used += int(req.footprint * self.margin)
        req.admitted = now

    def _retire(self, slot, now):
        req, ctx = self.active.pop(slot)
        self.batch.remove(slot)
        if self.keep_results:
            req.result = {"u": [ctx.get_velocity(d) for d in range(ctx.dim)],
                          "p": ctx.get_pressure(), "X": ctx.get_nodes(),
                          "broken": ctx.get_broken()}
        ctx.close()
        self.used -= int(req.footprint * self.margin)
        req.finished = now

    def run(self, requests, clock=time.perf_counter, max_ticks=None):
        """Serve requests (sorted by arrival time, seconds from start) until
        all are done. Returns the finished requests."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        finished = []
        t0 = clock()
        for r in pending:
            if int(r.footprint * self.margin) > self.budget:
                raise ValueError("request %s needs more memory than the whole budget" % r.rid)
        while pending or waiting or self.active:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            while waiting and self.used + int(waiting[0].footprint * self.margin) <= self.budget:
                self._admit(waiting.popleft(), now)
            if not self.active:
                if pending:
                    time.sleep(max(0.0, min(0.05, pending[0].arrival - now)))
                continue
            tb = clock()
            self.batch.step()
            self.batch.wait()
            self.ticks += 1
            self.busy += clock() - tb
            now = clock() - t0
            for slot in list(self.active):
                req, _ = self.active[slot]
                req.step_ms.append(self.batch.slot_ms(slot))
                req.done += 1
                if req.done >= req.steps:
                    self._retire(slot, now)
                    finished.append(req)
            if max_ticks is not None and self.ticks >= max_ticks:
                break
        self.elapsed = clock() - t0
        return finished

    def close(self):
        for slot in list(self.active):
            self._retire(slot, 0.0)
        self.batch.close()


def summarize(finished, elapsed, busy=None):
    """Throughput over the wall-clock span of the stream (arrival gaps
    included) and, given the server's busy time, over the ticks alone."""
    lat = np.concatenate([np.asarray(r.step_ms) for r in finished]) if finished else np.zeros(1)
    cell_steps = sum(r.cells * r.done for r in finished)
    turnaround = [r.finished - r.arrival for r in finished]
    queued = [r.admitted - r.arrival for r in finished]
    out = {"requests": len(finished), "cell_steps": cell_steps,
            "cell_steps_per_s": cell_steps / elapsed if elapsed > 0 else 0.0,
            "step_ms_p50": float(np.percentile(lat, 50)),
            "step_ms_p99": float(np.percentile(lat, 99)),
            "turnaround_s_p50": float(np.percentile(turnaround, 50)) if turnaround else 0.0,
            "queue_s_max": float(max(queued)) if queued else 0.0,
            "elapsed_s": elapsed}
    if busy is not None:
        out["busy_s"] = busy
        out["cell_steps_per_busy_s"] = cell_steps / busy if busy > 0 else 0.0
    return out


def serial(requests, precision=None, params=None, checks=None):
    """The same requests one after another, each alone (the baseline the
    service is compared with): one untimed step (it captures the step graph),
    then the request's steps timed on the device. Returns cell-steps per
    second of device time and the total device milliseconds; `checks`, a
    list, receives each request's statistics after its steps."""
    import torch
    total_ms = 0.0
    cell_steps = 0
    for r in requests:
        prm = dict(r.inst["params"])
        if params:
            prm.update(params)
        if precision is not None:
            prm["precision"] = precision
        s = torch.cuda.Stream()
        ctx = bfibm.load_instance(r.inst, stream=s, prm_override=prm)
        ctx.set_option(bfibm.OPT_STATS, 0)
        ctx.step(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        ctx.step(r.steps)
        e1.record(s)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        cell_steps += r.cells * r.steps
        if checks is not None:
            checks.append(ctx.get_stats())
        ctx.close()
    return cell_steps / (total_ms / 1e3), total_ms
