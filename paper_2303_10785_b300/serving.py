"""Continuous-batching serving of simulation jobs on one GPU (not in the paper, whose solver
runs one job per GPU).

A job is a grid, an initial state and a number of SSP-RK3 steps.  The server keeps every
admitted job's state and metrics resident in one device-memory pool and advances all of
them together through one ``gbr.Batch`` (one launch per phase and kind, one CUDA graph per
step).  Jobs that arrive while others run wait in a FIFO queue and are admitted as soon as
a batch slot is free and the pool (``gbr.Arena``) has a free range of the job's
``gbr_workspace_bytes``; a finished job's result is copied to the host and its slot and
memory are released at once.  All device work of one job is the same arithmetic whether it
runs alone or in the mix, so results do not depend on the mix.

``run_serial`` is the plain per-job form used as the comparison: one job at a time, in
arrival order, through ``gbr_rk_step``.
"""
import collections
import ctypes
import time

import numpy as np

from . import gbr


class Job:
    """One request: host inputs, steps, time-step rule (CFL > 0 or fixed step < 0), arrival time."""

    def __init__(self, job_id, case, nodes, q, steps, cfl, arrival=0.0, inflow=None, sponge=None):
        self.id = job_id
        self.case = case
        self.nodes = nodes
        self.q = q
        self.steps = int(steps)
        self.cfl = float(cfl)
        self.arrival = float(arrival)
        self.inflow = inflow
        self.sponge = sponge
        self.cells = int(np.prod(case["n"][: case["ndim"]]))
        self.admitted = None
        self.finished = None
        self.result = None
        self.time = None
        self.error = None

    @property
    def work(self):
        """cell-RK-stage updates"""
        return self.cells * self.steps * 3

    def footprint(self):
        p = gbr.make_params(self.case)
        return int(gbr.lib().gbr_workspace_bytes(ctypes.byref(p)))

    def make_solver(self, stream, workspace=None):
        s = gbr.Solver(self.case, self.nodes, stream=stream, workspace=workspace)
        if self.inflow is not None:
            s.set_inflow(self.inflow)
        if self.sponge is not None:
            s.set_sponge(*self.sponge)
        s.set_state(self.q)
        return s


def latency_stats(jobs):
    """Time-to-N-steps of the completed jobs and their aggregate throughput; failed jobs (a state
    that went non-finite, a job that could not be admitted) are counted apart."""
    done = [j for j in jobs if j.finished is not None and j.error is None]
    lat = np.array([j.finished - j.arrival for j in done])
    work = sum(j.work for j in done)
    if lat.size == 0:
        return {}
    start = min(j.arrival for j in jobs)
    end = max(j.finished for j in done)
    return {"jobs": int(lat.size), "failed": sum(1 for j in jobs if j.error is not None),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "makespan_s": end - start,
            "cell_rk_stage_updates_per_s": work / max(end - start, 1e-9)}


class Server:
    """Continuous batching over one device pool.

    pool_bytes   device memory for the jobs' workspaces (admission by footprint)
    max_active   batch slots
    chunk_steps  most steps queued between two looks at the queue
    """

    def __init__(self, pool_bytes, max_active=64, device="cuda", chunk_steps=8, use_graph=True, autotune=True):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.stream = torch.cuda.current_stream(self.device)
        self.pool = torch.empty(int(pool_bytes) + 256, dtype=torch.uint8, device=self.device)
        base = (self.pool.data_ptr() + 255) & ~255
        self.arena = gbr.Arena(base, int(pool_bytes))
        self.batch = gbr.Batch(max_active, device=self.device, stream=self.stream, use_graph=use_graph,
                               autotune=autotune)
        self.max_active = int(max_active)
        self.chunk = int(chunk_steps)
        self.queue = collections.deque()
        self.active = []  # [job, solver, pointer, steps done]
        self.done = []
        self.peak_active = 0
        self.peak_pool = 0

    def submit(self, job, now=0.0):
        """Queue a job; one that could never fit in the pool is rejected at once."""
        if job.footprint() > self.arena.capacity:
            job.error = "workspace larger than the device pool"
            job.finished = now
            self.done.append(job)
            return
        self.queue.append(job)

    def _admit(self, now):
        while self.queue and len(self.active) < self.max_active:
            job = self.queue[0]
            need = job.footprint()
            ptr = self.arena.alloc(need)
            if ptr is None:
                break  # first in, first admitted: wait for memory
            self.queue.popleft()
            try:
                s = job.make_solver(self.stream, workspace=(ptr, need))
                self.batch.add(s, job.cfl)
            except gbr.GbrError as e:
                self.arena.free(ptr)
                job.error = str(e)
                job.finished = now
                self.done.append(job)
                continue
            job.admitted = now
            self.active.append([job, s, ptr, 0])
        self.peak_active = max(self.peak_active, len(self.active))
        self.peak_pool = max(self.peak_pool, self.arena.stats()["used"])

    def _retire(self, clock):
        keep = []
        for entry in self.active:
            job, s, ptr, n = entry
            if n < job.steps:
                keep.append(entry)
                continue
            self.batch.remove(s)
            job.result = s.get_state()
            job.time = s.time()[0]
            job.finished = clock()
            s.close()
            self.arena.free(ptr)
            self.done.append(job)
        self.active = keep

    def _fail(self, entry, why, now):
        job, s, ptr, _ = entry
        self.batch.remove(s)
        s.close()
        self.arena.free(ptr)
        job.error = why
        job.finished = now
        self.done.append(job)
        self.active.remove(entry)

    def _sync_isolating(self, clock):
        """Drain the batch; a member whose state went non-finite fails alone (its job is retired
        with the error and its memory freed) and the others carry on."""
        while True:
            try:
                self.batch.sync()
                return
            except gbr.GbrError as e:
                if e.status != gbr.GBR_ENONFINITE or e.member < 0:
                    raise
                bad = self.batch.members[e.member]
                entry = next(x for x in self.active if x[1] is bad)
                self._fail(entry, f"job {entry[0].id}: {e}", clock())

    def run(self, jobs, clock=None, t0=None):
        """Serve `jobs` (their .arrival in seconds from the start); returns them when all are done."""
        clock = clock or time.perf_counter
        start = clock() if t0 is None else t0
        pending = sorted(jobs, key=lambda j: j.arrival)
        for j in pending:
            j.arrival += start  # absolute clock time
        i = 0
        while i < len(pending) or self.queue or self.active:
            now = clock()
            while i < len(pending) and pending[i].arrival <= now:
                self.submit(pending[i], now)
                i += 1
            self._admit(now)
            if not self.active:
                if i < len(pending):
                    time.sleep(max(0.0, min(pending[i].arrival - clock(), 0.01)))
                continue
            k = min(self.chunk, min(job.steps - n for job, _, _, n in self.active))
            self.batch.step(k)
            self._sync_isolating(clock)
            for entry in self.active:
                entry[3] += k
            self._retire(clock)
        for j in jobs:
            j.arrival -= start
            if j.finished is not None:
                j.finished -= start
            if j.admitted is not None:
                j.admitted -= start
        return jobs

    def close(self):
        for job, s, ptr, _ in self.active:
            s.close()
        self.active = []
        self.batch.close()
        self.arena.close()


def run_serial(jobs, device="cuda", precision=None, clock=None):
    """The plain per-job form: one job at a time in arrival order through gbr_rk_step (optionally
    forcing every job's precision, e.g. "fp64")."""
    import torch

    clock = clock or time.perf_counter
    stream = torch.cuda.current_stream(torch.device(device))
    start = clock()
    for job in sorted(jobs, key=lambda j: j.arrival):
        wait = start + job.arrival - clock()
        if wait > 0:
            time.sleep(wait)
        if precision is not None:
            job.case = dict(job.case, precision=precision)
        job.admitted = clock() - start
        s = job.make_solver(stream)
        for _ in range(job.steps):
            s.rk_step(job.cfl)
        try:
            s.sync()
            job.result = s.get_state()
            job.time = s.time()[0]
        except gbr.GbrError as e:  # this job's state went bad: it fails alone
            if e.status != gbr.GBR_ENONFINITE:
                raise
            job.error = f"job {job.id}: {e}"
        job.finished = clock() - start
        s.close()
    return jobs
