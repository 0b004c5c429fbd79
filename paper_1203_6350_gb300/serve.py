"""Continuous-batching server for lattice sweep jobs.

Jobs (a lattice problem plus its number of steps) arrive over time.  The
server keeps every admitted job's populations resident on the device, admits
waiting jobs in arrival order whenever their device memory fits under the HBM
budget, advances all resident jobs together (one batched launch per time step
and storage type for the small ones, graph-replayed chunks on a pool of
streams for the larger ones, so that lattices too small to fill the GPU run
side by side), and retires each job as soon as it has
taken its own number of steps, which frees memory for the next ones.  A job
added while others are running starts in the next chunk and shares their
launches; each job still takes exactly its own steps, so its result is the
same alone and in the mix.

Failures stay with their job.  A job the library refuses at admission (an
invalid problem, a failed allocation) is reported with its error and takes
no memory; a job whose state has gone non-finite is reported as such when it
is read out.  The other jobs carry on either way.

:func:`serial_loop` is the comparison: the same jobs one after another through
the single-lattice API.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import lbm
from .batch import Batch


@dataclass
class Job:
    id: int
    workload: object            # workloads.Workload (its storage field selects the format)
    arrival: float = 0.0        # seconds after the start of the run
    admitted: Optional[float] = None
    admitted_round: int = 0
    finished: Optional[float] = None
    result: Optional[np.ndarray] = None   # lbm diagnostics over the layer-free interior
    field: Optional[np.ndarray] = None    # final rho' (when the server keeps fields)
    error: Optional[str] = None           # why the job failed (None: it did not)
    charged: int = 0                      # device bytes counted against the budget while resident

    @property
    def latency(self) -> Optional[float]:
        return None if self.finished is None else self.finished - self.arrival

    @property
    def bytes(self) -> int:
        """Device bytes of the job as a batch instance."""
        w = self.workload
        return lbm.lbm_batch_instance_bytes(w.nx, w.ny, lbm.STORAGE[w.storage])

    def lattice_bytes(self, host_io: bool) -> int:
        """Device bytes of the job as a single lattice (its own diagnostics
        buffers and flags, and with host_io the FP64 staging of host transfers)."""
        w = self.workload
        return lbm.lbm_lattice_bytes(w.nx, w.ny, lbm.STORAGE[w.storage], lbm.BC[w.bc],
                                     1 if host_io else 0)


def interior(w):
    W = w.width
    return (W, W, w.nx - W, w.ny - W) if 2 * W < min(w.nx, w.ny) else (0, 0, w.nx, w.ny)


class Server:
    def __init__(self, hbm_budget: float = 150e9, chunk: int = 64, keep_fields=False,
                 tiling: Optional[tuple] = None, device: int = 0, stream=None,
                 max_resident_cells: Optional[int] = 8 << 20, init: str = "pulse",
                 solo_cells: Optional[int] = 1 << 14, batch_config: Optional[dict] = None,
                 streams: int = 8):
        """hbm_budget: device bytes the resident jobs may hold.  max_resident_cells:
        slot limit -- jobs are admitted while the resident lattices hold fewer
        cells than this (enough to keep the GPU's bandwidth busy; more only
        stretches every job's latency), always at least one job.  On the
        serving trace with 8 streams, 8M cells measured 27.3 solves/s (p50
        1.86 s), against 26.8 with 4M and 27.4 with 16M (p50 1.94 s).  init: "pulse"
        builds each job's initial pulse on the device, "fields" uploads it.
        solo_cells: a lattice this large runs through the single-lattice kernel
        (chunk by chunk as graph replays, on its own stream beside the batched
        launch of the smaller resident jobs); None sends every job through the
        batch.  The default, 16384 cells (128^2), batches only lattices too
        small to keep the GPU busy on their own: on the serving trace (one
        stream, 4M-cell limit), the graph-replayed chunks of jobs from 128^2 up
        measured faster than sharing a batched launch (24.2 against 22.5
        solves/s with a 1M-cell threshold).  A job's path depends only on its
        size, so its result does not depend on what else is resident.
        batch_config: kernel of the batched launches ({"cells", "steps_per_launch",
        "tile"}, as autotune.tuned_config gives); default: two cells per thread
        and two steps per launch for FP32 and 16-bit storage (the fastest on
        the mixed-size 256-lattice workload), the batch default for FP64;
        tiling overrides the tile of one-step launches.  streams: the
        single-lattice jobs step on this many streams, round robin, so that
        lattices too small to fill the GPU run side by side; each stream
        joins the stepping stream after every chunk.  On the serving trace
        (4M-cell limit) 1, 2, 4 and 8 streams measured 24.2, 25.9, 26.6 and
        26.8 solves/s."""
        import torch

        self.torch = torch
        self.solo_cells = solo_cells
        self.max_cells = max_resident_cells
        self.init = init
        self.cells = 0
        self.budget = float(hbm_budget)
        self.chunk = int(chunk)
        self.keep_fields = keep_fields
        self.tiling = tiling
        self.batch_config = batch_config
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.Stream(device)
        self.side = torch.cuda.Stream(device)  # set-up and read-out, off the stepping stream
        self.solo_streams = [torch.cuda.Stream(device) for _ in range(max(1, int(streams)))]
        self.admitted = 0
        self.batches = {}
        self.pending = deque()
        self.resident = {}  # job id -> (storage, instance id, job)
        self.used = 0
        self.done = []
        self.steps_run = 0
        self.round = 0

    def _batch(self, storage) -> Batch:
        if storage not in self.batches:
            cfg = self.batch_config
            if cfg is None and storage != "f64":
                cfg = {"cells": 2, "steps_per_launch": 2, "tile": self.tiling or (64, 16)}
            self.batches[storage] = Batch(storage, stream=self.stream, device=self.device,
                                          tiling=self.tiling, config=cfg)
        return self.batches[storage]

    def _solo(self, job: Job) -> bool:
        return self.solo_cells is not None and job.workload.cells >= self.solo_cells

    def charge(self, job: Job) -> int:
        """Device bytes the job holds while resident: a single lattice (with the
        staging of host transfers when fields are uploaded or read back) or a
        batch instance, by the path its size selects."""
        if self._solo(job):
            return job.lattice_bytes(self.init == "fields" or bool(self.keep_fields))
        return job.bytes

    def submit(self, job: Job) -> None:
        need = self.charge(job)
        if need > self.budget:
            raise ValueError(f"job {job.id} needs {need} bytes, more than the budget")
        self.pending.append(job)

    def admit(self, now: float) -> int:
        n = 0
        while self.pending and self.used + self.charge(self.pending[0]) <= self.budget:
            if (self.max_cells is not None and self.resident
                    and self.cells >= self.max_cells):
                break
            job = self.pending.popleft()
            w = job.workload
            try:
                if self._solo(job):
                    # created and initialised on the side stream (lbm_create waits
                    # for its stream), then handed to the stepping stream
                    lat = lbm.Lattice.from_workload(w, init=self.init, stream=self.side,
                                                    device=self.device)
                    st = self.solo_streams[self.admitted % len(self.solo_streams)]
                    st.wait_stream(self.side)
                    lat.set_stream(st)
                    self.resident[job.id] = ("solo", lat, job)
                else:
                    b = self._batch(w.storage)
                    i = b.add_workload(w, steps=w.steps, init=self.init)
                    self.resident[job.id] = (w.storage, i, job)
            except lbm.LbmError as e:  # refused: reported, holds nothing
                job.error = f"admission failed: {e}"
                job.finished = now
                self.done.append(job)
                continue
            job.charged = self.charge(job)
            self.used += job.charged
            self.cells += w.cells
            self.admitted += 1
            job.admitted = now
            job.admitted_round = self.round
            n += 1
        return n

    def _complete(self, st, h, job) -> bool:
        """Has every step of the job been issued?"""
        t = h.time if st == "solo" else self.batches[st].time(h)
        return t >= job.workload.steps

    def retire(self, clock, ids, after) -> int:
        """Read out and release the jobs `ids`, whose last steps were issued
        before the event `after`.  The read-out runs on the side stream, which
        waits for `after` only, so the chunk issued since keeps the GPU busy
        while the host waits for the results."""
        if not ids:
            return 0
        if after is not None:
            self.side.wait_event(after)
        else:
            self.side.wait_stream(self.stream)
        for jid in ids:
            st, h, job = self.resident.pop(jid)
            keep = self.keep_fields
            keep = keep is True or (isinstance(keep, (set, frozenset)) and job.id in keep)
            if st == "solo":
                h.set_stream(self.side)
                job.result = h.diagnostics(interior(job.workload))
                if keep:
                    job.field = h.moments()[0]
                h.close()  # waits for the side stream only
            else:
                b = self.batches[st]
                b.set_stream(self.side)
                job.result = b.diagnostics(h, interior(job.workload))
                if keep:
                    job.field = b.moments(h)[0]
                b.set_stream(self.stream)
                b.remove(h)  # freed once the launches issued so far have completed
            if job.result[5] > 0:
                job.error = (f"non-finite rho' or u in {int(job.result[5])} cells of the "
                             "read-out region")
            self.used -= job.charged
            self.cells -= job.workload.cells
            job.finished = clock()
            self.done.append(job)
        return len(ids)

    def advance(self) -> bool:
        """Issue one chunk of steps for every resident job that still needs
        steps; False if none does."""
        busy = False
        with self.torch.cuda.stream(self.stream):
            for st, b in self.batches.items():
                if len(b) and any(s == st and not self._complete(s, h, j)
                                  for s, h, j in self.resident.values()):
                    b.step(self.chunk)
                    busy = True
            for st, lat, job in self.resident.values():
                if st == "solo":
                    n = min(self.chunk, job.workload.steps - lat.time)
                    if n > 0:
                        lat.step(n)  # on the job's own stream
                        busy = True
            for st in self.solo_streams:  # this chunk's event covers every stream
                self.stream.wait_stream(st)
        if busy:
            self.steps_run += self.chunk
        return busy

    def run(self, jobs, realtime: bool = True):
        """Serve `jobs` (sorted by arrival).  realtime: arrivals follow the wall
        clock; otherwise every job is submitted at once in arrival order.

        Each round: admit what fits, note the resident jobs whose steps have all
        been issued, issue the next chunk for the others, then read out and
        release the noted ones (on the side stream, behind the event of the
        previous chunk)."""
        jobs = sorted(jobs, key=lambda j: j.arrival)
        t0 = time.perf_counter()

        def clock():
            return time.perf_counter() - t0

        k = 0
        prev = None  # event after the last chunk issued
        while k < len(jobs) or self.pending or self.resident:
            now = clock()
            while k < len(jobs) and (not realtime or jobs[k].arrival <= now):
                self.submit(jobs[k])
                k += 1
            self.round += 1
            self.admit(now)
            if not self.resident:
                if k < len(jobs) and realtime:
                    time.sleep(max(0.0, jobs[k].arrival - clock()))
                continue
            # jobs admitted this round are read out next round at the earliest, so
            # that the read-out is ordered after their initialisation
            finished = [jid for jid, (st, h, job) in self.resident.items()
                        if job.admitted_round < self.round and self._complete(st, h, job)]
            self.advance()
            ev = self.torch.cuda.Event()
            ev.record(self.stream)  # also covers this round's initialisations
            self.retire(clock, finished, prev)
            prev = ev
        self.stream.synchronize()
        self.side.synchronize()
        return self.done

    def close(self) -> None:
        for st, h, _ in self.resident.values():
            if st == "solo":
                h.close()
        self.resident.clear()
        for b in self.batches.values():
            b.close()
        self.batches.clear()


def serial_loop(jobs, keep_fields: bool = False, realtime: bool = True, init: str = "pulse",
                launch: str = "graph"):
    """The same jobs one after another, in arrival order, through lbm_create /
    lbm_step / lbm_diagnostics / lbm_destroy.  launch="plain": one kernel launch
    per step; "graph" (the library default): graph-replayed dependent launches."""
    jobs = sorted(jobs, key=lambda j: j.arrival)
    t0 = time.perf_counter()
    for job in jobs:
        if realtime:
            time.sleep(max(0.0, job.arrival - (time.perf_counter() - t0)))
        w = job.workload
        job.admitted = time.perf_counter() - t0
        with lbm.Lattice.from_workload(w, init=init) as lat:
            lbm.check(lbm.lbm_set_launch_mode(lat.h, lbm.LAUNCH_MODES[launch]), lat.h, "launch")
            lat.step(w.steps)
            job.result = lat.diagnostics(interior(w))
            if keep_fields:
                job.field = lat.moments()[0]
        job.finished = time.perf_counter() - t0
    return jobs


def summary(jobs, wall: float) -> dict:
    """Throughput and latency of the solved jobs (those with a result; jobs
    refused at admission count as failed)."""
    solved = [j for j in jobs if j.result is not None]
    lat = np.array([j.latency for j in solved if j.latency is not None])
    cells = sum(j.workload.cells * j.workload.steps for j in solved)
    return {
        "jobs": len(solved), "failed": len(jobs) - len(solved), "wall_s": wall,
        "solves_per_s": len(solved) / wall if wall > 0 else None,
        "mlups": cells / wall / 1e6 if wall > 0 else None,
        "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
        "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
    }
