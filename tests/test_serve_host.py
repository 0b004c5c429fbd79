"""The server's host logic on the CPU: admission in arrival order under the
memory budget and the slot limit, failures at admission (host-side fakes of
a failed allocation and of a refused problem) reported with their job while
the rest are admitted, and the summary's accounting of solved and failed
jobs.  The device side is replaced by fakes; nothing here touches a GPU."""
from dataclasses import dataclass

import numpy as np
import pytest

import workloads as wl
from paper_1203_6350_gb300 import lbm
from paper_1203_6350_gb300 import serve
from paper_1203_6350_gb300.serve import Job, Server, interior, summary


@dataclass
class FJob(Job):
    nbytes: int = 0

    @property
    def bytes(self) -> int:
        return self.nbytes

    def lattice_bytes(self, host_io):
        return self.nbytes


class FakeStream:
    def wait_stream(self, other):
        pass


class FakeLattice:
    def __init__(self, w):
        self.w, self.time = w, 0

    def set_stream(self, s):
        self.stream = s


class FakeBatch:
    def __init__(self, refuse):
        self.refuse, self.ids = refuse, []

    def add_workload(self, w, steps=None, init=None):
        if w.name in self.refuse:
            raise lbm.LbmError(lbm.LBM_ERR_OOM, "instance allocation failed (fake)")
        self.ids.append(w.name)
        return len(self.ids) - 1


def _server(budget, max_cells, solo_cells, refuse_solo=(), refuse_batch=(), monkeypatch=None):
    srv = Server.__new__(Server)  # no device: streams and lattices are fakes
    srv.pending, srv.resident, srv.done, srv.batches = serve.deque(), {}, [], {}
    srv.used, srv.cells, srv.admitted, srv.round = 0, 0, 0, 0
    srv.budget, srv.max_cells, srv.solo_cells = float(budget), max_cells, solo_cells
    srv.init, srv.device, srv.keep_fields = "pulse", 0, False
    srv.stream, srv.side = FakeStream(), FakeStream()
    srv.solo_streams = [FakeStream() for _ in range(3)]
    fb = FakeBatch(set(refuse_batch))
    srv._batch = lambda storage: fb

    def fake_from_workload(w, **kw):
        if w.name in refuse_solo:
            raise lbm.LbmError(lbm.LBM_ERR_ARG, "refused problem (fake)")
        return FakeLattice(w)

    monkeypatch.setattr(lbm.Lattice, "from_workload", staticmethod(fake_from_workload))
    return srv, fb


def _job(k, side, nbytes):
    w = wl.pulse_workload(side, side, steps=10, name=f"job{k}")
    return FJob(id=k, workload=w, arrival=0.001 * k, nbytes=nbytes)


def test_admission_follows_arrival_order_under_the_budget(monkeypatch):
    srv, _ = _server(budget=100, max_cells=None, solo_cells=None, monkeypatch=monkeypatch)
    for k, b in enumerate([40, 50, 30, 5]):
        srv.submit(_job(k, 16, b))
    assert srv.admit(0.0) == 2          # 40 + 50; the third (30) does not fit
    assert srv.used == 90 and [j.id for j in srv.pending] == [2, 3]
    # head of line: the 5-byte job behind it waits too, in arrival order
    st, h, job = srv.resident.pop(0)
    srv.used -= job.bytes
    srv.cells -= job.workload.cells
    assert srv.admit(0.1) == 2 and srv.used == 85 and not srv.pending


def test_slot_limit_admits_at_least_one_job(monkeypatch):
    srv, _ = _server(budget=1e9, max_cells=300, solo_cells=None, monkeypatch=monkeypatch)
    srv.submit(_job(0, 20, 1))           # 400 cells: over the limit, admitted alone
    srv.submit(_job(1, 10, 1))
    assert srv.admit(0.0) == 1 and srv.cells == 400
    srv.resident.clear()
    srv.cells = 0
    assert srv.admit(0.1) == 1


def test_refused_jobs_are_reported_and_hold_nothing(monkeypatch):
    srv, fb = _server(budget=1e9, max_cells=None, solo_cells=200,
                      refuse_solo={"job1"}, refuse_batch={"job3"}, monkeypatch=monkeypatch)
    sides = [20, 20, 10, 10, 20]         # 400-cell jobs run solo, 100-cell jobs batched
    for k, side in enumerate(sides):
        srv.submit(_job(k, side, 7))
    assert srv.admit(0.5) == 3
    assert sorted(srv.resident) == [0, 2, 4]
    assert srv.used == 21 and srv.cells == 400 + 100 + 400
    failed = {j.id: j for j in srv.done}
    assert sorted(failed) == [1, 3]
    assert "refused problem" in failed[1].error and failed[1].finished == 0.5
    assert "allocation failed" in failed[3].error and failed[3].result is None
    assert fb.ids == ["job2"]
    # solo jobs spread over the stream pool, round robin
    streams = [srv.resident[k][1].stream for k in (0, 4)]
    assert streams[0] is not streams[1]


def test_summary_counts_solved_and_failed_jobs():
    jobs = [_job(k, 10, 1) for k in range(4)]
    for k, j in enumerate(jobs):
        j.finished = j.arrival + 1.0 + k
        j.result = np.zeros(6) if k != 2 else None
        j.error = "admission failed: fake" if k == 2 else None
    s = summary(jobs, 2.0)
    assert s["jobs"] == 3 and s["failed"] == 1
    assert s["solves_per_s"] == pytest.approx(1.5)
    assert s["mlups"] == pytest.approx(3 * 100 * 10 / 2.0 / 1e6)
    assert s["p50_s"] == pytest.approx(2.0)


def test_interior_excludes_the_layer():
    w = wl.pulse_workload(100, 60, width=20)
    assert interior(w) == (20, 20, 80, 40)
    w = wl.pulse_workload(30, 30, width=20)  # no interior left: the whole lattice
    assert interior(w) == (0, 0, 30, 30)
