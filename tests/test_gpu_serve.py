"""Continuous batching: jobs that arrive while others run are admitted as memory
frees up, share the batched launches, and each result is the same alone and
in the mix (bit-exact: the batched per-cell arithmetic does not depend on the
other jobs) and agrees with the single-lattice API within the parity
tolerances (FP32 1e-5, FP16 deviations 1e-2)."""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _jobs():
    from paper_1203_6350_gb300.serve import Job

    reqs = wl.request_trace(seed=3, rate=400.0, duration=1.0, lo=48, hi=160, steps_lo=30,
                            steps_hi=200, max_requests=12)
    return [Job(id=k, workload=r.workload, arrival=0.004 * k) for k, r in enumerate(reqs)]


@pytest.mark.parametrize("solo_cells", [None, 12000])
def test_results_same_alone_in_the_mix_and_serial(solo_cells):
    """solo_cells=None: every job shares the batched launch.  12000: the larger
    jobs run through the single-lattice kernel, interleaved with the batch."""
    from paper_1203_6350_gb300.serve import Server, serial_loop

    jobs = _jobs()
    assert {j.workload.storage for j in jobs} == {"f32", "f16dev"}
    if solo_cells is not None:
        assert 0 < sum(j.workload.cells >= solo_cells for j in jobs) < len(jobs)
    per_job = max(j.bytes for j in jobs)
    srv = Server(hbm_budget=3.5 * per_job, chunk=16, keep_fields=True, solo_cells=solo_cells)
    peak = []
    orig_admit = srv.admit

    def admit(now):
        n = orig_admit(now)
        peak.append(srv.used)
        return n

    srv.admit = admit
    mixed = {j.id: j for j in srv.run(jobs)}
    srv.close()
    assert len(mixed) == len(jobs)
    assert max(peak) <= srv.budget
    # queueing happened: some job was admitted after another one finished
    first_finish = min(j.finished for j in mixed.values())
    assert any(j.admitted > first_finish for j in mixed.values())

    for j in _jobs():
        alone = Server(hbm_budget=1e12, chunk=16, keep_fields=True, solo_cells=solo_cells)
        (res,) = alone.run([j], realtime=False)
        alone.close()
        np.testing.assert_array_equal(res.field, mixed[j.id].field)
        np.testing.assert_array_equal(res.result, mixed[j.id].result)

    serial = {j.id: j for j in serial_loop(_jobs(), keep_fields=True, realtime=False)}
    tol = {"f32": 1e-5, "f16dev": 1e-2}
    for jid, j in mixed.items():
        w = j.workload
        if w.variant == "I" and w.s[7] + w.chi_max > 2:
            continue  # unstable (Eq. effectrelax): ulp differences grow without bound
        a, b = j.field, serial[jid].field
        assert np.linalg.norm(a - b) <= tol[j.workload.storage] * np.linalg.norm(b) + 1e-300


def test_oversized_job_is_refused():
    from paper_1203_6350_gb300.serve import Job, Server

    w = wl.pulse_workload(512, 512, steps=10)
    srv = Server(hbm_budget=1e6)
    with pytest.raises(ValueError):
        srv.submit(Job(id=0, workload=w))
    srv.close()


def test_failed_jobs_are_reported_and_the_rest_carry_on(monkeypatch):
    """Failures stay with their job.  Three jobs of the trace fail at admission:
    a host-side fake of a failed allocation (LBM_ERR_OOM) on the
    single-lattice path and on the batched path, and a poisoned problem
    (rho0 < 0, refused by the library).  They are reported with their error
    and hold no memory; every other job's result equals its result alone."""
    from paper_1203_6350_gb300 import lbm
    from paper_1203_6350_gb300.batch import Batch
    from paper_1203_6350_gb300.serve import Job, Server, summary

    jobs = _jobs()
    solo_cells = 12000
    solo = [j.id for j in jobs if j.workload.cells >= solo_cells]
    batched = [j.id for j in jobs if j.workload.cells < solo_cells]
    fail_solo, fail_batch = solo[1], batched[1]
    poisoned = batched[2]
    jobs[poisoned] = Job(id=poisoned, workload=jobs[poisoned].workload.with_(rho0=-1.0),
                         arrival=jobs[poisoned].arrival)
    victims = {fail_solo: "solo", fail_batch: "batch"}

    orig_lat = lbm.Lattice.from_workload.__func__
    orig_add = Batch.add_workload

    def fake_lattice(cls, w, *a, **kw):
        if w is jobs[fail_solo].workload:
            raise lbm.LbmError(lbm.LBM_ERR_OOM, "device allocation failed (fake)")
        return orig_lat(cls, w, *a, **kw)

    def fake_add(self, w, *a, **kw):
        if w is jobs[fail_batch].workload:
            raise lbm.LbmError(lbm.LBM_ERR_OOM, "instance allocation failed (fake)")
        return orig_add(self, w, *a, **kw)

    monkeypatch.setattr(lbm.Lattice, "from_workload", classmethod(fake_lattice))
    monkeypatch.setattr(Batch, "add_workload", fake_add)
    per_job = max(j.bytes for j in jobs)
    srv = Server(hbm_budget=3.5 * per_job, chunk=16, keep_fields=True, solo_cells=solo_cells)
    done = {j.id: j for j in srv.run(jobs)}
    assert srv.used == 0 and srv.cells == 0 and not srv.resident
    srv.close()
    monkeypatch.undo()

    assert len(done) == len(jobs)
    for jid in victims:
        assert done[jid].result is None and "fake" in done[jid].error
    assert done[poisoned].result is None and "far-field" in done[poisoned].error
    s = summary(list(done.values()), 1.0)
    assert s["failed"] == 3 and s["jobs"] == len(jobs) - 3

    for j in _jobs():
        if j.id in victims or j.id == poisoned:
            continue
        alone = Server(hbm_budget=1e12, chunk=16, keep_fields=True, solo_cells=solo_cells)
        (res,) = alone.run([j], realtime=False)
        alone.close()
        assert done[j.id].error is None or "non-finite" in done[j.id].error
        np.testing.assert_array_equal(res.field, done[j.id].field)
        np.testing.assert_array_equal(res.result, done[j.id].result)


def test_non_finite_job_is_reported():
    """A type I layer with s + chi > 2 (Eq. effectrelax) blows up; the server
    reports that job as non-finite at read-out and the stable job beside it
    as solved."""
    from paper_1203_6350_gb300.serve import Job, Server

    bad = wl.pulse_workload(64, 64, variant="I", storage="f32", chi_max=1.0, width=12,
                            steps=600, name="unstable")
    good = wl.pulse_workload(64, 64, variant="II", storage="f32", chi_max=0.3, width=12,
                             steps=600, name="stable")
    srv = Server(hbm_budget=1e9, chunk=64)
    done = {j.id: j for j in srv.run([Job(id=0, workload=bad), Job(id=1, workload=good)],
                                     realtime=False)}
    srv.close()
    assert done[0].result[5] > 0 and "non-finite" in done[0].error
    assert done[1].result[5] == 0 and done[1].error is None


@pytest.mark.parametrize("solo_cells", [None, 12000])
def test_served_results_match_the_oracle(solo_cells):
    """Each served job's final rho' against the FP64 oracle run of the same
    problem, relative to the oracle's final field: FP32 1e-5, FP16 deviations
    1e-2.  solo_cells=None sends every job through the batched launch; 12000
    runs the larger ones through the single-lattice kernel beside it.  The
    trace mixes FP32 and FP16 storage and types I, II and III.  A type I job
    with s + chi > 2 (Eq. effectrelax) amplifies every rounding difference
    without bound (reading C15): where the oracle's field is non-finite the
    served one must be too; where it has grown tenfold past the initial pulse
    the served one must have grown as well (or overflowed a 16-bit format to
    non-finite values); before that the error is taken in units of the initial
    pulse."""
    from helpers import run_oracle
    from paper_1203_6350_gb300.serve import Server

    jobs = _jobs()
    assert {j.workload.variant for j in jobs} == {"I", "II", "III"}
    srv = Server(hbm_budget=1e12, chunk=16, keep_fields=True, solo_cells=solo_cells)
    done = {j.id: j for j in srv.run(jobs, realtime=False)}
    srv.close()
    tol = {"f32": 1e-5, "f16dev": 1e-2}
    checked = set()
    for j in jobs:
        w = j.workload
        got = done[j.id].field
        ref = run_oracle(w)[0]
        den = np.linalg.norm(ref)
        if w.variant == "I" and w.s[7] + w.chi_max > 2:
            init = w.density_deviation()
            if not np.isfinite(ref).all():
                assert not np.isfinite(got).all(), j.id
                continue
            if np.abs(ref).max() > 10 * np.abs(init).max():
                # grown too, or past the 16-bit format's range (non-finite)
                assert (not np.isfinite(got).all()
                        or np.abs(got).max() > 10 * np.abs(init).max()), j.id
                continue
            den = np.linalg.norm(init)
        err = np.linalg.norm(got - ref) / den
        assert err <= tol[w.storage], (j.id, w.storage, w.variant, w.steps, err)
        checked.add((w.storage, w.variant))
    assert {s for s, _ in checked} == {"f32", "f16dev"} and len(checked) >= 4, checked


@pytest.mark.parametrize("storage", ["f64", "f32", "f16dev"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic", "channel"])
def test_lattice_bytes_are_what_the_allocator_hands_out(storage, bc, monkeypatch):
    """lbm_lattice_bytes(host_io = 1) is the peak a lattice holds through its
    allocator after a host-field initialisation and a host read-out, with TMA
    staging set up where it exists (FP32, Dirichlet): counted on a wrapped
    torch allocator."""
    from paper_1203_6350_gb300 import lbm

    live, peak = [0], [0]

    class Counting(lbm.TorchAllocator):
        def _alloc(self, nbytes, ctx):
            live[0] += int(nbytes)
            peak[0] = max(peak[0], live[0])
            return super()._alloc(nbytes, ctx)

        def _free(self, ptr, nbytes, ctx):
            live[0] -= int(nbytes)
            return super()._free(ptr, nbytes, ctx)

    monkeypatch.setattr(lbm, "TorchAllocator", Counting)
    w = wl.pulse_workload(333, 77, variant="II", storage=storage, steps=4, bc=bc, width=6)
    with lbm.Lattice.from_workload(w) as lat:
        if storage == "f32" and bc == "dirichlet":
            lat.cells_per_thread = 2
            lat.steps_per_launch = 2
            lat.tma_staging = True
        lat.step(w.steps)
        lat.moments()
    assert live[0] == 0
    want = lbm.lbm_lattice_bytes(w.nx, w.ny, lbm.STORAGE[storage], lbm.BC[bc], 1)
    assert peak[0] == want, (peak[0], want)
    assert lbm.lbm_lattice_bytes(w.nx, w.ny, lbm.STORAGE[storage], lbm.BC[bc], 0) == \
        want - 24 * w.nx * w.ny
