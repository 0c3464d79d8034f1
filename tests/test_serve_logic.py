"""Host-side scheduling of the serving loop, on the CPU: the library and the CUDA streams
are replaced by fakes whose solve_iterate advances a fake clock by a fixed cost per
iteration, so admission order, the memory budget, joins at tick boundaries, idle-gap
jumps and the latency bookkeeping are checked exactly."""
import contextlib
import types

import pytest

from paper_1809_04195_gb300 import serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeLib:
    """Stands in for the t2sh binding: a plan iterates by advancing the clock."""
    KSPACE_TE, KSPACE_PROJ = 0, 1

    def __init__(self, clock, cost_per_iter, admit_cost=0.0, end_cost=0.0):
        self.clock, self.cost = clock, cost_per_iter
        self.admit_cost, self.end_cost = admit_cost, end_cost
        self.closed = []
        lib = self

        class Plan:
            def __init__(self, dims, phi, mask, maps, stream=None):
                self.dims, self.done = dims, 0
                lib.clock.t += lib.admit_cost / 2

            def solve_begin(self, kspace, kform):
                self.done = 0
                lib.clock.t += lib.admit_cost / 2

            def solve_iterate(self, n):
                k = min(n, self.dims.iters - self.done)
                lib.clock.t += k * lib.cost
                self.done += k
                return self.done

            def solve_end(self):
                lib.clock.t += lib.end_cost
                return ("result", self.dims.tag)

            def close(self):
                lib.closed.append(self.dims.tag)

        self.Plan = Plan

    @staticmethod
    def workspace_bytes(dims):
        return dims.ws


class FakeTorch:
    class _Stream:
        def synchronize(self):
            pass

    cuda = types.SimpleNamespace(Stream=_Stream, stream=lambda s: contextlib.nullcontext())


def dims(tag, iters, ws, ny=16, nz=16, S=1, C=1, K=1):
    return types.SimpleNamespace(tag=tag, iters=iters, ws=ws, ny=ny, nz=nz, nslices=S, ncoils=C,
                                 nechoes=K, nbasis=K, nmaps=1)


class CheckedServer(serve.Server):
    """Asserts the budget before every tick and records who was resident."""

    def __init__(self, *a, **kw):
        super().__init__(*a, **kw)
        self.torch = FakeTorch
        self.resident = []

    def _tick(self):
        assert self.used <= self.budget
        assert self.used == sum(r.footprint for r in self.active)
        self.resident.append(sorted(r.scan_id for r in self.active))
        super()._tick()


def make_server(monkeypatch, budget, cost=0.01, iters_per_tick=10, admit_cost=0.0, end_cost=0.0):
    clock = FakeClock()
    monkeypatch.setattr(serve.time, "perf_counter", clock)
    lib = FakeLib(clock, cost, admit_cost, end_cost)
    return CheckedServer(lib, budget, iters_per_tick), lib, clock


def req(lib, i, t, iters, ws):
    return serve.ScanRequest(i, 0, t, 0, dims(i, iters, ws), None, None, None, None, lib.KSPACE_PROJ)


def footprint(d):
    return serve.footprint_bytes(FakeLib, d, FakeLib.KSPACE_PROJ)


def test_fcfs_no_overtaking_and_budget(monkeypatch):
    """A large scan at the head of the queue blocks a smaller later one that would fit:
    admission follows arrival order and the resident footprint never exceeds the budget."""
    per = footprint(dims(0, 10, 1000))
    srv, lib, _ = make_server(monkeypatch, budget=3 * per + 100)  # room for scan 3 beside 0 and 1, not for 2
    srv.submit(req(lib, 0, 0.0, 30, 1000))
    srv.submit(req(lib, 1, 0.0, 30, 1000))
    srv.submit(req(lib, 2, 0.01, 30, 4000))  # does not fit beside two others
    srv.submit(req(lib, 3, 0.02, 10, 1000))  # would fit, but must wait behind scan 2
    rep = srv.run()
    order = sorted(srv.done, key=lambda r: (r.admitted_s, r.scan_id))
    assert [r.scan_id for r in order] == [0, 1, 2, 3]
    assert all(r.result == ("result", r.scan_id) for r in srv.done)
    r2, r3 = (next(r for r in srv.done if r.scan_id == k) for k in (2, 3))
    assert r3.admitted_s >= r2.admitted_s
    assert rep["scans"] == 4 and srv.used == 0


def test_join_at_tick_boundary_and_latency(monkeypatch):
    """A scan arriving during a tick joins at the next tick boundary; latency is completion
    minus arrival on the virtual clock."""
    srv, lib, _ = make_server(monkeypatch, budget=10**9, cost=0.01, iters_per_tick=10)
    srv.submit(req(lib, 0, 0.0, 40, 1000))   # four ticks of 0.1 s alone
    srv.submit(req(lib, 1, 0.15, 20, 1000))  # arrives inside the second tick
    srv.run()
    a, b = sorted(srv.done, key=lambda r: r.scan_id)
    assert a.admitted_s == 0.0
    assert b.admitted_s == pytest.approx(0.2)            # end of tick 2
    assert srv.resident[:3] == [[0], [0], [0, 1]]
    # tick 3 and 4 cost 0.2 s each with both resident; scan 1 needs two of them
    assert b.done_s == pytest.approx(0.6)
    assert b.done_s - b.arrival_s == pytest.approx(0.45)
    assert a.done_s == pytest.approx(0.6)


def test_idle_gap_is_skipped(monkeypatch):
    """With nothing resident the clock jumps to the next arrival: busy time counts only ticks."""
    srv, lib, _ = make_server(monkeypatch, budget=10**9, cost=0.01, iters_per_tick=10)
    srv.submit(req(lib, 0, 0.0, 10, 1000))
    srv.submit(req(lib, 1, 300.0, 10, 1000))
    rep = srv.run()
    b = next(r for r in srv.done if r.scan_id == 1)
    assert b.admitted_s == 300.0 and b.done_s == pytest.approx(300.1)
    assert rep["busy_s"] == pytest.approx(0.2)
    assert rep["latency_p50_s"] == pytest.approx(0.1)
    assert rep["ticks"] == 2


def test_oversize_scan_is_refused(monkeypatch):
    srv, lib, _ = make_server(monkeypatch, budget=5000)
    with pytest.raises(ValueError):
        srv.submit(req(lib, 0, 0.0, 10, 10**6))


def test_cancel_queued_and_resident_scans(monkeypatch):
    """A queued scan withdrawn before admission never runs; a resident one is closed at the
    next tick boundary and its memory admits the waiting scan; cancelling a finished or
    unknown scan changes nothing."""
    per = footprint(dims(0, 10, 1000))
    srv, lib, _ = make_server(monkeypatch, budget=2 * per + 100, cost=0.01, iters_per_tick=10)
    srv.submit(req(lib, 0, 0.0, 40, 1000))
    srv.submit(req(lib, 1, 0.0, 40, 1000))
    srv.submit(req(lib, 2, 0.05, 10, 1000))   # waits: the budget holds two scans
    srv.submit(req(lib, 3, 0.06, 10, 1000))   # waits behind scan 2
    srv.cancel(3, at_s=0.1)                   # still queued then
    srv.cancel(1, at_s=0.15)                  # resident: leaves at the tick boundary 0.2
    srv.cancel(0, at_s=10.0)                  # finished long before
    srv.cancel(99, at_s=0.0)                  # unknown
    rep = srv.run()
    done = {r.scan_id: r for r in srv.done}
    gone = {r.scan_id: r for r in srv.cancelled}
    assert sorted(done) == [0, 2] and sorted(gone) == [1, 3]
    assert gone[3].admitted_s == -1.0 and gone[3].cancelled_s == pytest.approx(0.2)
    assert gone[1].cancelled_s == pytest.approx(0.2) and gone[1].result is None
    assert 1 in lib.closed and 3 not in lib.closed
    assert done[2].admitted_s == pytest.approx(0.2)        # admitted into the freed memory
    assert srv.resident[:3] == [[0, 1], [0, 2], [0]]
    assert rep["scans"] == 2 and rep["cancelled"] == 2 and srv.used == 0


def test_admission_and_completion_are_charged(monkeypatch):
    """The plan, A^H y and the result copy take GPU time too: the clock advances by them,
    so they count in latency and busy time (0.05 s to admit, 0.02 s to finish a scan)."""
    srv, lib, _ = make_server(monkeypatch, budget=10**9, cost=0.01, iters_per_tick=10, admit_cost=0.05,
                              end_cost=0.02)
    srv.submit(req(lib, 0, 0.0, 20, 1000))   # admitted at 0, ticks 0.05-0.15, 0.15-0.25, done 0.27
    srv.submit(req(lib, 1, 0.1, 10, 1000))   # arrives in the first tick; admitted at 0.15, 0.2 s to admit
    rep = srv.run()
    a, b = sorted(srv.done, key=lambda r: r.scan_id)
    assert a.admitted_s == 0.0 and b.admitted_s == pytest.approx(0.15)
    # after b's admission (0.15 -> 0.20) the second tick runs both: 0.20 -> 0.40
    assert a.done_s == pytest.approx(0.42)
    assert b.done_s == pytest.approx(0.44)
    assert b.done_s - b.arrival_s == pytest.approx(0.34)
    assert rep["admission_s"] == pytest.approx(0.10)
    assert rep["busy_s"] == pytest.approx(0.44)
