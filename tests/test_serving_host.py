"""Host-side failure handling of the serving layer (no GPU): a worker that
stops on a library error fails every request it holds and every later one,
and the stream's watchdog fails requests that make no progress, so a caller
of serve() never waits forever."""
import threading
import time

import pytest

pytest.importorskip("torch")
serving = pytest.importorskip("paper_2608_03515_b300.serving")


class _FakeServer:
    """The parts of Server that serve() and Group use, with no GPU behind it."""

    def __init__(self):
        self.t0 = time.perf_counter()
        self.groups = {}
        self.closing = False
        self.stalled = False

    def start(self):
        self.t0 = time.perf_counter()

    def submit(self, req):
        pass                                           # nothing ever runs: the watchdog must end the wait

    def close(self):
        self.closing = True


def _requests(n):
    return [serving.Request(i, 64, 0, 0.1, 2, 0.0, rhs_seed=i) for i in range(n)]


def test_watchdog_fails_requests_without_progress():
    srv = _FakeServer()
    reqs = _requests(3)
    t = time.perf_counter()
    out = serving.serve(srv, reqs, max_idle_s=0.3)
    assert time.perf_counter() - t < 10.0
    assert out["failed"] == 3 and out["not_converged"] == 0
    assert all(r.status == serving.FAILED and r.finish is not None for r in reqs)
    assert srv.stalled


def test_worker_error_fails_held_and_later_requests():
    srv = _FakeServer()
    g = object.__new__(serving.Group)                  # a worker without a hierarchy behind it
    g.server = srv
    g.cv = threading.Condition()
    g.error = None
    held, queued, later = _requests(3)
    g.queue = [(queued, 0), (queued, 1)]
    g.where = {0: (held, 0)}

    def boom():
        raise RuntimeError("amamg_batch_cycle: CUDA error (-3)")

    g._run = boom
    g.run()                                            # returns instead of raising
    assert "CUDA error" in g.error
    for r in (held, queued):
        assert r.status == serving.FAILED and r.finish is not None
    assert not g.queue and not g.where
    g.submit(later)
    assert later.status == serving.FAILED and later.finish is not None
