"""Host-side logic of the serving layer (no GPU): admission by free device memory counts the
workspace promised to admitted workers that have not allocated it yet, and an out-of-memory batch
is re-queued (at most twice per work item) while the extra worker that hit it retires."""
import collections
import threading
import types

import numpy as np

from paper_1801_08655_gb300 import hz, serving

GB = 1e9


class FakeSolver:
    def __init__(self):
        self.closed = False

    def close(self):
        self.closed = True


def make_server(free_bytes, need_bytes, monkeypatch):
    srv = object.__new__(serving.Server)
    srv.torch = types.SimpleNamespace(cuda=types.SimpleNamespace(mem_get_info=lambda: (free_bytes, 200 * GB)))
    srv.max_cols, srv.max_workers, srv.mem_reserve = 32, 3, 4 * GB
    srv.primaries = [FakeSolver()]
    srv.workers = [[]]
    srv.queues = [collections.deque()]
    srv.cv = threading.Condition()
    srv.threads, srv.errors, srv.admission_log = [], [], []
    srv.pending, srv.retries = {}, {}
    srv.running = True
    srv.log = None
    srv._work = lambda w, s: None
    monkeypatch.setattr(serving.Server, "worker_bytes", lambda self, cols: need_bytes)
    monkeypatch.setattr(serving.hz.Solver, "shared", classmethod(lambda cls, prim: FakeSolver()))
    return srv


def test_admission_counts_promised_workspace(monkeypatch):
    # room for one workspace beyond the reserve: the primary's (not yet allocated) takes it
    srv = make_server(free_bytes=4 * GB + 15 * GB, need_bytes=10 * GB, monkeypatch=monkeypatch)
    assert srv._admit_worker(0)             # primary: always admitted, its workspace promised
    assert srv.pending and sum(srv.pending.values()) == 10 * GB
    assert not srv._admit_worker(0)         # 15 GB free - 10 GB promised < 10 GB
    assert "promised" in srv.admission_log[-1]
    srv.pending.clear()                     # the primary has allocated (free memory unchanged here)
    assert srv._admit_worker(0)
    assert len(srv.workers[0]) == 2


def test_out_of_memory_batch_is_requeued_and_extra_worker_retires(monkeypatch):
    srv = make_server(free_bytes=100 * GB, need_bytes=1 * GB, monkeypatch=monkeypatch)
    srv._admit_worker(0)
    srv._admit_worker(0)
    extra = srv.workers[0][1]
    req = serving.Request(7, 0, np.zeros((40, 3), dtype=np.int64))
    req._left = 40
    items = [(req, 0, 32), (req, 32, 40)]
    oom = hz.HzError(hz.HZ_ERR_OOM, "device allocation failed")
    adm = hz.HzError(hz.HZ_ERR_ADMISSION, "workspace does not fit")
    srv._admit_worker(0)
    extra2 = srv.workers[0][-1]
    assert srv._failed_batch(0, extra2, items, adm) is True      # a workspace that does not fit: as OOM
    srv.queues[0].clear()
    srv.retries.clear()
    assert srv._failed_batch(0, extra, items, oom) is True       # extra worker retires
    assert list(srv.queues[0]) == items                          # same order, at the head
    assert extra not in srv.workers[0] and not srv.errors and req.status == 0
    prim = srv.primaries[0]
    srv.queues[0].clear()
    assert srv._failed_batch(0, prim, items, oom) is False      # second failure: retried again
    srv.queues[0].clear()
    assert srv._failed_batch(0, prim, items, oom) is False      # third: the requests fail
    assert not srv.queues[0] and srv.errors and req.status == -1 and req._left == 0
    # any other error fails the batch at once
    req2 = serving.Request(8, 0, np.zeros((3, 3), dtype=np.int64))
    req2._left = 3
    assert srv._failed_batch(0, prim, [(req2, 0, 3)], RuntimeError("boom")) is False
    assert req2.status == -1 and req2.t_done is not None


def test_failed_item_keeps_request_failed_when_a_later_item_succeeds(monkeypatch):
    srv = make_server(free_bytes=100 * GB, need_bytes=1 * GB, monkeypatch=monkeypatch)
    srv.batches, srv.max_requests_per_batch = 0, 0
    srv.torch = types.SimpleNamespace(empty=lambda shp, dtype=None, device=None: np.zeros(shp, dtype=dtype),
                                      cuda=srv.torch.cuda)
    srv._admit_worker(0)
    prim = srv.primaries[0]
    req = serving.Request(9, 0, np.zeros((40, 3), dtype=np.int64))
    req._left = 40
    noconv = hz.HzError(hz.HZ_ERR_NO_CONVERGENCE, "GMRES hit its iteration cap")
    assert srv._failed_batch(0, prim, [(req, 0, 32)], noconv) is False
    assert req.status == -1 and req.t_done is None and req._left == 8
    srv._deliver([(req, 32, 40)], [np.ones((8, 5), dtype=np.complex128)], now=1.0)
    assert req.status == -1 and req.result is None and req.t_done == 1.0 and req._left == 0
    # a request whose items all succeed is delivered whole
    ok = serving.Request(10, 0, np.zeros((3, 3), dtype=np.int64))
    ok._left = 3
    srv._deliver([(ok, 0, 2), (ok, 2, 3)], [np.full((2, 5), 1.0 + 0j), np.full((1, 5), 2.0 + 0j)], now=2.0)
    assert ok.status == 0 and ok.t_done == 2.0 and ok.result.shape == (3, 5) and ok.result[2, 0] == 2.0


def test_a_second_serve_restarts_the_admitted_workers(monkeypatch):
    """serve() called again (after a calibration run) runs every worker already admitted instead of
    admitting more: no frequency is left without a running worker."""
    srv = make_server(free_bytes=100 * GB, need_bytes=1 * GB, monkeypatch=monkeypatch)
    started = []
    srv._start = lambda w, solver: started.append((w, solver))
    srv.running = False
    srv.serve([], realtime=False, timeout=0.0)
    assert len(srv.workers[0]) == 1 and started == [(0, srv.primaries[0])]
    srv.serve([], realtime=False, timeout=0.0)
    srv.serve([], realtime=False, timeout=0.0)
    assert len(srv.workers[0]) == 1 and started == [(0, srv.primaries[0])] * 3


def test_requests_are_cut_into_column_items_and_batched_in_arrival_order(monkeypatch):
    """A request of R sources becomes work items of at most max_cols columns; a free worker takes
    items from the head of its frequency's queue, in arrival order, while they fit in one batch of
    max_cols columns (items of different requests share a batch)."""
    srv = make_server(free_bytes=100 * GB, need_bytes=1 * GB, monkeypatch=monkeypatch)
    srv.running = False                    # no admissions: only the queue logic
    a = serving.Request(1, 0, np.zeros((70, 3), dtype=np.int64))
    b = serving.Request(2, 0, np.zeros((5, 3), dtype=np.int64))
    c = serving.Request(3, 0, np.zeros((30, 3), dtype=np.int64))
    for r in (a, b, c):
        srv.submit(r)
    assert [(it[0].rid, it[1], it[2]) for it in srv.queues[0]] == [(1, 0, 32), (1, 32, 64), (1, 64, 70),
                                                                  (2, 0, 5), (3, 0, 30)]
    assert a._left == 70 and b._left == 5
    items, cols = srv._take(0)
    assert [(it[0].rid, it[1]) for it in items] == [(1, 0)] and cols == 32
    items, cols = srv._take(0)
    assert [(it[0].rid, it[1]) for it in items] == [(1, 32)] and cols == 32
    items, cols = srv._take(0)              # 6 + 5 columns fit, the 30 of the next request do not
    assert [(it[0].rid, it[1]) for it in items] == [(1, 64), (2, 0)] and cols == 11
    items, cols = srv._take(0)
    assert [(it[0].rid, it[1]) for it in items] == [(3, 0)] and cols == 30
    assert srv._take(0) == ([], 0)
