"""Host-side logic of the serving loop (CPU only): admission under a small
artificial HBM budget, oldest-first batching per context, batch size limit."""
from paper_2605_17222_gb300.serving import LtServer, Request, percentile, scratch_bytes


class FakeCtx:
    def __init__(self, N=1 << 12, k=1, alpha=1):
        self.N, self.k, self.alpha = N, k, alpha

    def beta(self, level):
        return -(-level // self.alpha)

    def choose_split(self, algo, level, n_diag):
        return (4, 4, n_diag // 16)


class FakeCt:
    def __init__(self, level):
        self.level = level


class FakeMatrix:
    n_diag = 64


def _req(i, key, level, t=0.0):
    return Request(i, key, FakeMatrix(), FakeCt(level), t)


def test_admission_respects_budget_and_order():
    ctxs = {"a": FakeCtx(), "b": FakeCtx(N=1 << 13)}
    one = scratch_bytes(ctxs["a"], 4, (4, 4, 4)) + 16 * 4 * (1 << 12)
    srv = LtServer(ctxs, hbm_budget=3.5 * one, resident_bytes=0, streams=2, max_batch=16)
    for i in range(6):
        srv.submit(_req(i, "a", 4))
    srv.submit(_req(6, "b", 4))
    batch = srv._take_batch()
    assert [r.rid for r in batch] == [0, 1, 2]          # three fit the budget
    srv.inflight_bytes += sum(r.scratch_bytes for r in batch)
    assert srv._take_batch() == []                      # nothing else fits while they run
    assert srv.stats.admission_waits == 1
    srv.inflight_bytes = 0
    assert [r.rid for r in srv._take_batch()] == [3, 4, 5]  # oldest first, same context only
    assert [r.rid for r in srv._take_batch()] == [6]


def test_batch_size_limit_and_resident_bytes():
    ctxs = {"a": FakeCtx()}
    srv = LtServer(ctxs, hbm_budget=1e12, resident_bytes=0, streams=1, max_batch=4)
    for i in range(10):
        srv.submit(_req(i, "a", 3))
    assert len(srv._take_batch()) == 4
    srv2 = LtServer(ctxs, hbm_budget=1e9, resident_bytes=1e9, streams=1)
    srv2.submit(_req(0, "a", 3))
    assert srv2._take_batch() == []                     # the resident set already fills the budget


def test_percentile():
    xs = list(range(1, 101))
    assert percentile(xs, 50) in (50, 51)
    assert percentile(xs, 99) == 99


def test_retire_while_another_thread_counts_pending():
    """Batches retire (their completion events fire) while a submitting thread
    keeps reading pending(): the in-flight table is only changed under the
    server's lock, so the reader never sees it mid-update, and every request,
    byte and batch is accounted for once."""
    import threading

    class Ev:
        def __init__(self, polls):
            self.polls = polls

        def query(self):
            self.polls -= 1
            return self.polls <= 0

    srv = LtServer({"a": FakeCtx()}, hbm_budget=1e12, resident_bytes=0, streams=64)
    for si in range(64):
        srv.inflight[si] = (Ev(1 + si % 5), [_req(si, "a", 3, t=0.0)], 100)
        srv.inflight_bytes += 100
    errors, seen = [], []
    stop = threading.Event()

    def reader():
        while not stop.is_set():
            try:
                seen.append(srv.pending())
            except Exception as e:  # a dict mutated during iteration would land here
                errors.append(e)
                return

    t = threading.Thread(target=reader)
    t.start()
    for _ in range(10):
        srv._retire()
    stop.set()
    t.join()
    assert not errors
    assert srv.inflight == {} and srv.inflight_bytes == 0
    assert srv.stats.completed == 64 and sorted(r.rid for r in srv.completed) == list(range(64))
    assert all(0 <= n <= 64 for n in seen)
