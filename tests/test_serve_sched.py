"""Host logic of the serving scheduler (no GPU): which pending requests one step launches.
A batch takes the requests of the head's kind in arrival order, passing over single-DFA-launch
requests and requests of the other kind (they keep their places), until it is full."""
from collections import deque

from paper_2410_22764_gb300 import serve


class _Req:
    def __init__(self, rid, n, k, closure=False):
        self.rid, self.n, self.k, self.closure = rid, n, k, closure
        self.nbytes = n * k
        self.admitted, self.attempts = None, 0


def _server(pending, max_batch=4, solo_work=100, budget=1 << 40, max_work=1 << 62):
    srv = serve.Server.__new__(serve.Server)          # no CUDA streams: scheduling only
    srv.free, srv.inflight, srv.used = [0, 1, 2, 3], [], 0
    srv.budget, srv.max_batch, srv.max_batch_work, srv.solo_work = budget, max_batch, max_work, solo_work
    srv.pending = deque(pending)
    srv.launched = []
    srv._launch = lambda reqs, cl: srv.launched.append(("batch", [r.rid for r in reqs], cl))
    srv._launch_solo = lambda r: srv.launched.append(("solo", r.rid))
    return srv


def test_batch_passes_over_single_launch_and_other_kind():
    srv = _server([_Req(0, 10, 2), _Req(1, 200, 2), _Req(2, 5, 2), _Req(3, 7, 2, True),
                   _Req(4, 3, 2), _Req(5, 9, 2), _Req(6, 4, 2)])
    srv.step()
    assert srv.launched == [("batch", [0, 2, 4, 5], False)]
    assert [r.rid for r in srv.pending] == [1, 3, 6]          # order kept
    srv.step()
    assert srv.launched[-1] == ("solo", 1)
    srv.step()
    assert srv.launched[-1] == ("batch", [3], True)
    srv.step()
    assert srv.launched[-1] == ("batch", [6], False) and not srv.pending


def test_batch_stops_at_work_and_budget_bounds():
    srv = _server([_Req(i, 10, 3) for i in range(6)], max_batch=10, max_work=70)
    srv.step()
    assert srv.launched == [("batch", [0, 1], False)]          # 30 + 30 <= 70 < 90
    srv = _server([_Req(i, 10, 3) for i in range(6)], max_batch=10, budget=95)
    srv.step()
    assert srv.launched == [("batch", [0, 1, 2], False)]       # 3 x 30 bytes fit in 95
    srv = _server([_Req(0, 10, 3)], solo_work=0)               # 0: never a single launch
    srv.step()
    assert srv.launched == [("batch", [0], False)]
