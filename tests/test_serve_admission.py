"""The server's admission by device-memory budget (host logic, no GPU): a round
takes pending requests in arrival order while they fit next to the memory that
earlier rounds still hold (query results not yet copied back), and a request
that does not fit waits until the finisher releases that memory."""
import collections
import threading
import time
import types

from paper_2601_05347_gb300.serve import Server


def bare_server(budget):
    """The admission state of a Server, without its CUDA streams and threads."""
    s = Server.__new__(Server)
    s.budget = budget
    s.pending = collections.deque()
    s.lock = threading.Condition()
    s.inflight = 0
    s.stop_flag = False
    return s


def req(i, nbytes):
    return types.SimpleNamespace(i=i, est_bytes=nbytes, held=False, t_admit=0.0)


def test_round_takes_requests_in_order_while_they_fit():
    s = bare_server(100)
    rs = [req(0, 40), req(1, 40), req(2, 40), req(3, 10)]
    s.pending.extend(rs)
    got = s._admit()
    # arrival order: request 2 does not fit, so request 3 waits behind it
    assert [r.i for r in got] == [0, 1]
    assert s.inflight == 80 and all(r.held for r in got)
    assert [r.i for r in s.pending] == [2, 3]


def test_waits_for_memory_held_by_earlier_rounds():
    s = bare_server(100)
    first = [req(0, 60), req(1, 30)]
    s.pending.extend(first)
    assert [r.i for r in s._admit()] == [0, 1]
    s.pending.append(req(2, 50))  # 90 held + 50 > 100: must wait
    released = []

    def finisher():
        time.sleep(0.2)
        released.append(time.perf_counter())
        s._release([first[0]])  # request 0's results are on the host

    t = threading.Thread(target=finisher, daemon=True)
    t.start()
    out = {}

    def admit():
        out["got"] = s._admit()
        out["after_release"] = bool(released)  # read as soon as the round is admitted

    a = threading.Thread(target=admit, daemon=True)  # a deadlock fails the test instead of hanging it
    a.start()
    a.join(timeout=10)
    t.join(timeout=10)
    assert not a.is_alive() and out["after_release"]
    got = out["got"]
    assert [r.i for r in got] == [2]
    assert s.inflight == 30 + 50
    # releasing twice frees nothing more
    s._release([first[0]])
    assert s.inflight == 80
    s._release([first[1], got[0]])
    assert s.inflight == 0


def test_empty_queue_returns_on_stop():
    s = bare_server(100)
    s.stop_flag = True
    assert s._admit() == []
