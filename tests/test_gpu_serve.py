"""Continuous-batching server: requests submitted concurrently must each get the
result they would get alone on the tree holding exactly the updates admitted
before them.  The expected answers come from the oracle replaying the requests
in admission order."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2601_05347_gb300 import gen  # noqa: E402

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2601_05347_gb300 import psi, serve


def T(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to("cuda")


def make_requests(base, rng_seed, count):
    rng = np.random.default_rng(rng_seed)
    reqs, next_id, deletable = [], 10_000_000, list(range(len(base)))
    rng.shuffle(deletable)
    for t in range(count):
        r = rng.random()
        if r < 0.15:
            m = int(rng.integers(50, 3000))
            p = gen.varden(m, 2, 30, 100 + t, x_range=(1 << 29, 1 << 30) if t % 2 else None)
            ids = np.arange(next_id, next_id + m, dtype=np.uint32)
            next_id += m
            reqs.append(serve.Request("insert", p, ids))
        elif r < 0.3:
            m = int(rng.integers(50, 2000))
            take, deletable = deletable[:m], deletable[m:]
            reqs.append(serve.Request("delete", base[take], np.array(take, np.uint32)))
        elif r < 0.6:
            nq = int(rng.integers(1, 3000))
            k = int(rng.choice([1, 10, 100]))
            q = base[rng.integers(0, len(base), nq)]
            reqs.append(serve.Request("knn", q, k=k))
        elif r < 0.8:
            nq = int(rng.integers(1, 2000))
            c = base[rng.integers(0, len(base), nq)]
            reqs.append(serve.Request("count", gen.centred_boxes(c, 1 << 21, 30)))
        else:
            nq = int(rng.integers(1, 300))
            c = base[rng.integers(0, len(base), nq)]
            reqs.append(serve.Request("report", gen.centred_boxes(c, 1 << 20, 30)))
    return reqs


def test_server_results_equal_serial_replay():
    base = gen.varden(40000, 2, 30, 77)
    ids = np.arange(len(base), dtype=np.uint32)
    ix = psi.Index(T(base), T(ids), kind="spac_h", leaf_size=32)
    srv = serve.Server(ix)
    reqs = make_requests(base, 3, 120)
    # submit from two threads at once, interleaved
    halves = [reqs[0::2], reqs[1::2]]
    ths = [threading.Thread(target=lambda rs=h: [srv.submit(r) for r in rs]) for h in halves]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    results = {r.seq: (r, r.future.result(timeout=300)) for r in reqs}
    srv.close()
    assert any(n > 1 for n, _ in srv.rounds), "no round admitted more than one request"
    o = O.Index(base, ids, kind=O.SPAC_H, phi=32)
    for seq in sorted(results):
        r, got = results[seq]
        if r.kind == "insert":
            o.insert(r.a, r.b)
        elif r.kind == "delete":
            assert got == o.delete(r.a, r.b)
        elif r.kind == "knn":
            oi, od = o.knn(r.a, r.k)
            assert (got[0] == oi).all() and (got[1] == od).all(), seq
        elif r.kind == "count":
            assert (got == o.range_count(r.a)).all(), seq
        else:
            ooff, oid = o.range_report(r.a)
            assert (got[0] == ooff).all(), seq
            for j in range(len(r.a)):
                assert sorted(got[1][got[0][j]:got[0][j + 1]].tolist()) == oid[ooff[j]:ooff[j + 1]].tolist()
    ix.close()


def test_server_refuses_request_over_budget():
    base = gen.uniform(5000, 2, 30, 5)
    ix = psi.Index(T(base), T(np.arange(5000, dtype=np.uint32)), kind="spac_z")
    srv = serve.Server(ix, mem_budget=1 << 16)
    big = serve.Request("knn", base[np.arange(5000)], k=10)
    small = serve.Request("count", gen.centred_boxes(base[:4], 1000, 30))
    f_big = srv.submit(big)
    f_small = srv.submit(small)
    with pytest.raises(MemoryError):
        f_big.result(timeout=60)
    assert len(f_small.result(timeout=60)) == 4
    srv.close()
    ix.close()


def test_plain_form_matches_server():
    base = gen.varden(20000, 2, 30, 9)
    ids = np.arange(len(base), dtype=np.uint32)
    a = psi.Index(T(base), T(ids), kind="spac_h")
    b = psi.Index(T(base), T(ids), kind="spac_h")
    reqs = make_requests(base, 11, 40)
    srv = serve.Server(a)
    futs = [srv.submit(r) for r in reqs]
    got = [f.result(timeout=300) for f in futs]
    srv.close()
    for r, g in zip(reqs, got):
        p = serve.serve_plain(b, serve.Request(r.kind, r.a, r.b, r.k))
        if r.kind == "knn":
            assert (g[0] == p[0]).all() and (g[1] == p[1]).all()
        elif r.kind == "count":
            assert (g == p).all()
        elif r.kind == "delete":
            assert g == p
        elif r.kind == "report":
            assert (g[0] == p[0]).all() and sorted(g[1].tolist()) == sorted(p[1].tolist())
    a.close()
    b.close()
