"""The server's round planning (host logic, no GPU): every admitted request runs
exactly once, updates keep their arrival order, and each query sees exactly the
updates that arrived before it -- the same state as one-at-a-time execution."""
import random
import types

from paper_2601_05347_gb300.serve import plan_epochs


def req(kind, i):
    return types.SimpleNamespace(kind=kind, i=i)


def replay(epochs):
    """Query -> number of updates applied before it; updates in applied order."""
    seen, applied = {}, []
    for queries, updates in epochs:
        for q in queries:
            seen[q.i] = len(applied)
        for u in updates or []:
            applied.append(u.i)
    return seen, applied


def test_random_rounds_match_arrival_order():
    rng = random.Random(7)
    for trial in range(2000):
        n = rng.randint(0, 25)
        kinds = [rng.choice(["insert", "insert", "delete", "knn", "count", "report"]) for _ in range(n)]
        batch = [req(k, i) for i, k in enumerate(kinds)]
        epochs = plan_epochs(batch)
        assert epochs[-1][1] is None
        got = [r.i for q, u in epochs for r in list(q) + list(u or [])]
        assert sorted(got) == list(range(n))
        seen, applied = replay(epochs)
        assert applied == [i for i, k in enumerate(kinds) if k in ("insert", "delete")]
        for i, k in enumerate(kinds):
            if k not in ("insert", "delete"):
                assert seen[i] == sum(1 for kk in kinds[:i] if kk in ("insert", "delete")), (kinds, i)
        for _, updates in epochs[:-1]:
            # one delete alone, or inserts only
            assert len(updates) == 1 or all(u.kind == "insert" for u in updates)


def test_consecutive_inserts_share_one_epoch():
    batch = [req("knn", 0), req("insert", 1), req("insert", 2), req("insert", 3), req("count", 4),
             req("insert", 5), req("delete", 6), req("delete", 7), req("report", 8)]
    epochs = plan_epochs(batch)
    assert [([q.i for q in qs], [u.i for u in us] if us else None) for qs, us in epochs] == [
        ([0], [1, 2, 3]), ([4], [5]), ([], [6]), ([], [7]), ([8], None)]
