"""Many independent indexes built in one persistent launch: every index must get
exactly the layout and query results of its own build (oracle, bit-exact), for
every block size, and the whole build + query sequence must replay from a CUDA
graph with the same results."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2601_05347_gb300 import gen  # noqa: E402

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2601_05347_gb300 import psi


def T(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to("cuda")


def make_batch(sizes, dim=2, bits=30, seed=1):
    pts, ids = [], []
    for i, n in enumerate(sizes):
        p = gen.varden(n, dim, bits, seed * 1000 + i) if i % 2 else gen.uniform(n, dim, bits, seed * 1000 + i)
        if i % 5 == 3 and n:
            p = (p >> (bits - 5)).astype(np.int32)  # piles of duplicate points
        pts.append(p)
        ids.append((np.arange(n, dtype=np.uint32) * 2654435761 + i * 7919) & 0xFFFFFFFF)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return np.concatenate(pts).astype(np.int32).reshape(-1, dim), np.concatenate(ids).astype(np.uint32), off


def queries(sizes, pts, off, dim, bits, seed):
    qs, qoff = [], [0]
    for i, n in enumerate(sizes):
        nq = 1 + (i * 37) % 90
        q = gen.uniform(nq, dim, bits, seed + i)
        if n:
            q[: nq // 2] = pts[off[i] + gen.sample_with_replacement(n, nq // 2, seed + 3 * i)]
        qs.append(q)
        qoff.append(qoff[-1] + nq)
    return np.concatenate(qs).astype(np.int32), np.array(qoff, np.int64)


SIZES = [0, 1, 31, 32, 33, 1000, 4095, 4097, 12345, 70001, 5, 800, 0, 3000, 9000, 40]


@pytest.mark.parametrize("kind", ["spac_z", "spac_h"])
@pytest.mark.parametrize("threads,radix_bits", [(256, 8), (512, 8), (1024, 8), (256, 11), (512, 11)])
@pytest.mark.parametrize("phi", [16, 32, 64])
def test_batch_layout_and_knn_match_oracle(kind, threads, radix_bits, phi):
    # every leaf size, block size and digit width the autotuner can choose
    pts, ids, off = make_batch(SIZES)
    b = psi.Batch(off, kind=kind, leaf_size=phi, threads=threads, radix_bits=radix_bits)
    b.build(T(pts), T(ids))
    q, qoff = queries(SIZES, pts, off, 2, 30, 5)
    gi, gd = b.knn(T(q), T(qoff), 10)
    b.sync()
    gi, gd = gi.cpu().numpy().view(np.uint32), gd.cpu().numpy()
    okind = O.SPAC_Z if kind == "spac_z" else O.SPAC_H
    for i, n in enumerate(SIZES):
        o = O.Index(pts[off[i]:off[i + 1]], ids[off[i]:off[i + 1]], kind=okind, phi=phi)
        lv = o.levels()
        gl = b.leaves(i)
        if n == 0:
            assert gl["count"].numel() == 0
        else:
            assert (gl["count"].cpu().numpy() == lv[0]["count"]).all()
            assert (gl["lo"].cpu().numpy() == lv[0]["lo"]).all()
            assert (gl["hi"].cpu().numpy() == lv[0]["hi"]).all()
        oi, od = o.knn(q[qoff[i]:qoff[i + 1]], 10)
        assert (gi[qoff[i]:qoff[i + 1]] == oi).all(), i
        assert (gd[qoff[i]:qoff[i + 1]] == od).all(), i


@pytest.mark.parametrize("kind", ["spac_z", "spac_h"])
def test_batch_3d_and_k100(kind):
    sizes = [500, 20000, 3, 7000]
    pts, ids, off = make_batch(sizes, dim=3, bits=21, seed=4)
    b = psi.Batch(off, dim=3, kind=kind, leaf_size=16, coord_bits=21, threads=256, radix_bits=11)
    b.build(T(pts), T(ids))
    q, qoff = queries(sizes, pts, off, 3, 21, 9)
    gi, gd = b.knn(T(q), T(qoff), 100)
    gi, gd = gi.cpu().numpy().view(np.uint32), gd.cpu().numpy()
    for i in range(len(sizes)):
        oi, od = O.knn_brute_raw(pts[off[i]:off[i + 1]], ids[off[i]:off[i + 1]], q[qoff[i]:qoff[i + 1]], 100)
        assert (gi[qoff[i]:qoff[i + 1]] == oi).all() and (gd[qoff[i]:qoff[i + 1]] == od).all()


def test_batch_replays_from_cuda_graph():
    pts, ids, off = make_batch(SIZES, seed=7)
    b = psi.Batch(off, kind="spac_h", leaf_size=32)
    q, qoff = queries(SIZES, pts, off, 2, 30, 11)
    dp, di, dq, dqo = T(pts), T(ids), T(q), T(qoff)
    b.reserve(len(q))
    out_i = torch.empty((len(q), 10), dtype=torch.int32, device="cuda")
    out_d = torch.empty((len(q), 10), dtype=torch.int64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up outside the capture
        b.build(dp, di)
        b.knn(dq, dqo, 10, out_i, out_d)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    want_i, want_d = out_i.clone(), out_d.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.build(dp, di)
        b.knn(dq, dqo, 10, out_i, out_d)
    out_i.zero_()
    out_d.zero_()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out_i, want_i) and torch.equal(out_d, want_d)
    o = O.Index(pts[off[9]:off[10]], ids[off[9]:off[10]], kind=O.SPAC_H, phi=32)
    oi, od = o.knn(q[qoff[9]:qoff[10]], 10)
    assert (out_i.cpu().numpy().view(np.uint32)[qoff[9]:qoff[10]] == oi).all()


def test_batch_knn_instrumented_matches_and_counts():
    pts, ids, off = make_batch(SIZES, seed=13)
    b = psi.Batch(off, kind="spac_h", leaf_size=32)
    b.build(T(pts), T(ids))
    q, qoff = queries(SIZES, pts, off, 2, 30, 17)
    gi, gd = b.knn(T(q), T(qoff), 10)
    si, sd, st = b.knn_stats(T(q), T(qoff), 10)
    assert torch.equal(gi, si) and torch.equal(gd, sd)
    assert st["queries"] == len(q)
    # every query of a non-empty index scans at least one leaf; points scanned
    # are at most 2*phi per leaf
    nonempty = sum(int(qoff[i + 1] - qoff[i]) for i, n in enumerate(SIZES) if n)
    assert st["leaves"] >= nonempty and st["points"] <= 64 * st["leaves"]
