"""Node sharding (the guide's second level of parallelism, "Using the
FEAST-MPI version") exercised as G logical shards on one device: G threads,
each with its own handle and stream, call gbf_dsygv_dev_shard /
gbf_zhegv_dev_shard for shard g of G, and exchange the node solution blocks
through host-ordered device copies (paper_1203_4031_gb300.shard.ThreadShards).

Every shard factors and solves only its own nodes; after the exchange all of
them sum Q in node order and run the same Rayleigh-Ritz step, so each shard's
E, X, res, M and loop must equal, bit for bit, those of the unsharded
gbf_dsygv_dev / gbf_zhegv_dev on the same inputs -- for shard counts that
divide Ne, that do not, and that leave a shard without nodes."""
import threading

import numpy as np
import pytest
import scipy.linalg as sl

from paper_1203_4031_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _problem(herm, gen, n, count, seed):
    r = np.random.default_rng(seed)
    M = r.standard_normal((n, n)) + (1j * r.standard_normal((n, n)) if herm else 0)
    A = 0.5 * (M + M.conj().T)
    B = None
    if gen:
        G = r.standard_normal((n, n)) + (1j * r.standard_normal((n, n)) if herm else 0)
        B = G @ G.conj().T / n + np.eye(n)
    w = sl.eigh(A, B, eigvals_only=True)
    mid = n // 2
    return A, B, 0.5 * (w[mid - 1] + w[mid]), 0.5 * (w[mid - 1 + count] + w[mid + count])


def _run_sharded(gbf, shard, A, B, emin, emax, m0, fpm, G):
    import torch

    ts = shard.ThreadShards(G)
    out = [None] * G
    err = []

    def worker(g):
        try:
            torch.cuda.set_device(A.device)
            h = gbf.Handle()
            s = torch.cuda.Stream(device=A.device)
            out[g] = shard.feast_dev_shard(A, B, emin, emax, m0, ts.callbacks(g), fpm=fpm, handle=h, stream=s)
            s.synchronize()
            h.close()
        except Exception as e:  # noqa: BLE001 - surfaced by the assertion below
            err.append(e)

    th = [threading.Thread(target=worker, args=(g,)) for g in range(G)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not err, err
    return out


def _same(a, b):
    for k in ("info", "M", "loop", "m0", "epsout"):
        assert a[k] == b[k], (k, a[k], b[k])
    for k in ("E", "res", "X"):
        assert a[k].shape == b[k].shape
        assert bool((a[k] == b[k]).all()), k


CASES = [
    # herm, gen, n, count, m0, ne, prec, shard counts
    (False, True, 300, 30, 45, 8, 0, (2, 3, 5)),
    (True, False, 257, 20, 32, 8, 0, (2, 3)),
    (True, True, 130, 15, 24, 8, 1, (2, 4)),
    (False, False, 200, 12, 20, 6, 1, (4,)),
]


@pytest.mark.parametrize("herm,gen,n,count,m0,ne,prec,Gs", CASES)
def test_logical_shards_bitwise_equal_to_unsharded(gbf, herm, gen, n, count, m0, ne, prec, Gs):
    import torch

    from paper_1203_4031_gb300 import shard

    A, B, emin, emax = _problem(herm, gen, n, count, seed=n + ne)
    At = gbf.fortran(torch.from_numpy(A).cuda())
    Bt = gbf.fortran(torch.from_numpy(B).cuda()) if B is not None else None
    fpm = gbf.gbf_init()
    fpm[1] = ne
    fpm[41] = prec
    h = gbf.Handle()
    ref = gbf.feast_dev(At, Bt, emin, emax, m0, fpm=fpm, handle=h)
    torch.cuda.synchronize()
    h.close()
    assert ref["info"] == 0 and ref["M"] == count, (ref["info"], gbf.last_error())
    for G in Gs:
        outs = _run_sharded(gbf, shard, At, Bt, emin, emax, m0, fpm, G)
        for g, o in enumerate(outs):
            _same(o, ref)
        # the shards' node sets partition the nodes
        got = []
        for g in range(G):
            first, count_g, _ = shard.shard_nodes(ne, g, G)
            got += list(range(first, first + count_g))
        assert got == list(range(ne))


def test_shard_nonfinite_input_stops_every_shard(gbf):
    """A NaN in A is found while the shifted systems are formed (-2); with 5
    shards of 8 nodes the last shard holds no node and learns it through the
    status agreement, so every shard stops with -2 at the same point."""
    import torch

    from paper_1203_4031_gb300 import shard

    A, B, emin, emax = _problem(False, True, 96, 8, seed=3)
    A[5, 7] = A[7, 5] = np.nan
    At = gbf.fortran(torch.from_numpy(A).cuda())
    Bt = gbf.fortran(torch.from_numpy(B).cuda())
    assert shard.shard_nodes(8, 4, 5)[1] == 0
    outs = _run_sharded(gbf, shard, At, Bt, emin, emax, 16, gbf.gbf_init(), 5)
    assert [o["info"] for o in outs] == [-2] * 5
    h = gbf.Handle()
    assert gbf.feast_dev(At, Bt, emin, emax, 16, handle=h)["info"] == -2
    assert "non-finite" in gbf.last_error()
    h.close()


def test_shard_full_size_real_generalized(gbf):
    """The n=4096 benchmark problem (Ne=8) as 2 logical shards: same result
    bits as the unsharded solve."""
    import torch

    from paper_1203_4031_gb300 import shard

    p = W.dense_real_generalized()
    A = gbf.fortran(torch.from_numpy(np.ascontiguousarray(p.A)).cuda())
    B = gbf.fortran(torch.from_numpy(np.ascontiguousarray(p.B)).cuda())
    fpm = p.apply_fpm(gbf.gbf_init())
    h = gbf.Handle()
    ref = gbf.feast_dev(A, B, p.emin, p.emax, p.m0, fpm=fpm, handle=h)
    torch.cuda.synchronize()
    h.close()
    assert ref["info"] == 0 and ref["M"] == 200
    outs = _run_sharded(gbf, shard, A, B, p.emin, p.emax, p.m0, fpm, 2)
    for o in outs:
        _same(o, ref)
