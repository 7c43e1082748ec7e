"""Host logic of the node sharding (the guide's second level of parallelism,
"Using the FEAST-MPI version") on CPU with two gloo ranks, no GPU:

* the node partition of gbf_shard_nodes (the C library's own rule) covers
  every node exactly once, in equal-sized exchange chunks;
* the exchange step (paper_1203_4031_gb300.shard.DistExchange, the same
  all-gather the GPU path calls back into) delivers every rank's node
  solution blocks to every rank, and the status agreement returns the
  minimum code;
* a FEAST subspace iteration in which each rank solves only its own nodes
  with the oracle's LU and triangular solves, then gathers all node blocks,
  sums Q in node order and runs the Rayleigh-Ritz step itself, reproduces the
  oracle's first filtered subspace (fpm(14)=1) and its converged eigenpairs,
  with the same result on both ranks.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_nodes_partition():
    from paper_1203_4031_gb300 import shard

    for ne in range(1, 21):
        for G in range(1, 13):
            seen = []
            chunks = set()
            for g in range(G):
                first, count, chunk = shard.shard_nodes(ne, g, G)
                assert 0 <= count <= chunk and chunk == -(-ne // G)
                seen += list(range(first, first + count))
                chunks.add(chunk)
            assert seen == list(range(ne)) and len(chunks) == 1
    with pytest.raises(ValueError):
        shard.shard_nodes(8, 2, 2)


def _problem(n=60, count=6, seed=7):
    r = np.random.default_rng(seed)
    M = r.standard_normal((n, n))
    A = 0.5 * (M + M.T)
    G = r.standard_normal((n, n))
    B = G @ G.T / n + np.eye(n)
    import scipy.linalg as sl

    w = sl.eigh(A, B, eigvals_only=True)
    mid = n // 2
    return A, B, 0.5 * (w[mid - 1] + w[mid]), 0.5 * (w[mid - 1 + count] + w[mid + count])


def _rank(rank, world, port, out_dir):
    import scipy.linalg as sl
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import oracle
    from paper_1203_4031_gb300 import shard

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ex = shard.DistExchange()
    out = {}

    # status agreement: the minimum over ranks
    out["agree"] = [ex.agree(0), ex.agree(-2 if rank == 1 else 0), ex.agree(-4 if rank == 0 else -2)]

    A, B, emin, emax = _problem()
    n, m0, ne = A.shape[0], 12, 8
    z, w = oracle.contour(emin, emax, ne)
    first, count, chunk = shard.shard_nodes(ne, rank, world)
    fpm = oracle.feastinit()
    # the oracle's initial subspace (fpm(5)=0) is not exposed; start both the
    # sharded loop and a second oracle run from the same explicit subspace
    Y = np.asarray(np.random.default_rng(11).uniform(-1, 1, (n, m0)), order="F")
    fpm5 = fpm.copy()
    fpm5[4] = 1
    ref1 = oracle.feast(A, B, emin, emax, m0, fpm=np.where(np.arange(64) == 13, 1, fpm5).astype(np.int32), X0=Y)
    ref = oracle.feast(A, B, emin, emax, m0, fpm=fpm5, X0=Y)
    alpha = max(abs(emin), abs(emax))
    m = m0
    for k in range(20):
        RHS = B @ Y
        buf = torch.zeros((world * chunk, n, m), dtype=torch.complex128)
        for e in range(first, first + count):
            lu, ipiv, info = oracle.zgetrf(z[e] * B - A)
            assert info == 0
            buf[e] = torch.from_numpy(np.ascontiguousarray(oracle.zgetrs(lu, ipiv, RHS)))
        flat = torch.view_as_real(buf).reshape(-1)
        ex.allgather_(flat, flat.numel() // world)
        Ys = buf.numpy()
        Q = np.zeros((n, m))
        for e in range(ne):                    # node order, as the library sums
            Q += np.real(w[e] * Ys[e])
        if k == 0:
            out["q0_err"] = float(np.max(np.abs(Q - ref1["X"][:, :m])) / np.max(np.abs(Q)))
        Aq, Bq = Q.T @ A @ Q, Q.T @ B @ Q
        lam, W = sl.eigh(0.5 * (Aq + Aq.T), 0.5 * (Bq + Bq.T))
        X = Q @ W
        R = A @ X - (B @ X) * lam[None, :]
        res = np.sum(np.abs(R), axis=0) / np.sum(np.abs(alpha * (B @ X)), axis=0)
        inside = (lam >= emin) & (lam <= emax)
        code = 0 if np.max(res[inside]) < 10.0 ** -fpm[2] else 1
        # both ranks hold the same numbers, so they stop together; the
        # agreement is the library's guard for that
        if ex.agree(-code) == 0:
            break
        Y = np.asarray(X, order="F")
    out["loops"] = k
    out["E"] = lam[inside].tolist()
    out["ref_E"] = ref["E"][:ref["M"]].tolist()
    out["ref_M"] = ref["M"]
    np.save(os.path.join(out_dir, f"X{rank}.npy"), X[:, inside])
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(repr(out))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sharded_feast(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world, port = 2, _free_port()
    mp.spawn(_rank, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    outs = [eval(open(tmp_path / f"r{r}.txt").read()) for r in range(world)]  # noqa: S307 - our own repr
    for o in outs:
        assert o["agree"] == [0, -2, -4]
        assert o["q0_err"] < 1e-12
        assert o["ref_M"] == 6 and len(o["E"]) == 6
        E, Er = np.array(o["E"]), np.array(o["ref_E"])
        assert np.max(np.abs(E - Er) / np.maximum(np.abs(Er), 1e-3)) < 1e-10
    assert outs[0]["E"] == outs[1]["E"] and outs[0]["loops"] == outs[1]["loops"]
    assert np.array_equal(np.load(tmp_path / "X0.npy"), np.load(tmp_path / "X1.npy"))
