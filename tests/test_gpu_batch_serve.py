"""Independent problems through gbf_batch_solve and the serving loop.

Each problem's result must be bitwise the one it gets when solved alone
(same kernels, launch shapes that depend only on the problem, no atomics in
floating-point sums), its eigenvalues must match the known spectrum, and the
server must keep the admitted workspace within its HBM budget."""
import numpy as np
import pytest

from paper_1203_4031_gb300 import workloads as W

from feast_check import TOL_E, compare_eigs

pytestmark = pytest.mark.gpu


def make_problems(gbf, prec):
    import torch

    out = []
    for p in W.batched_generalized(count=10, nmin=64, nmax=320):
        A = gbf.fortran(torch.from_numpy(p.A).cuda())
        B = gbf.fortran(torch.from_numpy(p.B).cuda())
        f = p.apply_fpm(gbf.gbf_init())
        f[41] = prec
        out.append((p, gbf.DeviceProblem(A, B, p.emin, p.emax, p.m0, fpm=f)))
    for i, req in enumerate(W.serving_requests(count=6, nmin=96, nmax=400, seed=77)):
        A, B, a, b = W.serving_matrices(req)
        f = gbf.gbf_init()
        f[2] = 10
        f[41] = prec
        lam = np.sort(W.uniform(W.derive_seed(req["seed"], 1), req["n"]))
        p = W.Problem(f"serve-{i}", req["hermitian"], None, None, a, b, req["m0"], spectrum=lam)
        out.append((p, gbf.DeviceProblem(A, B, a, b, req["m0"], fpm=f)))
    return out


def alone(gbf, dp):
    import torch

    h = gbf.Handle()
    f = np.array(dp.p.fpm[:], dtype=np.int32)
    r = gbf.feast_dev(dp.A, dp.B, dp.p.emin, dp.p.emax, dp.p.m0, fpm=f, handle=h)
    torch.cuda.synchronize()
    h.close()
    return r


def check_result(p, dp, res):
    assert res.info == 0, (p.name, res.info)
    w = p.spectrum
    ref = w[(w >= p.emin) & (w <= p.emax)]
    assert res.M == len(ref)
    E = dp.E.cpu().numpy()[: res.M]
    assert compare_eigs(E, ref, p.emin, p.emax) < TOL_E


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_matches_alone(gbf, prec):
    probs = make_problems(gbf, prec)
    rc, outs = gbf.batch_solve([dp for _, dp in probs], nworkers=4)
    import torch

    torch.cuda.synchronize()
    assert rc == 0
    got = [(dp.E.clone(), dp.X.clone(), r.as_dict()) for (_, dp), r in zip(probs, outs)]
    for (p, dp), r in zip(probs, outs):
        check_result(p, dp, r)
    for (p, dp), (E, X, rd) in zip(probs, got):
        ra = alone(gbf, dp)
        assert ra["info"] == rd["info"] and ra["M"] == rd["M"] and ra["loop"] == rd["loop"]
        assert torch.equal(ra["E"], E) and torch.equal(ra["X"], X)


def test_server_alone_vs_mix_and_budget(gbf):
    import torch

    probs = make_problems(gbf, 1)
    sizes = [dp.bytes() for _, dp in probs]
    budget = 3 * max(sizes)
    srv = gbf.Server(budget, nworkers=4)
    tickets = [srv.submit(dp) for _, dp in probs]
    results = [srv.wait(t) for t in tickets]
    st = srv.stats()
    assert st["peak"] <= budget and st["in_use"] == 0
    mixed = [(dp.E.clone(), dp.X.clone()) for _, dp in probs]
    for (p, dp), r in zip(probs, results):
        check_result(p, dp, r)
        assert r.queue_ms >= 0.0 and r.run_ms > 0.0
    for (p, dp), (E, X) in zip(probs, mixed):
        ra = alone(gbf, dp)
        assert torch.equal(ra["E"], E) and torch.equal(ra["X"], X)
    # a request that can never fit the budget fails with info -1
    small = gbf.Server(min(sizes) // 2, nworkers=1)
    r = small.wait(small.submit(probs[0][1]))
    assert r.info == -1
    small.close()
    srv.close()


def test_batch_full_range_and_worker_counts(gbf):
    """Config 4's whole size range (n up to 1024): every count exact, and the
    results bitwise the same for 1, 5 and 12 workers (the worker count only
    changes what overlaps on the GPU)."""
    import torch

    ps = W.batched_generalized(count=12, nmin=512, nmax=1024, seed=99)
    assert max(p.n for p in ps) > 800
    runs = []
    for nw in (1, 5, 12):
        dps = []
        for p in ps:
            A = gbf.fortran(torch.from_numpy(p.A).cuda())
            B = gbf.fortran(torch.from_numpy(p.B).cuda())
            dps.append(gbf.DeviceProblem(A, B, p.emin, p.emax, p.m0, fpm=p.apply_fpm(gbf.gbf_init())))
        rc, outs = gbf.batch_solve(dps, nworkers=nw)
        torch.cuda.synchronize()
        assert rc == 0
        for p, dp, r in zip(ps, dps, outs):
            check_result(p, dp, r)
        runs.append([(dp.E.cpu().numpy().copy(), dp.X.cpu().numpy().copy()) for dp in dps])
    for other in runs[1:]:
        for (e0, x0), (e1, x1) in zip(runs[0], other):
            assert np.array_equal(e0, e1) and np.array_equal(x0, x1)


def test_autotuner_picks_and_applies(gbf, tmp_path):
    """The autotuner times the batched solve, returns a worker count among
    its candidates and a width per size bucket, and its table (saved and
    loaded back) drives batch_solve to exact counts."""
    import torch

    from paper_1203_4031_gb300 import autotune

    ps = W.batched_generalized(count=8, nmin=64, nmax=400, seed=5)

    def make():
        out = []
        for p in ps:
            A = gbf.fortran(torch.from_numpy(p.A).cuda())
            B = gbf.fortran(torch.from_numpy(p.B).cuda())
            out.append(gbf.DeviceProblem(A, B, p.emin, p.emax, p.m0, fpm=p.apply_fpm(gbf.gbf_init())))
        return out

    entry = autotune.tune(make(), workers=(2, 4), widths=(0, 16), reps=1)
    assert entry["workers"] in (2, 4)
    assert set(entry["width"].values()) <= {0, 16}
    path = autotune.save(autotune.merge([entry], name="test"), str(tmp_path / "tune.json"))
    table = autotune.load(path)
    dps = make()
    rc, outs = autotune.batch_solve(dps, table)
    torch.cuda.synchronize()
    assert rc == 0
    for p, dp, r in zip(ps, dps, outs):
        check_result(p, dp, r)
