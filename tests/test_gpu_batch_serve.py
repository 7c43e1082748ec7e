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
