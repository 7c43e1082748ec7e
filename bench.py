#!/usr/bin/env python
"""Benchmark: converged eigenpairs/s of FEAST (Hermitian family) on one GB300.

Workload (default): the n=4096 dense real symmetric generalized problem
A = Q diag(lam) Q^T, B = Q_B diag(mu) Q_B^T (8 seeded Householder reflectors
each, lam ~ U[-1,1], mu log-uniform [1,100]), interval [-delta, delta]
holding 200 eigenvalues, M0 = 300, Ne = 8 Gauss-Legendre half-contour
nodes, residual criterion 1e-10.  Synthetic inputs, seeded.

A step = one complete FEAST solve through the C ABI (gbf_dsygv_dev): shifted
LU of all nodes, every subspace iteration (solves, quadrature sum,
Rayleigh-Ritz GEMMs, reduced eigenproblem, residuals) until convergence,
inputs resident in HBM.  value = eigenpairs with per-pair residual
||Ax - lBx||/(||A|| ||x||) <= 1e-10 per second.  On N > 1 GPUs (torchrun,
NCCL) the one problem is node-sharded (gbf_dsygv_dev_shard: each rank
factors and solves Ne/N of the contour nodes, one all-gather of the node
solution blocks per iteration, Rayleigh-Ritz replicated): strong scaling,
value = the problem's pairs over the slowest rank's time.
The FP64 path (fpm(42)=0) gives `value`; the mixed path (FP32 factor/solve
with FP64 correction, fpm(42)=1) is measured the same way under "mixed".

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_PEAK_NOMINAL = 1.25e12      # GB300 FP64 (CUDA cores), nominal
FP32_PEAK_NOMINAL = 152 * 128 * 2 * 2.07e9   # 152 SMs x 128 FP32 FMA/clk x 2 x 2.07 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbf", choices=["gbf", "reference"])
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--only", choices=["fp64", "mixed"], default=None,
                    help="time one path only (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving and batched samples")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the headline serving run (mixed path, 0.7 x saturated rate)")
    ap.add_argument("--serve-side-requests", type=int, default=500,
                    help="requests of the other serving runs (0.5 / 0.9 load, FP64 path, small budget)")
    ap.add_argument("--serve-pool", type=int, default=256,
                    help="distinct serving problems the requests cycle through")
    ap.add_argument("--batch-problems", type=int, default=256)
    ap.add_argument("--no-herm", action="store_true", help="skip the complex Hermitian n=8192 sample")
    ap.add_argument("--no-stoch", action="store_true", help="skip the stochastic-count sample (fpm(14)=2)")
    ap.add_argument("--no-gen", action="store_true", help="skip the non-Hermitian samples")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1].split()[0]))
                mx.append(float(p[2].split()[0]))
            except ValueError:
                continue
            for k, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- workload --
def workload():
    from paper_1203_4031_gb300 import workloads as W

    return W.dense_real_generalized()


METRIC = "converged eigenpairs/s at residual<=1e-10 (FP64 FEAST; mixed under 'mixed')"


def workload_name(p):
    return (f"{p.name}: dense real symmetric generalized, n={p.n}, M0={p.m0}, Ne=8, "
            f"[-{p.emax:.6g},{p.emax:.6g}] holding 200, res<1e-10")


def combine_shards(ms, pairs, dist, device):
    """Whole-job figures of one node-sharded problem: the slowest rank's time
    (max) and the problem's pairs (every rank holds the same result; the
    minimum guards against a rank that disagrees)."""
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    tot = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.MIN)
    return t.item(), tot.item()


def combine_ranks(ms, pairs, dist, device):
    """Whole-job figures over the ranks (independent replicas, no data-path
    collective): the slowest rank's time (max) and the pairs of all ranks
    (sum).  `dist` is torch.distributed (nccl on GPUs, gloo in the CPU test)
    or None for one rank."""
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    tot = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return t.item(), tot.item()


def gate_count(A, B, X, E, M, torch):
    """Pairs (of the first M) with ||Ax - lBx||_2 / (||A||_1 ||x||_2) <= 1e-10."""
    Xm = X[:, :M]
    Em = E[:M]
    R = A @ Xm - (B @ Xm) * Em[None, :]
    nA = torch.linalg.matrix_norm(A, ord=1)
    rel = torch.linalg.vector_norm(R, dim=0) / (nA * torch.linalg.vector_norm(Xm, dim=0))
    return int((rel <= 1e-10).sum().item()), float(rel.max().item()) if M else 0.0


def run_gbf(args):
    import torch

    import paper_1203_4031_gb300 as g

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    g.load()
    p = workload()
    n, m0 = p.n, p.m0
    dev = torch.device("cuda", local)
    A = g.fortran(torch.from_numpy(np.ascontiguousarray(p.A)).to(dev))
    B = g.fortran(torch.from_numpy(np.ascontiguousarray(p.B)).to(dev))
    h = g.Handle()
    stream = torch.cuda.current_stream(dev)
    cbs = None
    if dist:
        from paper_1203_4031_gb300 import shard

        cbs = shard.DistExchange().callbacks()

    def fpm_for(prec):
        f = p.apply_fpm(g.gbf_init())
        f[41] = prec
        return f

    def solve(prec, A_=None, B_=None):
        A_ = A if A_ is None else A_
        B_ = B if B_ is None else B_
        if cbs is not None:
            return shard.feast_dev_shard(A_, B_, p.emin, p.emax, m0, cbs, fpm=fpm_for(prec), handle=h,
                                         stream=stream)
        return g.feast_dev(A_, B_, p.emin, p.emax, m0, fpm=fpm_for(prec), handle=h, stream=stream)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()

    def timed(prec, steps, warm, profile=False, clocks=None):
        for _ in range(warm):
            r = solve(prec)
            if r["info"] != 0:
                raise RuntimeError(f"warm-up solve failed: info {r['info']} ({g.last_error()})")
        barrier()
        if clocks:
            clocks.start()
        if profile:
            g.lib().gbf_profile(1)
        l0 = g.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        rs = [solve(prec) for _ in range(steps)]
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        launches = g.launch_count() - l0
        cl = clocks.stop() if clocks else None
        prof = tc = None
        if profile:
            import ctypes as C

            L = g.lib()
            L.gbf_profile_name.restype = C.c_char_p
            prof = {}
            for c in range(L.gbf_profile_categories()):
                nl, t, fl = C.c_longlong(), C.c_double(), C.c_double()
                L.gbf_profile_read(c, C.byref(nl), C.byref(t), C.byref(fl))
                prof[L.gbf_profile_name(c).decode()] = (nl.value, t.value, fl.value)
            nl, t, fl, tf = C.c_longlong(), C.c_double(), C.c_double(), C.c_double()
            L.gbf_profile_tc(C.byref(nl), C.byref(t), C.byref(fl), C.byref(tf))
            tc = (nl.value, t.value, fl.value, tf.value)
            L.gbf_profile(0)
        r = rs[-1]
        if any(x["info"] != 0 for x in rs):
            raise RuntimeError(f"timed solve failed: {[x['info'] for x in rs]}")
        ok, worst = gate_count(A, B, r["X"], r["E"], r["M"], torch)
        ms_all, pairs_all = combine_shards(ms, ok * steps, dist, dev)
        return dict(ms=ms_all, pairs=pairs_all, M=r["M"], ok=ok, worst=worst, loop=r["loop"],
                    launches=launches, prof=prof, tc=tc, clocks=cl)

    if args.only == "mixed":
        mx = timed(1, args.steps, args.warmup)
        mx["prof"] = timed(1, 1, 0, profile=True)["prof"]
        if rank == 0:
            print(json.dumps({"path": "mixed", "ms_per_step": mx["ms"] / args.steps, "M": mx["M"],
                              "kernels_ms": {k: v[1] for k, v in mx["prof"].items()}}), flush=True)
        return
    # the timed steps run without per-launch profiling events; one more
    # profiled step gives the per-category kernel times
    clocks = ClockSampler(local)
    fp = timed(0, args.steps, args.warmup, clocks=clocks)
    pr = timed(0, 1, 0, profile=True)
    fp["prof"], fp["tc"] = pr["prof"], pr["tc"]
    value = fp["pairs"] / (fp["ms"] / 1e3)
    mixed = None
    if not args.no_mixed and args.only is None:
        mx = timed(1, args.steps, args.warmup)
        pr = timed(1, 1, 0, profile=True)
        mx["prof"], mx["tc"] = pr["prof"], pr["tc"]
        mixed = {"value": mx["pairs"] / (mx["ms"] / 1e3), "ms_per_step": mx["ms"] / args.steps,
                 "M": mx["M"], "loops": mx["loop"], "max_rel_residual": mx["worst"],
                 "gpu_launches": mx["launches"], "dtype": "c32 factor/solve + f64 correction",
                 "kernels_ms": {k: round(v[1], 3) for k, v in mx["prof"].items()},
                 "roofline": roofline(mx["prof"], mx["tc"], "mixed", p.n, int(p.fpm.get(2, 8)))}

    # end to end through the public API from pinned host buffers: H2D of A
    # and B and D2H of E, X, res inside the timed region
    e2e = None
    if not args.no_e2e:
        Ah = torch.from_numpy(np.asfortranarray(p.A).ravel(order="F")).pin_memory()
        Bh = torch.from_numpy(np.asfortranarray(p.B).ravel(order="F")).pin_memory()
        a_np = Ah.numpy().reshape((n, n), order="F")
        b_np = Bh.numpy().reshape((n, n), order="F")
        ks = max(1, min(args.steps, 3))
        if dist is None:
            def e2e_step():
                return g.feast_host(a_np, b_np, p.emin, p.emax, m0, fpm=fpm_for(0))
            api = "gbf_dsygv (host pointers, pinned)"
        else:
            Ad = torch.empty((n, n), dtype=torch.float64, device=dev)
            Bd = torch.empty((n, n), dtype=torch.float64, device=dev)
            Eh = torch.empty(m0, dtype=torch.float64).pin_memory()
            Rh = torch.empty(m0, dtype=torch.float64).pin_memory()
            Xh = torch.empty((m0, n), dtype=torch.float64).pin_memory()

            def e2e_step():
                Ad.copy_(Ah.view(n, n), non_blocking=True)   # column-major bytes as a row-major view
                Bd.copy_(Bh.view(n, n), non_blocking=True)
                r = solve(0, Ad.t(), Bd.t())
                Eh.copy_(r["E"], non_blocking=True)
                Rh.copy_(r["res"], non_blocking=True)
                Xh.copy_(r["X"].t(), non_blocking=True)
                torch.cuda.synchronize(dev)
                return r
            api = "gbf_dsygv_dev_shard (pinned host buffers copied in and out)"
        rh = e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(ks):
            rh = e2e_step()
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        dt_all, _ = combine_shards(dt, 0, dist, dev)
        e2e = {"value": (rh["M"] * ks) / dt_all, "unit": "eigenpairs/s",
               "h2d_bytes_per_step": 2 * n * n * 8, "d2h_bytes_per_step": (n * m0 + 2 * m0) * 8,
               "steps": ks, "api": api}

    stoch = None
    if not args.no_stoch and args.only is None and world == 1:
        stoch = run_stochastic(g, torch, p, A, B, h, stream)

    serving = batched = herm = None
    if not args.no_serve and args.only is None and world == 1:
        from paper_1203_4031_gb300 import workloads as W

        # config 5 is quoted on the mixed path with the FP64 run beside it;
        # config 4 on both
        serving = run_serving_suite(g, torch, W, args)
        batched = run_batched_suite(g, torch, W, args.batch_problems)
        if not args.no_herm:
            herm = run_hermitian(g, torch, W)
    gen = None
    if not args.no_gen and args.only is None and world == 1:
        from paper_1203_4031_gb300 import workloads as W

        gen = run_nonhermitian(g, torch, W)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(p, fp["M"])

    if rank == 0:
        sv = (serving or {}).get("mixed", {}).get("load_0.7", {})
        summary = {"fp64_eigenpairs_per_s": round(value, 1), "fp64_ms_per_step": round(fp["ms"] / args.steps, 2),
                   "mixed_eigenpairs_per_s": round(mixed["value"], 1) if mixed else None,
                   "mixed_ms_per_step": round(mixed["ms_per_step"], 2) if mixed else None,
                   "serving_mixed_p50_ms": sv.get("p50_ms"), "serving_mixed_p99_ms": sv.get("p99_ms"),
                   "serving_mixed_eigenpairs_per_s": sv.get("eigenpairs_per_s"),
                   "batched_fp64_eigenpairs_per_s": (batched or {}).get("fp64", {}).get("eigenpairs_per_s"),
                   "batched_mixed_eigenpairs_per_s": (batched or {}).get("mixed", {}).get("eigenpairs_per_s"),
                   "cpu_oracle_eigenpairs_per_s": cpu["value"] if cpu else None}
        line = {
            "metric": METRIC,
            "value": value, "unit": "eigenpairs/s", "n_gpus": world, "steps": args.steps,
            "mixed_value": mixed["value"] if mixed else None,
            "mixed_ms_per_step": mixed["ms_per_step"] if mixed else None,
            "warmup": args.warmup, "ms_per_step": fp["ms"] / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(p),
                       "M": fp["M"], "loops": fp["loop"],
                       "parallelism": "1 GPU" if world == 1 else f"node-shard x{world} (NCCL all-gather)",
                       "l2": "inputs A,B (2 x 134 MB) exceed L2 (129 MB)"},
            "max_rel_residual": fp["worst"], "gpu_launches": fp["launches"],
            "kernels_ms": {k: round(v[1], 3) for k, v in fp["prof"].items()},
            "roofline": roofline(fp["prof"], fp["tc"], "fp64"),
            "clocks": fp["clocks"], "e2e": e2e, "mixed": mixed, "serving": serving, "batched": batched,
            "hermitian_n8192": herm, "stochastic_count": stoch, "nonhermitian_n4096": gen,
            "cpu_baseline": cpu,
            "summary": summary,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()


class ServingPool:
    """The serving workload's problems (config 5 distribution: n log-uniform
    in [128, 4096], real symmetric generalized or complex Hermitian 50/50,
    intervals holding 8-64 eigenvalues, known spectra), built on the device
    once for the first `pool` request descriptors; request i solves problem
    i mod pool with its own output buffers (the server keeps no result cache,
    so every request is a full solve)."""

    def __init__(self, g, W, pool):
        self.g = g
        self.descs = W.serving_requests(count=pool, nmin=128, nmax=4096, rate=1.0)
        self.mats = [W.serving_matrices(rq) for rq in self.descs]

    def problem(self, i, prec):
        rq = self.descs[i % len(self.descs)]
        A, B, a, b = self.mats[i % len(self.descs)]
        f = self.g.gbf_init()
        f[2] = 10
        f[41] = prec
        return rq, self.g.DeviceProblem(A, B, a, b, rq["m0"], fpm=f)


def run_serving(g, torch, W, pool, n_req, rate, budget=120e9, nworkers=4, prec=0):
    """One serving run: n_req requests with Poisson arrivals at `rate`/s
    (rate None: all at once, the saturation run), submitted at their arrival
    times to gbf_server (HBM admission budget `budget`); latency = queue +
    run time per request; eigenpairs/s and requests/s over the span from the
    first arrival to the last completion.  A request whose workspace exceeds
    the whole budget is rejected (info -1) and counted apart."""
    arr = W.serving_requests(count=n_req, nmin=128, nmax=4096, rate=rate or 1.0)
    probs = [pool.problem(i, prec) for i in range(n_req)]
    torch.cuda.synchronize()
    srv = g.Server(budget, nworkers=nworkers)
    t0 = time.perf_counter()
    tickets = []
    for rq, (_, dp) in zip(arr, probs):
        if rate:
            dt = rq["t_arrival"] - arr[0]["t_arrival"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
        tickets.append(srv.submit(dp))
    res = [srv.wait(t) for t in tickets]
    span = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat = np.array([r.queue_ms + r.run_ms for r in res])
    rejected = sum(1 for r in res if r.info == -1)
    ok = all((r.info == 0 and r.M == rq["count"]) or r.info == -1 for (rq, _), r in zip(probs, res))
    return {"requests": n_req, "offered_rate_per_s": rate, "workers": nworkers, "hbm_budget_gb": budget / 1e9,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "eigenpairs_per_s": float(sum(r.M for r in res) / span),
            "requests_per_s": n_req / span, "span_s": span, "peak_admitted_gb": st["peak"] / 1e9,
            "rejected": rejected, "all_counts_exact": bool(ok)}


def run_serving_suite(g, torch, W, args):
    """Config 5: the saturated request rate of each path (all requests
    submitted at once), then Poisson streams offered at 0.5, 0.7 and 0.9 x
    that rate on the mixed path (headline: 0.7, args.serve_requests
    requests), the FP64 path at 0.7, and the mixed path at 0.7 under a 2 GB
    budget so that admission binds."""
    pool = ServingPool(g, W, args.serve_pool)
    side = args.serve_side_requests
    out = {"workload": f"serving requests (config 5 distribution): {args.serve_pool} distinct problems, "
                       "requests cycle through them"}
    for name, prec in (("mixed", 1), ("fp64", 0)):
        run_serving(g, torch, W, pool, 16, None, prec=prec)  # warm-up
        sat = run_serving(g, torch, W, pool, min(args.serve_pool, side), None, prec=prec)
        cap = sat["requests_per_s"]
        runs = {"saturated": sat}
        loads = (0.5, 0.7, 0.9) if name == "mixed" else (0.7,)
        for ld in loads:
            nr = args.serve_requests if (name == "mixed" and ld == 0.7) else side
            runs[f"load_{ld}"] = run_serving(g, torch, W, pool, nr, ld * cap, prec=prec)
        if name == "mixed":
            # a budget that holds the largest request with little to spare, so
            # that admission binds while every request still fits
            big = 1.25 * max(pool.problem(i, prec)[1].bytes() for i in range(len(pool.descs)))
            runs["load_0.7_tight_budget"] = run_serving(g, torch, W, pool, side, 0.7 * cap, budget=big, prec=prec)
        runs["paths"] = ("FP32 factors + FP64 correction (3xTF32 updates)" if prec
                         else "FP64 (tensor-core engine)")
        out[name] = runs
    return out


def run_stochastic(g, torch, p, A, B, h, stream, reps=3):
    """Stochastic eigenvalue count (fpm(14)=2) on the resident n=4096
    generalized problem (200 eigenvalues inside): one contour over M0 +-1
    probes, no Rayleigh-Ritz.  Device time per estimate (CUDA events, two
    warm-ups, `reps` timed calls) for the settings the guide suggests (few
    nodes, FP32 factors, small M0) and an FP64 one."""
    out = {"workload": f"{p.name}: estimate of the count in [-{p.emax:.6g},{p.emax:.6g}] (exact 200)"}
    for name, ne, m0, prec in (("ne3_m16_mixed", 3, 16, 1), ("ne3_m64_mixed", 3, 64, 1),
                               ("ne8_m64_fp64", 8, 64, 0)):
        f = p.apply_fpm(g.gbf_init())
        f[1], f[13], f[41] = ne, 2, prec
        E = torch.zeros(m0, dtype=torch.float64, device=A.device)
        res = torch.zeros(m0, dtype=torch.float64, device=A.device)
        X = torch.zeros((m0, p.n), dtype=A.dtype, device=A.device).t()
        for _ in range(2):
            r = g.feast_dev(A, B, p.emin, p.emax, m0, fpm=f, E=E, X=X, res=res, handle=h, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            r = g.feast_dev(A, B, p.emin, p.emax, m0, fpm=f, E=E, X=X, res=res, handle=h, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"ms": e0.elapsed_time(e1) / reps, "M": r["M"], "info": r["info"],
                     "mean": float(r["res"][m0 - 1].item()), "ne": ne, "m0": m0,
                     "dtype": "c32 factor/solve" if prec else "f64"}
    return out


def run_hermitian(g, torch, W):
    """Config 3: complex Hermitian standard problem n = 8192, Ne = 16, M0 = 240,
    interval [0, 0.04]; mixed and FP64 paths, one warm-up and one timed solve
    each; pairs pass the same 1e-10 residual gate and are checked against the
    known spectrum."""
    p = W.dense_complex_hermitian()
    A = g.fortran(torch.from_numpy(np.ascontiguousarray(p.A)).cuda())
    lam = p.spectrum
    ref = lam[(lam >= p.emin) & (lam <= p.emax)]
    h = g.Handle()
    out = {"workload": f"{p.name}: U diag(lam) U^H, B = I, [0, 0.04] holding {len(ref)}, M0 = {p.m0}, Ne = 16"}
    for name, prec in (("mixed", 1), ("fp64", 0)):
        f = p.apply_fpm(g.gbf_init())
        f[41] = prec
        g.feast_dev(A, None, p.emin, p.emax, p.m0, fpm=f, handle=h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = g.feast_dev(A, None, p.emin, p.emax, p.m0, fpm=f, handle=h)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        M = r["M"]
        ok, worst = gate_count(A, torch.eye(p.n, dtype=A.dtype, device=A.device), r["X"], r["E"].to(A.dtype), M,
                               torch) if r["info"] == 0 else (0, float("nan"))
        err = float(np.max(np.abs(r["E"][:M].cpu().numpy() - ref))) if M == len(ref) else float("nan")
        out[name] = {"eigenpairs_per_s": ok / dt, "ms": dt * 1e3, "M": M, "loops": r["loop"], "info": r["info"],
                     "max_rel_residual": worst, "max_abs_eig_err": err}
    h.close()
    return out


def run_nonhermitian(g, torch, W, n=4096, count=40, m0=64):
    """Non-Hermitian FEAST samples (dual subspaces, full contour, 16 nodes):
    a real non-symmetric generalized pencil (conjugate node pairs: 8
    factorisations) and a complex non-symmetric standard matrix (16), n =
    4096, a circle holding `count` eigenvalues of the known spectrum, M0 =
    m0; FP64 factors and FP32 factors with the FP64 residual correction
    (`_mixed`).  One warm-up and one timed solve each (CUDA events around the
    call, per-category kernel times and the sliced GEMMs' roofline from one
    more profiled solve); pairs counted when both residuals pass 1e-10 and
    the eigenvalue matches the known one to 1e-10."""
    import ctypes as C

    out = {}
    L = g.lib()
    for name, cplx, gen in (("real_generalized", False, True), ("complex_standard", True, False)):
        P = W.dense_nonsymmetric(n, count=count, m0=m0, complex_=cplx, generalized=gen)
        A = g.fortran(torch.from_numpy(np.ascontiguousarray(P.A)).cuda())
        B = g.fortran(torch.from_numpy(np.ascontiguousarray(P.B)).cuda()) if P.B is not None else None
        known = P.spectrum[np.abs(P.spectrum - P.emid) <= P.r]
        for prec in (0, 1):
            f = P.apply_fpm(g.gbf_init())
            f[41] = prec
            h = g.Handle()
            stream = torch.cuda.current_stream()
            r = g.feast_gen_dev(A, B, P.emid, P.r, P.m0, f, handle=h)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            l0 = g.launch_count()
            e0.record(stream)
            r = g.feast_gen_dev(A, B, P.emid, P.r, P.m0, f, handle=h)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            launches = g.launch_count() - l0
            L.gbf_profile(1)
            g.feast_gen_dev(A, B, P.emid, P.r, P.m0, f, handle=h)
            torch.cuda.synchronize()
            prof, prof_full = {}, {}
            for c in range(L.gbf_profile_categories()):
                nl, t, fl = C.c_longlong(), C.c_double(), C.c_double()
                L.gbf_profile_read(c, C.byref(nl), C.byref(t), C.byref(fl))
                prof[L.gbf_profile_name(c).decode()] = round(t.value, 3)
                prof_full[L.gbf_profile_name(c).decode()] = (nl.value, t.value, fl.value)
            nl, t, fl, tf = C.c_longlong(), C.c_double(), C.c_double(), C.c_double()
            L.gbf_profile_tc(C.byref(nl), C.byref(t), C.byref(fl), C.byref(tf))
            tc = (nl.value, t.value, fl.value, tf.value)
            L.gbf_profile(0)
            M = r["M"]
            E = r["E"][:M].cpu().numpy()
            res = r["res"].cpu().numpy()
            ok = 0
            err = float("nan")
            if r["info"] == 0 and M == len(known):
                d = np.array([np.min(np.abs(known - e)) for e in E])
                err = float(np.max(d))
                ok = int(np.sum((d < 1e-10) & (res[:M] < 1e-10) & (res[P.m0:P.m0 + M] < 1e-10)))
            key = name + ("_mixed" if prec else "")
            out[key] = {"workload": f"{P.name}: {P.note}; circle |z - {P.emid}| <= {P.r:.6g} holding {count}, "
                                    f"M0 = {P.m0}, fpm(8) = 16",
                        "factors": "c32 + f64 residual correction" if prec else "f64",
                        "eigenpairs_per_s": ok / (ms / 1e3), "ms": ms, "M": M, "loops": r["loop"],
                        "info": r["info"], "pairs_passing": ok, "max_abs_eig_err": err,
                        "max_res_right": float(np.max(res[:M])) if M else None,
                        "max_res_left": float(np.max(res[P.m0:P.m0 + M])) if M else None,
                        "biorth_defect": r["biorth"], "gpu_launches": launches, "kernels_ms": prof,
                        "roofline": roofline(prof_full, tc, "fp64") if prec == 0 else None}
            h.close()
        del A, B
        torch.cuda.empty_cache()
    return out


def run_batched_suite(g, torch, W, count, tune_sample=48):
    """Config 4: `count` independent real symmetric generalized problems
    (n log-uniform in [64, 1024], intervals holding 10-40, M0 = 1.5 count,
    Ne = 8), FP64 and mixed paths.  The autotuner (paper_1203_4031_gb300.
    autotune) first times gbf_batch_solve on the first `tune_sample`
    problems for each path (worker count, then the LU width per size
    bucket) and saves its table; the whole batch then runs once with the
    tuned settings (eigenpairs/s over the call), and once with the untuned
    default (4 workers, width 32) for comparison."""
    from paper_1203_4031_gb300 import autotune

    t0 = time.perf_counter()
    gen = W.batched_generalized(count=count, nmin=64, nmax=1024)
    mats = [(g.fortran(torch.from_numpy(p.A).cuda()), g.fortran(torch.from_numpy(p.B).cuda())) for p in gen]
    gen_s = time.perf_counter() - t0
    out = {"workload": f"batched generalized problems (config 4 distribution): {count} problems, "
                       f"n log-uniform in [64, 1024]", "generation_s": gen_s}
    entries = []
    for name, prec in (("fp64", 0), ("mixed", 1)):
        def make(ps):
            dps = []
            for p, (A, B) in ps:
                f = p.apply_fpm(g.gbf_init())
                f[41] = prec
                dps.append(g.DeviceProblem(A, B, p.emin, p.emax, p.m0, fpm=f))
            return dps
        pairs = list(zip(gen, mats))
        t0 = time.perf_counter()
        entry = autotune.tune(make(pairs[:tune_sample]))
        entries.append(entry)
        tune_s = time.perf_counter() - t0
        table = autotune.merge([entry])
        res = {}
        for label, tbl in (("tuned", table), ("default_4_workers", autotune.DEFAULT)):
            dps = make(pairs)
            nw = autotune.apply(dps, tbl) if label == "tuned" else 4
            if label != "tuned":
                for q in dps:
                    q.p.fpm[42] = 0
            g.batch_solve(dps[:nw], nworkers=nw)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, outs = g.batch_solve(dps, nworkers=nw)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            ok = rc == 0
            for p, r in zip(gen, outs):
                w = p.spectrum
                ok = ok and r.info == 0 and r.M == int(((w >= p.emin) & (w <= p.emax)).sum())
            res[label] = {"eigenpairs_per_s": sum(r.M for r in outs) / dt, "ms": dt * 1e3, "workers": nw,
                          "all_counts_exact": bool(ok)}
        res["tuning"] = {"workers": entry["workers"], "width": entry["width"], "tune_s": tune_s,
                         "sample": tune_sample}
        res["eigenpairs_per_s"] = res["tuned"]["eigenpairs_per_s"]
        out[name] = res
    try:
        out["tuning_file"] = os.path.relpath(autotune.save(autotune.merge(entries)), ROOT)
    except OSError:
        out["tuning_file"] = None
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of
# the sliced GEMM kernel on the solve shape 4096 x 300 x 32, 8 nodes (the
# capture in profiles/), or None when the kernel changed since it was taken
SLICED_TRAFFIC_BYTES = None
# ctf32_kernel on the early trailing-update shape 4096 x 4096 x 32, 2 nodes
# (profiles/ctf32_kernel_lu-update-shape_4096x4096x32x2.md): DRAM read +
# write and the algorithmic bytes of that launch (C read + written, TF32
# planes of A and B)
CTF32_CAPTURE = {"dram_bytes": 284.2e6 + 208.1e6, "algorithmic_bytes": 549.5e6,
                 "shape": "4096 x 4096 x 32, 2 nodes"}


def lu_update_bytes(n, ne, nb=32, entry_bytes=8):
    """Algorithmic bytes of one factorisation's trailing updates: every
    update reads and writes its C block once ((n - k - w)^2 entries per
    node, each entry_bytes wide: complex FP32 = 8)."""
    tot = 0
    for k in range(0, n, nb):
        r = n - k - min(nb, n - k)
        tot += r * r
    return 2.0 * entry_bytes * ne * tot


def roofline(prof, tc, path, n=None, ne=None):
    """Dominant kernel by device time.  The FP64 factor / solve / projection
    products run as sliced tensor-core GEMMs (zgemm_sliced_kernel for k <= 32,
    7 digits; gemm_sliced_k_kernel for any k, 8 digits): their work is the
    digit-pair bf16 products they issue (S(S+1)/2 products of each padded
    128 x 32 x 64 tile), rated against the measured bf16 tensor peak; the
    FP64 flops they deliver are reported beside as "useful".  The other
    kernels run on the FP64 ALUs (nominal 1.25 TFLOP/s)."""
    tn, tms, tfl, ttf = tc
    if path == "mixed" and n and prof.get("lu_update_gemm", (0, 0.0, 0.0))[1] > 0:
        # the FP32 factorisation's trailing updates (3xTF32 on the tensor
        # cores, C staged through shared memory): bound by C's traffic
        ln, lms, _ = prof["lu_update_gemm"]
        byt = lu_update_bytes(n, ne)
        pk = measured_peaks().get("hbm_gbs", 6800.0) * 1e9
        ach = byt / (lms / 1e3)
        cap = CTF32_CAPTURE
        ratio = cap["dram_bytes"] / cap["algorithmic_bytes"]
        return {"kernel": "ctf32_kernel (FP32 LU trailing updates, C read and written once per step)",
                "bound": "hbm", "achieved": ach / 1e9, "peak": pk / 1e9, "unit": "GB/s", "frac": ach / pk,
                "traffic": byt * ratio,
                "traffic_source": (f"per step: algorithmic bytes x the DRAM/algorithmic ratio {ratio:.3f} of one "
                                   f"ncu capture ({cap['shape']}: {cap['dram_bytes'] / 1e6:.1f} MB DRAM for "
                                   f"{cap['algorithmic_bytes'] / 1e6:.1f} MB algorithmic)"),
                "algorithmic_bytes_per_step": byt, "launches": ln,
                "avg_launch_ms": lms / max(ln, 1), "ms_per_step": lms,
                "peak_source": "measured HBM copy (MEASURED_PEAKS.json), of measured"}
    other = {k: v for k, v in prof.items() if k not in ("lu_update_gemm", "solve_gemm")}
    oname, (onl, oms, ofl) = max(other.items(), key=lambda kv: kv[1][1])
    if tms > 0 and tms >= oms:
        pk = measured_peaks().get("bf16_tflops_sustained", 1721.2) * 1e12
        ach = ttf / (tms / 1e3)
        return {"kernel": "sliced tensor-core GEMMs (zgemm_sliced_kernel, gemm_sliced_k_kernel)",
                "bound": "tensor", "achieved": ach / 1e12, "peak": pk / 1e12, "unit": "TFLOP/s",
                "frac": ach / pk, "traffic": SLICED_TRAFFIC_BYTES,
                "useful_fp64_tflops": tfl / (tms / 1e3) / 1e12, "launches": tn,
                "avg_launch_ms": tms / max(tn, 1), "ms_per_step": tms,
                "peak_source": "measured bf16 sustained (MEASURED_PEAKS.json), of measured"}
    if oms <= 0:
        return None
    useful = ofl / (oms / 1e3)
    return {"kernel": oname, "bound": "alu", "achieved": useful / 1e12, "peak": FP64_PEAK_NOMINAL / 1e12,
            "unit": "TFLOP/s", "frac": useful / FP64_PEAK_NOMINAL, "traffic": None, "launches": onl,
            "avg_launch_ms": oms / max(onl, 1), "ms_per_step": oms,
            "peak_source": "nominal FP64 1.25 TFLOP/s (GB300 table), of fallback nominal"}


# ------------------------------------------------------------- CPU oracle --
GOLD = os.path.join(ROOT, "tests", "golden", "real_generalized_n4096.json")
SAMPLE_K = 2048


def nproc():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_contours():
    """Contours the oracle runs on this workload: its loop count + 1 (every
    oracle loop forms, factors and solves all Ne shifted systems again), from
    its full run recorded in the golden file."""
    with open(GOLD) as f:
        gold = json.load(f)
    return gold["loop"] + 1, gold


def cpu_baseline(p, M):
    """The oracle (plain FP64 C, OpenMP over the contour nodes) timed on this
    host's cores on a bounded sample of the workload:
      all cores: one full contour of the n=4096 problem (oracle FEAST with
        fpm(14)=1: RHS = B Y, form, factor and solve all Ne = 8 shifted
        systems, the node-ordered sum), x the oracle's contour count;
      one core: one node's full-size form + factor + M0-column solve,
        x Ne x the contour count.
    Both leave out the oracle's Rayleigh-Ritz steps (about 5 % of a
    contour's flops), so both are upper bounds of the oracle's rate."""
    import oracle

    contours, gold = oracle_contours()
    nt = nproc()
    f = p.apply_fpm(oracle.feastinit())
    f[13] = 1
    t0 = time.perf_counter()
    r = oracle.feast(p.A, p.B, p.emin, p.emax, p.m0, fpm=f, nthreads=nt)
    t_c = time.perf_counter() - t0
    assert r["info"] == 4, r["info"]
    z, _ = oracle.contour(p.emin, p.emax, 8)
    Y = np.asfortranarray(np.random.default_rng(1).uniform(-1, 1, (p.n, p.m0)))
    t0 = time.perf_counter()
    lu, ipiv, _ = oracle.zgetrf(z[0] * p.B - p.A)
    oracle.zgetrs(lu, ipiv, p.B @ Y)
    t_node = time.perf_counter() - t0
    return {"value": M / (contours * t_c), "unit": "eigenpairs/s", "cores": nt, "kind": "oracle",
            "sample": f"one oracle contour of the full n={p.n} problem (8 nodes formed, factored and solved, "
                      f"OpenMP over nodes, {nt} threads): {t_c:.1f} s, x {contours} contours (the oracle's loop "
                      f"count on this workload); Rayleigh-Ritz steps not timed (upper bound)",
            "one_core": {"value": M / (contours * 8 * t_node), "unit": "eigenpairs/s", "cores": 1,
                         "sample": f"one node's form + zgetrf + {p.m0}-column zgetrs at n={p.n}: {t_node:.1f} s, "
                                   f"x 8 nodes x {contours} contours (upper bound)"},
            "full_run_on_record": {"seconds": gold.get("oracle_seconds"), "threads": gold.get("threads"),
                                   "note": "the oracle's complete FEAST on this workload when the golden file "
                                           "was written (x86 host): M, loops and eigenvalues are the parity "
                                           "test's expected values"}}


def oracle_node_sample(p, Y):
    """One oracle node on the leading SAMPLE_K block (one core): form +
    zgetrf, then the M0-column zgetrs; returns (t_factor, t_solve)."""
    import oracle

    z, _ = oracle.contour(p.emin, p.emax, 8)
    k = SAMPLE_K
    t0 = time.perf_counter()
    lu, ipiv, _ = oracle.zgetrf(z[0] * p.B[:k, :k] - p.A[:k, :k])
    t1 = time.perf_counter()
    oracle.zgetrs(lu, ipiv, Y)
    return t1 - t0, time.perf_counter() - t1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p = workload()
    M = 200
    contours, _ = oracle_contours()
    Y = np.asfortranarray(np.random.default_rng(1).uniform(-1, 1, (SAMPLE_K, p.m0)))
    for _ in range(args.warmup):
        oracle_node_sample(p, Y)
    ts = [oracle_node_sample(p, Y) for _ in range(args.steps)]
    tf = float(np.mean([t[0] for t in ts]))
    tsol = float(np.mean([t[1] for t in ts]))
    r = p.n / SAMPLE_K
    t_node = tf * r ** 3 + tsol * r ** 2       # factor ~ n^3, M0-column solve ~ n^2
    value = M / (contours * 8 * t_node)
    sample = (f"per step: one oracle node (form + zgetrf + {p.m0}-column zgetrs) on the leading "
              f"{SAMPLE_K}^2 block, one core; scaled to n={p.n} (factor x {r ** 3:.0f}, solve x {r ** 2:.0f}) "
              f"and x 8 nodes x {contours} contours (upper bound: Rayleigh-Ritz not timed)")
    line = {
        "impl": "reference", "metric": METRIC,
        "value": value, "unit": "eigenpairs/s", "n_gpus": int(os.environ.get("WORLD_SIZE", args.gpus)),
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * (tf + tsol), "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(p), "M": M, "parallelism": "oracle on one host core (no GPU)"},
        "cpu_baseline": {"value": value, "unit": "eigenpairs/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gbf(a)
