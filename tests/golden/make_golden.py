"""Write stored expected values for the full-size parity tests.

Calls only the CPU oracle (oracle/) on inputs from the seeded generator
(paper_1203_4031_gb300.workloads); nothing here touches the CUDA path.

  python tests/golden/make_golden.py real-generalized-4096
      -> tests/golden/real_generalized_n4096.json
         oracle FEAST eigenvalues/residuals of the n=4096 real symmetric
         generalized workload (M0=300, Ne=8, residual criterion 1e-10), plus
         the Sylvester inertia count of its interval.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1203_4031_gb300 import workloads as W  # noqa: E402


def real_generalized_4096():
    p = W.dense_real_generalized()
    fpm = p.apply_fpm(oracle.feastinit())
    t0 = time.time()
    r = oracle.feast(p.A, p.B, p.emin, p.emax, p.m0, fpm=fpm, hermitian=False)
    t1 = time.time()
    count = oracle.eigcount(p.A, p.B, p.emin, p.emax)
    t2 = time.time()
    M = r["M"]
    out = dict(
        workload=p.name, note=p.note, n=p.n, emin=p.emin, emax=p.emax, m0=p.m0, fpm=p.fpm,
        info=r["info"], M=M, loop=r["loop"], epsout=r["epsout"], m0_out=r["m0"],
        E=[float(v) for v in r["E"][:M]], res=[float(v) for v in r["res"][:M]],
        sylvester_count=count, oracle_seconds=t1 - t0, inertia_seconds=t2 - t1,
        threads=int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1)),
        generator="oracle.feast + oracle.eigcount (tests/golden/make_golden.py)",
    )
    with open(os.path.join(HERE, "real_generalized_n4096.json"), "w") as f:
        json.dump(out, f, indent=1)
    return out


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "real-generalized-4096"
    if which == "real-generalized-4096":
        o = real_generalized_4096()
        print({k: o[k] for k in ("info", "M", "loop", "sylvester_count", "oracle_seconds", "inertia_seconds")})
    else:
        raise SystemExit(f"unknown workload {which}")
