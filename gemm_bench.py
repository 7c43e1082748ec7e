"""Times one sliced tensor-core GEMM shape through the C ABI (the kernels the
FP64 factorisation, solves and projections run on), for profiling a single
kernel in isolation:

  python gemm_bench.py --kind k32 --m 4096 --n 300 --k 32 --batch 8
  python gemm_bench.py --kind anyk --cplx 1 --m 2048 --n 300 --k 2048
  python gemm_bench.py --kind tf32 --m 4096 --n 4096 --k 32 --batch 2
  python gemm_bench.py --kind lu --m 4096 --batch 8 --prec 1
  python gemm_bench.py --kind gen --m 4096 --cplx 0 --reps 1

k32: gbf_zgemm_sliced (k <= 32, 7 digits, complex FP64), C -= A B.
tf32: gbf_zgemm_sliced with S = 1 (k <= 32, complex FP32, 3xTF32 products),
C -= A B: the engine of the FP32 factorisation's trailing updates.
anyk: gbf_gemm_sliced (any k, 8 digits, real or complex FP64), C -= op(A) B with
op(A) = A^T read from an (m x k)-transposed store, as the projections use it.
lu: gbf_factor_dev, the blocked LU of `batch` shifted systems z_e I - A of one
m x m complex Hermitian A (panels, swaps, trailing updates), FP64 factors
(--prec 0) or FP32 (--prec 1).
gen: one non-Hermitian FEAST solve (gbf_dgegv_dev / gbf_zgegv_dev) of the
seeded n = m pencil with a known spectrum (real generalized with --cplx 0,
complex standard with --cplx 1), 40 eigenvalues inside, M0 = 64, 16 nodes.
Prints the time per call (CUDA events, after warm-up) and the useful FP64
rate; inputs are seeded normal values resident on the device."""
import argparse
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from paper_1203_4031_gb300 import _ptr, _stream_ptr, last_error, lib  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--kind", choices=["k32", "anyk", "tf32", "lu", "gen"], default="k32")
    ap.add_argument("--prec", type=int, default=0)
    ap.add_argument("--cplx", type=int, default=1)
    ap.add_argument("--m", type=int, default=4096)
    ap.add_argument("--n", type=int, default=300)
    ap.add_argument("--k", type=int, default=32)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    a = ap.parse_args(argv)
    L = lib()
    g = torch.Generator(device="cuda").manual_seed(1)
    if a.kind == "lu":
        return factor_bench(a, g)
    if a.kind == "gen":
        return gen_bench(a)
    cplx = 1 if a.kind in ("k32", "tf32") else a.cplx
    dt = torch.complex128 if cplx else torch.float64
    m, n, k, bt = a.m, a.n, a.k, a.batch

    def rnd(*shape):
        x = torch.randn(shape, device="cuda", dtype=torch.float64, generator=g)
        if cplx:
            x = torch.complex(x, torch.randn(shape, device="cuda", dtype=torch.float64, generator=g))
        return x

    st = torch.cuda.current_stream()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = rnd(bt, n, m)
    if a.kind == "tf32":
        A, B = rnd(bt, k, m).to(torch.complex64), rnd(bt, n, k).to(torch.complex64)
        C = C.to(torch.complex64)
        work = torch.empty(L.gbf_zgemm_sliced_work(m, n, bt, 1), dtype=torch.uint8, device="cuda")

        def run():
            return L.gbf_zgemm_sliced(_stream_ptr(st), 1, 1, b"N", b"N", m, n, k, -1.0, _ptr(A), m, m * k, _ptr(B),
                                      k, k * n, 1, _ptr(C), m, m * n, bt, _ptr(work), work.numel(), _ptr(err))
    elif a.kind == "k32":
        A, B = rnd(bt, k, m), rnd(bt, n, k)   # column-major m x k and k x n
        work = torch.empty(L.gbf_zgemm_sliced_work(m, n, bt, 7), dtype=torch.uint8, device="cuda")

        def run():
            return L.gbf_zgemm_sliced(_stream_ptr(st), 0, 7, b"N", b"N", m, n, k, -1.0, _ptr(A), m, m * k, _ptr(B),
                                      k, k * n, 1, _ptr(C), m, m * n, bt, _ptr(work), work.numel(), _ptr(err))
    else:
        A, B = rnd(bt, m, k), rnd(bt, n, k)   # column-major k x m (op T) and k x n
        work = torch.empty(L.gbf_gemm_sliced_work(cplx, m, n, k, bt), dtype=torch.uint8, device="cuda")

        def run():
            return L.gbf_gemm_sliced(_stream_ptr(st), cplx, b"T", b"N", m, n, k, -1.0, _ptr(A), k, m * k, _ptr(B),
                                     k, k * n, 1, _ptr(C), m, m * n, bt, _ptr(work), work.numel(), _ptr(err))
    for _ in range(a.warmup):
        if run() != 0:
            raise RuntimeError(last_error())
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(a.reps):
        run()
    e1.record(st)
    torch.cuda.synchronize()
    if err.item() != 0:
        raise RuntimeError(f"bounded wait timed out (code {err.item()})")
    ms = e0.elapsed_time(e1) / max(a.reps, 1)
    flops = (8.0 if cplx else 2.0) * m * n * k * bt
    what = "FP32" if a.kind == "tf32" else "FP64"
    cbytes = 2 * C.numel() * C.element_size()   # C read and written once
    print(f"{a.kind} cplx={cplx} m={m} n={n} k={k} batch={bt}: {ms * 1e3:.1f} us per call "
          f"(slicing included), {flops / ms / 1e9:.2f} useful {what} TFLOP/s, C traffic {cbytes / ms / 1e6:.0f} GB/s")


def factor_bench(a, g):
    import numpy as np

    import paper_1203_4031_gb300 as gb

    n, ne = a.m, a.batch
    X = torch.complex(torch.randn(n, n, device="cuda", dtype=torch.float64, generator=g),
                      torch.randn(n, n, device="cuda", dtype=torch.float64, generator=g))
    A = gb.fortran(0.5 * (X + X.conj().T))
    zne = np.exp(1j * np.pi * (np.arange(ne) + 0.5) / ne)   # nodes on the unit half-circle
    h = gb.Handle()
    for _ in range(a.warmup):
        if gb.gbf_factor_dev(h, A, None, zne, prec=a.prec) != 0:
            raise RuntimeError(last_error())
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(a.reps):
        gb.gbf_factor_dev(h, A, None, zne, prec=a.prec)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(a.reps, 1)
    flops = 8.0 / 3.0 * n ** 3 * ne
    print(f"lu prec={a.prec} n={n} nodes={ne}: {ms:.2f} ms per factorisation of all nodes, "
          f"{flops / ms / 1e9:.2f} useful TFLOP/s")
    h.close()


def gen_bench(a):
    import numpy as np

    import paper_1203_4031_gb300 as gb
    from paper_1203_4031_gb300 import workloads as W

    P = W.dense_nonsymmetric(a.m, count=40, m0=64, complex_=bool(a.cplx), generalized=not a.cplx)
    A = gb.fortran(torch.from_numpy(np.ascontiguousarray(P.A)).cuda())
    B = gb.fortran(torch.from_numpy(np.ascontiguousarray(P.B)).cuda()) if P.B is not None else None
    f = P.apply_fpm(gb.gbf_init())
    h = gb.Handle()
    for _ in range(a.warmup):
        gb.feast_gen_dev(A, B, P.emid, P.r, P.m0, f, handle=h)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(a.reps):
        r = gb.feast_gen_dev(A, B, P.emid, P.r, P.m0, f, handle=h)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(a.reps, 1)
    print(f"gen {P.name}: {ms:.1f} ms per solve, info {r['info']}, M {r['M']}, loops {r['loop']}")
    h.close()


if __name__ == "__main__":
    main()
