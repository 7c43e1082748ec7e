"""Node sharding of one FEAST solve across processes (one GPU each): the
guide's second level of parallelism ("Using the FEAST-MPI version": the
contour nodes of one search interval are spread over the ranks and the
filtered subspace is summed over them once per iteration).

The library (``gbf_dsygv_dev_shard`` / ``gbf_zhegv_dev_shard`` in
include/gbfeast.h) factors and solves only the shard's own nodes and calls
back for the one exchange step per iteration, an all-gather of the node
solution blocks, and for a status agreement.  This module supplies those two
callbacks:

* ``DistExchange`` -- ``torch.distributed`` collectives (NCCL between GPUs,
  gloo on CPU): ``all_gather_into_tensor`` into the library's buffer, on the
  library's stream, and an ``all_reduce(MIN)`` of the status code.
* ``ThreadShards`` -- several logical shards inside one process (threads,
  one handle and stream each, all on one device), exchanging through
  device-to-device copies after a host barrier.  No kernel of one shard ever
  waits for another shard's kernels; the host orders them.

Argument marshalling only: every step of the solve runs in the library.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import (_check_colmajor, _ip, _ptr, _scalars, gbf_init, lib)

ALLGATHER_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t)
AGREE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_int))


class ShardSpec(C.Structure):
    """gbf_shard (include/gbfeast.h)."""
    _fields_ = [("rank", C.c_int), ("nranks", C.c_int), ("allgather", ALLGATHER_FN), ("agree", AGREE_FN),
                ("user", C.c_void_p)]


def shard_nodes(ne, rank, nranks):
    """(first node, node count, chunk) of shard `rank` (gbf_shard_nodes)."""
    first, count = C.c_int(), C.c_int()
    chunk = lib().gbf_shard_nodes(int(ne), int(rank), int(nranks), C.byref(first), C.byref(count))
    if chunk < 0:
        raise ValueError(f"gbf_shard_nodes: {chunk}")
    return first.value, count.value, chunk


class _DeviceBytes:
    """A raw device range as a uint8 CUDA array (zero copy, via the CUDA array
    interface), so torch collectives and copies can act on library buffers."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 2, "strides": None}


def device_bytes(ptr, nbytes, device=None):
    import torch

    if device is None:
        device = torch.device("cuda", torch.cuda.current_device())
    return torch.as_tensor(_DeviceBytes(ptr, nbytes), device=device)


class _Callbacks:
    """Keeps the ctypes callback objects alive for the life of a ShardSpec."""

    def __init__(self, rank, nranks, allgather, agree):
        def ag(_user, stream, dbuf, chunk_bytes):
            try:
                allgather(stream, dbuf, chunk_bytes)
                return 0
            except Exception as e:  # noqa: BLE001 - reported to the library as a failed callback
                self.error = e
                return 1

        def ar(_user, code):
            try:
                code[0] = int(agree(int(code[0])))
                return 0
            except Exception as e:  # noqa: BLE001
                self.error = e
                return 1

        self.error = None
        self._ag = ALLGATHER_FN(ag)
        self._ar = AGREE_FN(ar)
        self.spec = ShardSpec(rank, nranks, self._ag, self._ar, None)


class DistExchange:
    """Exchange step over a torch.distributed process group."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.nranks = dist.get_world_size(group)

    def allgather_(self, buf, chunk_elems):
        """In place: chunk `rank` of the flat tensor `buf` (nranks chunks of
        chunk_elems) is gathered into every other rank's buffer."""
        # the own chunk is sent from a copy: the collective then never reads
        # and writes the same range
        own = buf[self.rank * chunk_elems:(self.rank + 1) * chunk_elems].clone()
        self.dist.all_gather_into_tensor(buf[:self.nranks * chunk_elems], own, group=self.group)

    def agree(self, code, device=None):
        import torch

        t = torch.tensor([int(code)], dtype=torch.int64, device=device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN, group=self.group)
        return int(t.item())

    def callbacks(self):
        import torch

        dev = torch.device("cuda", torch.cuda.current_device())

        def allgather(stream, dbuf, chunk_bytes):
            buf = device_bytes(dbuf, chunk_bytes * self.nranks, dev)
            with torch.cuda.stream(torch.cuda.ExternalStream(stream or 0, device=dev)):
                self.allgather_(buf, chunk_bytes)

        return _Callbacks(self.rank, self.nranks, allgather, lambda c: self.agree(c, dev))


class ThreadShards:
    """`nranks` logical shards in one process on one device, one thread each.
    The exchange is host-ordered: each shard finishes its own stream, meets
    the others at a barrier, copies their chunks into its buffer on its own
    stream, finishes it, and meets them again before any shard goes on."""

    def __init__(self, nranks):
        self.nranks = nranks
        self.bar = threading.Barrier(nranks)
        self.bufs = [None] * nranks
        self.codes = [0] * nranks

    def callbacks(self, rank):
        import torch

        dev = torch.device("cuda", torch.cuda.current_device())

        def allgather(stream, dbuf, chunk_bytes):
            s = torch.cuda.ExternalStream(stream or 0, device=dev)
            s.synchronize()
            self.bufs[rank] = device_bytes(dbuf, chunk_bytes * self.nranks, dev)
            self.bar.wait()
            with torch.cuda.stream(s):
                mine = self.bufs[rank]
                for g in range(self.nranks):
                    if g != rank:
                        sl = slice(g * chunk_bytes, (g + 1) * chunk_bytes)
                        mine[sl].copy_(self.bufs[g][sl])
            s.synchronize()
            self.bar.wait()

        def agree(code):
            self.codes[rank] = code
            self.bar.wait()
            out = min(self.codes)
            self.bar.wait()
            return out

        return _Callbacks(rank, self.nranks, allgather, agree)


def feast_dev_shard(A, B, emin, emax, m0, callbacks, fpm=None, E=None, X=None, res=None, uplo="F", handle=None,
                    stream=None, Zne=None, Wne=None):
    """gbf_dsygv_dev_shard / gbf_zhegv_dev_shard on torch CUDA tensors (as
    feast_dev); `callbacks` from DistExchange.callbacks() or
    ThreadShards.callbacks(rank).  Returns the feast_dev dict."""
    import torch

    if fpm is None:
        fpm = gbf_init()
    fpm = np.ascontiguousarray(fpm, dtype=np.int32).copy()
    herm = A.is_complex()
    n = A.shape[0]
    lda = _check_colmajor(A, n)
    ldb = _check_colmajor(B, n) if B is not None else n
    dev = A.device
    if E is None:
        E = torch.zeros(m0, dtype=torch.float64, device=dev)
    if res is None:
        res = torch.zeros(m0, dtype=torch.float64, device=dev)
    if X is None:
        X = torch.zeros((m0, n), dtype=A.dtype, device=dev).t()
    eps, loop, M, info = _scalars()
    M0 = C.c_int(int(m0))
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    sp = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    zp = wp = None
    if Zne is not None:
        zne = np.ascontiguousarray(Zne, dtype=np.complex128)
        wne = np.ascontiguousarray(Wne, dtype=np.complex128)
        zp, wp = _ptr(zne), _ptr(wne)
    fn = lib().gbf_zhegv_dev_shard if herm else lib().gbf_dsygv_dev_shard
    fn(handle.h if handle is not None else None, sp, C.c_char(uplo.encode()), n, _ptr(A), lda, _ptr(B), ldb,
       _ip(fpm), C.byref(eps), C.byref(loop), float(emin), float(emax), C.byref(M0), _ptr(E), _ptr(X),
       C.byref(M), _ptr(res), C.byref(info), zp, wp, C.c_void_p(C.addressof(callbacks.spec)))
    if callbacks.error is not None:
        raise RuntimeError(f"shard callback failed: {callbacks.error!r}")
    return dict(E=E, X=X, res=res, M=M.value, loop=loop.value, epsout=eps.value, m0=M0.value, info=info.value)
