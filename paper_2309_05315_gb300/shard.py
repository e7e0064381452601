"""Measure-sharded MAM across ranks (argument marshalling and collectives).

``mam_create_sharded`` (include/mam.h) gives every rank a contiguous range of
the measures of one problem; the only exchange Algorithm 1 then needs is the
sum over ranks of the partial averages sum_m a_m p^(m) (eq. pr), which the
library hands to an all-reduce callback as 64-bit fixed-point integers (plus
four FP64 values when t^k or diagnostics are needed).  This module provides
the pieces around that call:

* ``partition_measures``: contiguous measure ranges of about equal
  sum_m S_m (a rank's plan entries are R times that sum);
* ``buffer_view``: a torch tensor over a raw buffer the library passes (a
  device pointer, or a host pointer for CPU process groups);
* ``torch_allreduce``: the callback for a torch.distributed process group
  (NCCL between GPUs; gloo on host buffers), enqueued on the library's
  stream;
* ``sharded``: creates this rank's ``Mam`` handle.

Nothing here computes any part of the method.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Sequence, Tuple

import numpy as np

from . import _capi

_TYPESTR = {_capi.SUM_I64: "<i8", _capi.SUM_F64: "<f8"}


def partition_measures(S_kept: Sequence[int], world: int) -> List[Tuple[int, int]]:
    """Ranges [m_begin, m_end) of consecutive measures, one per rank, with
    about equal kept-column counts sum_m S_m (every rank gets at least one
    measure, so world <= M).  The k-th cut is the prefix whose column count
    is nearest to k/world of the total, among the cuts that leave every rank
    at least one measure."""
    S = [int(s) for s in S_kept]
    M = len(S)
    if not 1 <= world <= M:
        raise ValueError(f"need 1 <= world ({world}) <= number of measures ({M})")
    cum = np.concatenate([[0], np.cumsum(S)]).astype(np.float64)
    total = cum[-1]
    cuts = [0]
    for k in range(1, world):
        lo, hi = cuts[-1] + 1, M - (world - k)      # admissible prefix lengths
        target = total * k / world
        c = lo + int(np.argmin(np.abs(cum[lo:hi + 1] - target)))
        cuts.append(c)
    cuts.append(M)
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


class _CudaBuf:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": (int(n),),
                                         "typestr": typestr, "version": 2}


def buffer_view(ptr: int, count: int, dtype: int, device: str = "cuda"):
    """A torch tensor aliasing `count` values of type `dtype` (SUM_I64 or
    SUM_F64) at `ptr`: device memory, or host memory for device="cpu"."""
    import torch
    if device == "cpu":
        ct = C.c_int64 if dtype == _capi.SUM_I64 else C.c_double
        arr = np.ctypeslib.as_array(C.cast(C.c_void_p(ptr), C.POINTER(ct)), shape=(int(count),))
        return torch.from_numpy(arr)
    return torch.as_tensor(_CudaBuf(ptr, count, _TYPESTR[dtype]), device=device)


def torch_allreduce(group=None, device: str = "cuda"):
    """An ``_capi.ALLREDUCE_FN`` that sums the buffer over ``group`` with
    torch.distributed, ordered on the library's stream (device buffers) or
    synchronously (host buffers, device="cpu").  Returns 0, or 1 after an
    exception (the library then reports MAM_ERR_COMM)."""
    import torch
    import torch.distributed as dist

    def cb(buf, count, dtype, stream, user):
        try:
            t = buffer_view(buf, count, dtype, device)
            if device == "cpu":
                dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
            else:
                with torch.cuda.stream(torch.cuda.ExternalStream(int(stream or 0))):
                    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
            return 0
        except Exception:
            return 1

    return _capi.ALLREDUCE_FN(cb)


def single_rank_allreduce():
    """The exchange of a world of one rank: the sum over one rank is the
    buffer itself, so the callback leaves it as it is."""
    return _capi.ALLREDUCE_FN(lambda buf, count, dtype, stream, user: 0)


def sharded(problem, rank: int, world: int, allreduce=None, ranges=None, **kw):
    """This rank's handle of a measure-sharded problem: measures
    ``ranges[rank]`` (default: ``partition_measures`` of the kept sizes) and
    the exchange ``allreduce`` (default: ``torch_allreduce()`` over the
    default process group, or nothing for a world of one).  Keyword
    arguments go to ``Mam``."""
    from .mam import Mam
    if ranges is None:
        S_kept = [int((np.asarray(q) > 0).sum()) for q in problem.q]
        ranges = partition_measures(S_kept, world)
    if allreduce is not None:
        fn = allreduce
    else:
        fn = single_rank_allreduce() if world == 1 else torch_allreduce()
    m0, m1 = ranges[rank]
    return Mam(problem, shard=(m0, m1, fn), **kw)
