"""Host side of the measure-sharded solver, on the CPU with gloo ranks.

* ``partition_measures``: contiguous, complete, non-empty ranges with about
  equal kept-column counts.
* ``torch_allreduce``: the callback the library calls, driven here through
  its C function pointer on host buffers over 2 and 4 gloo ranks.
* The exchange protocol of the sharded Step 1 (Prop. 2, eq. pr), run on the
  FP64 oracle's per-measure Step 2 (``column_step``): each rank forms its
  partial sum of a_m p^(m) as fixed-point integers, the callback sums them
  over the ranks, and the resulting p, and every shift and plan after it,
  are bit for bit those of a single rank holding every measure, for 20
  iterations and for any partition (balanced problems, t^k = 1).  With
  gamma finite, t^k takes its distance from a second, FP64 exchange whose
  association depends on the partition, so the iterates agree to rounding
  (1e-12 relative) rather than bit for bit.
"""
import ctypes as C
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2309_05315_gb300 import _capi  # noqa: E402
from paper_2309_05315_gb300.shard import partition_measures  # noqa: E402


def test_partition_measures():
    rng = np.random.default_rng(3)
    for _ in range(50):
        M = int(rng.integers(1, 40))
        S = rng.integers(1, 300, size=M)
        for world in range(1, M + 1):
            r = partition_measures(S, world)
            assert len(r) == world and r[0][0] == 0 and r[-1][1] == M
            assert all(a < b for a, b in r)
            assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
            if 4 * world > M:   # few measures per rank: the one-measure rule may force cuts
                continue
            share = S.sum() / world
            cum = np.cumsum(S)
            for k, (a, b) in enumerate(r[:-1]):
                # each cut is within one measure of its target share
                assert abs(cum[b - 1] - share * (k + 1)) <= S.max() + 1e-9
    with pytest.raises(ValueError):
        partition_measures([1, 2], 3)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spawn(fn, world, *args):
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=fn, args=(r, world, port, q) + args) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out, key=lambda x: x[0])


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _callback_rank(rank, world, port, q):
    from paper_2309_05315_gb300.shard import torch_allreduce
    dist = _init(rank, world, port)
    fn = torch_allreduce(device="cpu")
    ptr = C.cast(fn, C.c_void_p).value
    call = _capi.ALLREDUCE_FN(ptr)
    ib = np.array([rank + 1, -7 * rank, 2 ** 61 + rank], dtype=np.int64)
    fb = np.array([0.5 * rank, -1.25, 1e300], dtype=np.float64)
    r1 = call(ib.ctypes.data, 3, _capi.SUM_I64, None, None)
    r2 = call(fb.ctypes.data, 2, _capi.SUM_F64, None, None)   # only the first two
    q.put((rank, r1, r2, ib.tolist(), fb.tolist()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_allreduce_callback_over_gloo(world):
    out = _spawn(_callback_rank, world)
    n = world
    want_i = [n * (n + 1) // 2, -7 * n * (n - 1) // 2, n * 2 ** 61 + n * (n - 1) // 2]
    want_i = [((v + 2 ** 63) % 2 ** 64) - 2 ** 63 for v in want_i]    # int64 wraparound
    for rank, r1, r2, ib, fb in out:
        assert r1 == 0 and r2 == 0
        assert ib == want_i
        assert fb[:2] == [0.5 * n * (n - 1) / 2, -1.25 * n] and fb[2] == 1e300


# ---------------------------------------------------------------- protocol

FX_E = 50                      # fixed point F = 2^50 for p^(m) (masses <= 1)
A_SHIFT = 62                   # a_m held as round(a_m 2^62)


def _protocol_run(problem, ranges, rank, exchange, iters, gamma):
    """Algorithm 1 on this rank's measures with the sharded Step 1."""
    from oracle.mam_oracle import column_step, prepare
    prep = prepare(problem)
    m0, m1 = ranges[rank]
    S, R = prep.S, prep.R
    a = (1.0 / S) / (1.0 / S).sum()
    aq = [int(round(float(v) * 2 ** A_SHIFT)) for v in a]
    theta = {m: np.repeat((prep.q[m] / R)[:, None], R, axis=1) for m in range(m0, m1)}
    traj = []
    for _ in range(iters):
        pm_fx = {m: np.rint(theta[m].sum(axis=0) * 2.0 ** FX_E).astype(np.int64)
                 for m in range(m0, m1)}
        part = np.zeros(R, dtype=np.int64)
        for m in range(m0, m1):
            part += np.array([(int(v) * aq[m]) >> A_SHIFT for v in pm_fx[m]], dtype=np.int64)
        exchange(part, _capi.SUM_I64)               # sum of a_m p^(m) over all ranks
        p = part.astype(np.float64) / 2.0 ** FX_E
        dist2 = np.array([sum(float(np.dot(p - pm_fx[m] / 2.0 ** FX_E,
                                           p - pm_fx[m] / 2.0 ** FX_E)) / S[m]
                              for m in range(m0, m1))])
        exchange(dist2, _capi.SUM_F64)
        D = math.sqrt(dist2[0])
        t = 1.0 if (math.isinf(gamma) or problem.rho * D <= gamma) else gamma / (problem.rho * D)
        for m in range(m0, m1):
            d = t * (p - pm_fx[m] / 2.0 ** FX_E) / S[m]
            theta[m] = column_step(theta[m], d, prep.c[m], prep.q[m], problem.rho)[0]
        traj.append(part.copy())
    return traj, {m: theta[m] for m in theta}


def _protocol_rank(rank, world, port, q, gamma):
    from paper_2309_05315_gb300.shard import torch_allreduce
    from workloads import tiny_problem
    dist = _init(rank, world, port)
    fn = torch_allreduce(device="cpu")

    def exchange(arr, dtype):
        assert fn(arr.ctypes.data, arr.size, dtype, None, None) == 0

    masses = None if math.isinf(gamma) else [0.7, 1.0, 1.3, 0.9, 1.2, 0.8]
    prob = tiny_problem(71, M=6, K=5, rho=6.0, masses=masses)
    S = [int((np.asarray(v) > 0).sum()) for v in prob.q]
    ranges = partition_measures(S, world)
    traj, theta = _protocol_run(prob, ranges, rank, exchange, 20, gamma)
    q.put((rank, [t.tolist() for t in traj], {m: v.tolist() for m, v in theta.items()}))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("gamma", [math.inf, 0.02])
def test_sharded_protocol_is_bitwise_the_single_rank_run(gamma):
    runs = {w: _spawn(_protocol_rank, w, gamma) for w in (1, 2, 4)}
    ref_traj = runs[1][0][1]
    ref_theta = runs[1][0][2]
    for w in (2, 4):
        for rank, traj, theta in runs[w]:
            if math.isinf(gamma):
                assert traj == ref_traj, (w, rank)           # p at every iteration, bitwise
                for m, v in theta.items():
                    assert v == ref_theta[m], (w, rank, m)   # the plans of its measures
            else:
                for x, y in zip(traj, ref_traj):
                    x, y = np.array(x, dtype=np.float64), np.array(y, dtype=np.float64)
                    assert np.abs(x - y).sum() <= 1e-12 * np.abs(y).sum()
                for m, v in theta.items():
                    np.testing.assert_allclose(v, ref_theta[m], rtol=0, atol=1e-12)
