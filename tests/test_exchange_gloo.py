"""The segment layout of Sec. III B over several ranks, on CPU (gloo, 127.0.0.1).

One GPU runs all segments of a chain, so the library never exchanges tensors.
With one GPU per group of segments, the ranks would run the stages in
lockstep and exchange, at every boundary update between two ranks, the
tensors of tdvp_exchange_plan (the right rank's Psi_{e+1} and gamma_{e+1}
before it, the left rank's Psi_{e+1}, V_e and beta_{e+1} after it). This test
checks that plan: two or three CPU ranks (the middle one exchanging with both
neighbours) each run the oracle's local operations for their own segments
only, send and receive exactly the planned tensors, and must end with the
one-rank oracle's state bit for bit -- for the two-site sweep and the
segmented one-site sweep.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

N = 14
SEG = [3, 4, 4, 3]
RANK_OF_SEG = [0, 0, 1, 1]
# the segment layouts run: two ranks with one boundary between them, and three
# ranks where the middle one exchanges with both neighbours
LAYOUTS = {"two_ranks": ([3, 4, 4, 3], [0, 0, 1, 1]), "three_ranks": ([3, 3, 3, 3, 2], [0, 1, 1, 2, 2])}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _setup(seg):
    import tdvp_inputs as I
    from oracle import models
    from oracle import mps as M
    from oracle import tdvp as T
    x, lam = models.fit_power_law(2.0, 3, N - 1)
    W = models.build_mpo_site(models.ISING, 1.0, 0.7, x, lam)
    mps = M.canonicalize(I.random_mps_tensors(N, 6, seed=21), 8, 1e-14)
    p = T.Params(dt=0.04, chi_max=8, krylov_max=12, krylov_tol=0.0, seg_len=seg)
    return W, mps, p


def _send(dist, torch, a, dst):
    a = np.ascontiguousarray(a)
    is_c = np.iscomplexobj(a)
    head = torch.tensor([a.ndim, int(is_c)] + list(a.shape) + [0] * (4 - a.ndim), dtype=torch.int64)
    dist.send(head, dst)
    data = a.view(np.float64).reshape(-1) if is_c else a.astype(np.float64).reshape(-1)
    dist.send(torch.from_numpy(data.copy()), dst)


def _recv(dist, torch, src):
    head = torch.zeros(6, dtype=torch.int64)
    dist.recv(head, src)
    nd, is_c = int(head[0]), int(head[1])
    shape = [int(v) for v in head[2:2 + nd]]
    n = int(np.prod(shape)) * (2 if is_c else 1)
    buf = torch.zeros(n, dtype=torch.float64)
    dist.recv(buf, src)
    a = buf.numpy()
    return (a.view(np.complex128) if is_c else a).reshape(shape).copy()


def _rank_main(rank, world, port, scheme, steps, seg, rank_of_seg, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from oracle import tdvp as T
    from oracle import tdvp1 as T1
    from paper_1912_06127_gb300 import tdvp
    dist.init_process_group("gloo", rank=rank, world_size=world)
    W, mps, p = _setup(seg)
    eng = T.Engine(mps, W)
    bounds = T.segment_bounds(N, seg)
    mine = {k for k in range(len(seg)) if rank_of_seg[k] == rank}
    owner = {j: rank_of_seg[k] for k, (s, e) in enumerate(bounds) for j in range(s, e + 1)}
    halves = ([T.build_half(N, seg, h, p.merge_turning) for h in (1, 2)] if scheme == 2 else
              [T1.build_half1(N, seg, h, p.merge_turning) for h in (1, 2)])
    plans = [tdvp.exchange_plan(N, seg, rank_of_seg, scheme, p.merge_turning, h) for h in (1, 2)]
    store = {0: eng.mps.Psi, 1: eng.mps.V, 2: eng.beta, 3: eng.gamma}
    n_sent = 0

    def exchange(plan, stage, after):
        nonlocal n_sent
        for st, aft, src, dst, kind, j in plan:
            if st != stage or aft != after:
                continue
            if rank == src:
                _send(dist, torch, store[kind][j], dst)
                n_sent += 1
            elif rank == dst:
                store[kind][j] = _recv(dist, torch, src)

    for _ in range(steps):
        if scheme == 1:   # step1_segmented's rebuilds at the start of a step, by the owning ranks
            if owner[0] == rank and T.sweeps_right_first(0, len(seg)):
                eng.gamma[0] = T.env_right(eng.gamma[1], eng._B(0), W)
            if owner[N - 1] == rank and not T.sweeps_right_first(len(seg) - 1, len(seg)):
                eng.beta[N - 1] = T.env_left(eng.beta[N - 2], eng._A(N - 2), W)
        for ops, plan in zip(halves, plans):
            for stage in range(max(o.stage for o in ops) + 1):
                exchange(plan, stage, 0)
                for op in ops:
                    if op.stage == stage and op.seg in mine:
                        if scheme == 2:
                            eng.run_op(op, p)
                        else:
                            T1.run_op1(eng, op, p)
                exchange(plan, stage, 1)
    # gather: every site tensor and the bond to its right from the owning rank
    if rank != 0:
        for j in range(N):
            if owner[j] == rank:
                _send(dist, torch, eng.mps.Psi[j], 0)
                if j < N - 1:
                    _send(dist, torch, eng.mps.V[j], 0)
        out.put((rank, None, None, n_sent))
    else:
        psi, v = [None] * N, [None] * (N - 1)
        for j in range(N):
            if owner[j] == 0:
                psi[j] = eng.mps.Psi[j]
                if j < N - 1:
                    v[j] = eng.mps.V[j]
            else:
                psi[j] = _recv(dist, torch, owner[j])
                if j < N - 1:
                    v[j] = _recv(dist, torch, owner[j])
        out.put((rank, psi, v, n_sent))
    dist.destroy_process_group()


@pytest.mark.parametrize("layout", sorted(LAYOUTS))
@pytest.mark.parametrize("scheme", [2, 1], ids=["two_site", "one_site"])
def test_ranks_reproduce_one_rank(scheme, layout):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__.build()
    from oracle import tdvp as T
    from oracle import tdvp1 as T1
    steps = 2
    seg, rank_of_seg = LAYOUTS[layout]
    world = max(rank_of_seg) + 1
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, scheme, steps, seg, rank_of_seg, q))
             for r in range(world)]
    for pr in procs:
        pr.start()
    res = {}
    for _ in range(world):
        r, psi, v, n_sent = q.get(timeout=300)
        res[r] = (psi, v, n_sent)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    # one rank, the oracle's own sweep
    W, mps, p = _setup(seg)
    eng = T.Engine(mps, W)
    if scheme == 2:
        eng.step(p, steps)
    else:
        T1.step1_segmented(eng, p, steps)
    psi, v, _ = res[0]
    for j in range(N):
        assert np.array_equal(psi[j], eng.mps.Psi[j]), j
    for j in range(N - 1):
        assert np.array_equal(v[j], eng.mps.V[j]), j
    # exactly the planned messages were sent: 2 before and 3 after each update
    # of a boundary between two ranks
    from paper_1912_06127_gb300 import tdvp
    planned = sum(len(tdvp.exchange_plan(N, seg, rank_of_seg, scheme, p.merge_turning, h)) for h in (1, 2))
    assert planned % 5 == 0 and sum(r[2] for r in res.values()) == steps * planned
    if layout == "two_ranks":
        # the one boundary between the ranks (after segment 1) is updated in both halves
        assert planned == 2 * 5


def test_exchange_plan_host_rules():
    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_06127_gb300 import tdvp
    # all segments on one rank: nothing to exchange
    assert len(tdvp.exchange_plan(N, SEG, [0, 0, 0, 0], 2, 1, 1)) == 0
    # one rank per segment: every boundary update is between ranks
    plan = tdvp.exchange_plan(N, SEG, [0, 1, 2, 3], 2, 1, 1)
    assert len(plan) == 5 * (len(SEG) - 1)
    for st, aft, src, dst, kind, j in plan:
        assert abs(src - dst) == 1 and kind in ((0, 3) if aft == 0 else (0, 1, 2))
    with pytest.raises(tdvp.TdvpError):
        tdvp.exchange_plan(N, SEG, [1, 0, 0, 0], 2, 1, 1)
