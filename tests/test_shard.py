"""Sharding over processes with virtual patches (DISPATCH I, Sec. 3 C), on
CPU: the partition and the share lists, and the lock-step sweep / package
exchange of paper_1705_10774_gb300.shard with the oracle as each process's
engine -- in one process (several shares) and over torch.distributed with the
gloo backend, world size 2 -- against the one-process oracle run: the same
per-patch schedule and bit-identical states."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_1705_10774_gb300 import ics, shard
from oracle import Oracle

from shard_oracle import OracleEngine

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
T_END = 0.003


def lts_case():
    return ics.config_lts(patches=6, n=4, sigma_ln=1.0, hot_radius=0.15, hot_factor=100.0)


def kw_of(lay, f):
    return dict(gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)


def one_process(lay, f, state):
    o = Oracle(lay.n, lay.lo, time_mode=1, **kw_of(lay, f))
    o.set_state(*state)
    o.advance(t_end=T_END)
    return o


def per_patch(lay, arrays):
    n = np.asarray(lay.n, np.int64)
    nx, ny, nz = n[:, 0], n[:, 1], n[:, 2]
    per = [5 * nx * ny * nz, (nx + 1) * ny * nz, nx * (ny + 1) * nz, nx * ny * (nz + 1)]
    out = []
    for a, s in zip(arrays, per):
        off = np.concatenate([[0], np.cumsum(s)])
        out.append([a[off[i]:off[i + 1]] for i in range(len(s))])
    return out


def test_neighbours_match_the_oracle():
    for lay in (ics.cartesian(3, 5), ics.cartesian((2, 3, 1), (8, 6, 12)), ics.mixed_blocks(2, 24, sizes=(6, 8, 12),
                                                                                             probs=(1, 1, 1), seed=2)):
        nb = shard.neighbours(lay.n, lay.lo, lay.base_cells, 3)
        o = Oracle(lay.n, lay.lo, gamma=5 / 3, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)
        for i in range(lay.npatch):
            ref = np.sort(o.nbors(i))
            assert np.array_equal(nb[i], ref[ref != i]), i      # the oracle lists a patch that wraps onto itself


def test_partition_is_balanced_and_contiguous_along_the_curve():
    lay = ics.cartesian(8, 4)
    for nr in (2, 3, 5, 8):
        owner = shard.partition(lay.n, lay.lo, nr)
        counts = np.bincount(owner, minlength=nr)
        assert counts.sum() == lay.npatch and counts.max() - counts.min() <= 1
        key = shard.morton_key(lay.lo[:, 0] // 4, lay.lo[:, 1] // 4, lay.lo[:, 2] // 4)
        assert np.all(np.diff(owner[np.argsort(key)]) >= 0)      # contiguous stretches of the curve
    # a 2^3 split of 8^3 patches gives the octants
    owner = shard.partition(lay.n, lay.lo, 8)
    oct_ = (lay.lo[:, 0] >= 16) + 2 * (lay.lo[:, 1] >= 16) + 4 * (lay.lo[:, 2] >= 16)
    assert np.array_equal(owner, oct_)


def test_share_lists_are_symmetric():
    lay = ics.mixed_blocks(2, 24, sizes=(6, 8, 12), probs=(1, 1, 1), seed=5)
    owner = shard.partition(lay.n, lay.lo, 3)
    plans = [shard.RankPlan(lay.n, lay.lo, lay.base_cells, owner, r) for r in range(3)]
    nb = shard.neighbours(lay.n, lay.lo, lay.base_cells, 3)
    for r, p in enumerate(plans):
        assert set(p.ids[p.owned == 1].tolist()) == set(np.nonzero(owner == r)[0].tolist())
        for q in range(3):
            if q == r:
                continue
            a = p.send.get(q, np.zeros(0, np.int64))
            b = plans[q].recv.get(r, np.zeros(0, np.int64))
            assert np.array_equal(a, b), (r, q)
        # every neighbour of an owned patch is in the share
        for g in p.ids[p.owned == 1]:
            assert set(nb[g].tolist()) <= set(p.ids.tolist())
        # boundary = owned patches with a foreign neighbour
        bnd = {int(g) for g in p.ids[p.owned == 1] if any(owner[q] != r for q in nb[g])}
        assert bnd == set(p.boundary.tolist())


def _check_against_one_process(lay, f, state, finals, scheds):
    o = one_process(lay, f, state)
    ref = per_patch(lay, o.get_state())
    for g, arrays in finals.items():
        for k in range(4):
            assert np.array_equal(arrays[k], ref[k][g]), (g, k)
    assert sorted(finals) == list(range(lay.npatch))
    rp, rt, rd = o.schedule()
    key = lambda p, t, d: sorted(zip(p.tolist(), t.tolist(), d.tolist()))
    allp = np.concatenate([s[0] for s in scheds])
    allt = np.concatenate([s[1] for s in scheds])
    alld = np.concatenate([s[2] for s in scheds])
    assert key(allp, allt, alld) == key(rp, rt, rd)
    assert len(np.unique(rd)) >= 3             # the steps do differ between patches


def _collect(plan, eng):
    st = per_patch(type("L", (), {"n": plan.n})(), eng.state())
    finals = {int(g): [st[k][j] for k in range(4)] for j, g in enumerate(plan.ids) if plan.owned[j]}
    p, t, d = eng.schedule()
    return finals, (plan.ids[p], t, d)


@pytest.mark.parametrize("nranks", [2, 3])
def test_shares_in_one_process_equal_the_one_process_run(nranks):
    lay, f = lts_case()
    state = ics.to_patches(lay, f)
    owner = shard.partition(lay.n, lay.lo, nranks)
    runners = []
    for r in range(nranks):
        plan = shard.RankPlan(lay.n, lay.lo, lay.base_cells, owner, r)
        eng = OracleEngine(plan, **kw_of(lay, f))
        eng.set_state(plan.cut(state, lay.n))
        runners.append(shard.ShardRunner(eng, plan))
    rounds = shard.run_local(runners, T_END)
    assert rounds > 3
    finals, scheds = {}, []
    for r in runners:
        fin, sch = _collect(r.plan, r.engine)
        finals.update(fin)
        scheds.append(sch)
    _check_against_one_process(lay, f, state, finals, scheds)


def _rank_main(rank, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    from paper_1705_10774_gb300 import ics, shard
    from shard_oracle import OracleEngine
    dist.init_process_group("gloo", rank=rank, world_size=2)
    lay, f = lts_case()
    state = ics.to_patches(lay, f)
    owner = shard.partition(lay.n, lay.lo, 2)
    plan = shard.RankPlan(lay.n, lay.lo, lay.base_cells, owner, rank)
    eng = OracleEngine(plan, **kw_of(lay, f))
    eng.set_state(plan.cut(state, lay.n))
    runner = shard.ShardRunner(eng, plan)
    rounds = shard.run_distributed(runner, T_END, device="cpu")
    finals, sched = _collect(plan, eng)
    q.put((rank, rounds, finals, sched, len(plan.boundary), int((plan.owned == 0).sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_the_one_process_run():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ps = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(2)), key=lambda x: x[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == res[1][1]                    # the ranks ran the same number of rounds
    assert all(r[4] > 0 and r[5] > 0 for r in res)   # both have boundary and virtual patches
    lay, f = lts_case()
    finals = {**res[0][2], **res[1][2]}
    _check_against_one_process(lay, f, ics.to_patches(lay, f), finals, [res[0][3], res[1][3]])
