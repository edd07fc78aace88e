"""Sharding on the GPU (DISPATCH I, Sec. 3 C): several processes' shares,
each a library context holding its own patches and virtual copies of their
neighbours (dsp_params.owned), advanced in lock-step sweeps with the
packages handed over between them (dsp_pack / dsp_unpack) -- here all on
one GPU in one process, driven from the host (no kernel waits on another
context) -- give the schedule and the states of one context holding every
patch, bit for bit, and of the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_10774_gb300 import ics, shard
from paper_1705_10774_gb300.dispatch import DSP_ERR_INVALID_ARG, DSP_ERR_UNSUPPORTED, Dispatch, DispatchError
from oracle import Oracle

from test_shard import T_END, _check_against_one_process, lts_case, per_patch


def kw_of(lay, f):
    return dict(gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)


@pytest.mark.parametrize("nranks,precision", [(2, 0), (3, 0), (2, 1)])
def test_gpu_shares_equal_one_context(nranks, precision):
    lay, f = lts_case()
    state = ics.to_patches(lay, f)
    owner = shard.partition(lay.n, lay.lo, nranks)
    runners = []
    for r in range(nranks):
        plan = shard.RankPlan(lay.n, lay.lo, lay.base_cells, owner, r)
        eng = shard.DispatchEngine(plan, lay.base_cells, lay.box_len, gamma=f.gamma, cfl=0.4, precision=precision,
                                   sched_capacity=1 << 20)
        eng.set_state(plan.cut(state, lay.n))
        runners.append(shard.ShardRunner(eng, plan))
    shard.run_local(runners, T_END)
    finals, scheds = {}, []
    for r in runners:
        st = per_patch(type("L", (), {"n": r.plan.n})(), r.engine.g.get_state())
        for j, g in enumerate(r.plan.ids):
            if r.plan.owned[j]:
                finals[int(g)] = [st[k][j] for k in range(4)]
        p, t, d = r.engine.g.schedule()
        scheds.append((r.plan.ids[p], t, d))
        r.engine.close()
    one = Dispatch(lay.n, lay.lo, precision=precision, time_mode=1, sched_capacity=1 << 20, **kw_of(lay, f))
    one.set_state(*state)
    one.advance(t_end=T_END)
    ref = per_patch(lay, one.get_state())
    for g, arrays in finals.items():
        for k in range(4):
            assert np.array_equal(arrays[k], ref[k][g]), (g, k)
    key = lambda p, t, d: sorted(zip(p.tolist(), t.tolist(), d.tolist()))
    cat = lambda i: np.concatenate([s[i] for s in scheds])
    assert key(cat(0), cat(1), cat(2)) == key(*one.schedule())
    if precision == 0:
        _check_against_one_process(lay, f, state, finals, scheds)


def test_packages_round_trip_and_reject_owned_patches():
    lay, f = lts_case()
    state = ics.to_patches(lay, f)
    owner = shard.partition(lay.n, lay.lo, 2)
    plans = [shard.RankPlan(lay.n, lay.lo, lay.base_cells, owner, r) for r in range(2)]
    engs = [shard.DispatchEngine(p, lay.base_cells, lay.box_len, gamma=f.gamma, cfl=0.4) for p in plans]
    for p, e in zip(plans, engs):
        e.set_state(p.cut(state, lay.n))
    engs[0].sweep(T_END)
    gids = plans[0].send[1][:5]
    vals, meta = engs[0].pack(plans[0].to_local(gids))
    loc1 = plans[1].to_local(gids)
    engs[1].unpack(loc1, vals, meta)
    v2, m2 = engs[1].pack(loc1)
    assert torch.equal(vals, v2) and torch.equal(meta, m2)
    h_vals, h_meta = engs[1].g.pack(loc1, device=False)          # host path
    assert np.array_equal(h_vals, vals.cpu().numpy()) and np.array_equal(h_meta, meta.cpu().numpy())
    assert np.array_equal(engs[1].times()[loc1], meta[:, 0].cpu().numpy())
    owned_local = np.nonzero(plans[1].owned)[0][:1]
    with pytest.raises(DispatchError) as e:
        engs[1].g.unpack(owned_local, vals[:engs[1].package_len(owned_local)], meta[:1])
    assert e.value.code == DSP_ERR_INVALID_ARG
    for e_ in engs:
        e_.close()


def test_share_layouts_are_checked():
    lay, f = lts_case()
    owner = shard.partition(lay.n, lay.lo, 2)
    plan = shard.RankPlan(lay.n, lay.lo, lay.base_cells, owner, 0)
    kw = kw_of(lay, f)
    with pytest.raises(DispatchError) as e:          # a global step needs every process
        Dispatch(plan.n, plan.lo, owned=plan.owned, time_mode=0, **kw)
    assert e.value.code == DSP_ERR_UNSUPPORTED
    keep = [k for k in range(len(plan.ids)) if not (plan.owned[k] == 0 and k % 2)]    # drop some virtual patches
    with pytest.raises(DispatchError) as e:          # guard cells of owned patches not covered
        Dispatch(plan.n[keep], plan.lo[keep], owned=plan.owned[keep], time_mode=1, **kw)
    assert e.value.code == DSP_ERR_INVALID_ARG
