"""Sharding the patches over processes with virtual patches (DISPATCH I,
Sec. 3 C, the MPI process view).

Each process owns a contiguous stretch of the patches along a Morton
(Z-order) curve, so that its share is compact and its boundary small.  It
holds its own patches and a *virtual* copy of every patch of another process
that neighbours one of its own ('boundary' patches are its own patches with
such neighbours; the rest are 'internal').  After a sweep the process sends
every boundary patch it updated to each process holding it as a virtual
copy: the whole interior and the time parameters, proactively, as the paper
ships them, so that the receivers' neighbour tests see the new time at once.
A receiver stores the package as the virtual copy's new slice.

The processes advance in lock-step sweeps: sweep (each process updates its
ready patches from the slices before the sweep), exchange the packages, then
test for the end.  Because a sweep updates exactly the patches that are
ready by Eq. (1) and reads only slices from before the sweep, the union of
the processes' sweeps is the one-process sweep: the schedule and the states
are identical to a single process's, bit for bit.  Local time steps with
g = 0 (a global step would need a minimum over all processes every sweep).

This module holds the host logic: the partition, each process's share and
its send and receive lists, and the sweep / exchange / end-test loop over an
`engine` (the CUDA library's context, `DispatchEngine`, or any object with
the same methods) and a transport (torch.distributed point-to-point calls, or
an in-process loop over several engines).  There is no collective on the
data path: packages go point to point, and the end test is one small sum.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- geometry

def neighbours(n, lo, base_cells, nguard):
    """Neighbour lists of a one-level periodic layout: patch j neighbours
    patch i if j's interior meets i's box padded by nguard cells (periodic
    images), i itself excluded -- the library's definition.  Returns a list
    of sorted index arrays."""
    n = np.asarray(n, np.int64).reshape(-1, 3)
    lo = np.asarray(lo, np.int64).reshape(-1, 3)
    L = np.asarray(base_cells, np.int64)
    hit = np.ones((n.shape[0], n.shape[0]), bool)
    for d in range(3):
        a, la = lo[:, d] - nguard, np.minimum(n[:, d] + 2 * nguard, L[d])   # padded interval of i
        b, lb = lo[:, d], n[:, d]                                           # interior of j
        # two arcs of a circle of length L meet iff either starts inside the other
        d1 = np.mod(b[None, :] - a[:, None], L[d])
        d2 = np.mod(a[:, None] - b[None, :], L[d])
        hit &= (d1 < la[:, None]) | (d2 < lb[None, :])
    np.fill_diagonal(hit, False)
    return [np.nonzero(hit[i])[0] for i in range(n.shape[0])]


def morton_key(ix, iy, iz, bits=21):
    """Interleave the bits of three non-negative integer arrays (x lowest)."""
    key = np.zeros(np.shape(ix), np.int64)
    for b in range(bits):
        key |= ((np.asarray(ix, np.int64) >> b) & 1) << (3 * b)
        key |= ((np.asarray(iy, np.int64) >> b) & 1) << (3 * b + 1)
        key |= ((np.asarray(iz, np.int64) >> b) & 1) << (3 * b + 2)
    return key


def partition(n, lo, nranks):
    """Owner rank of each patch: the patches sorted along a Morton curve
    through their first cells (in units of the smallest patch size), cut into
    nranks contiguous stretches of about equal cell counts."""
    n = np.asarray(n, np.int64).reshape(-1, 3)
    lo = np.asarray(lo, np.int64).reshape(-1, 3)
    unit = max(int(n.min()), 1)
    key = morton_key(lo[:, 0] // unit, lo[:, 1] // unit, lo[:, 2] // unit)
    order = np.argsort(key, kind="stable")
    cells = np.prod(n, axis=1)[order]
    cum = np.cumsum(cells) - cells                     # cells before each patch
    owner = np.empty(n.shape[0], np.int64)
    owner[order] = np.minimum((cum * nranks) // cells.sum(), nranks - 1)
    return owner


class RankPlan:
    """One process's share: its own patches and the virtual copies of their
    neighbours on other processes, in ascending global order (`ids`; local
    index k is global patch ids[k]), the ownership mask, and per peer
    process the boundary patches to send and the virtual patches to
    receive (both sorted by global index, so that a sender's list to q is
    q's receive list from it)."""

    def __init__(self, n, lo, base_cells, owner, rank, nguard=3):
        n = np.asarray(n, np.int64).reshape(-1, 3)
        lo = np.asarray(lo, np.int64).reshape(-1, 3)
        owner = np.asarray(owner, np.int64)
        nb = neighbours(n, lo, base_cells, nguard)
        mine = np.nonzero(owner == rank)[0]
        virt = sorted({int(q) for p in mine for q in nb[p] if owner[q] != rank})
        self.rank = rank
        self.ids = np.array(sorted(set(mine.tolist()) | set(virt)), np.int64)
        self.owned = (owner[self.ids] == rank).astype(np.uint8)
        self.local = {int(g): k for k, g in enumerate(self.ids)}
        self.n, self.lo = n[self.ids], lo[self.ids]
        send = {}
        for p in mine:
            for q in nb[p]:
                r = int(owner[q])
                if r != rank:
                    send.setdefault(r, set()).add(int(p))
        self.send = {r: np.array(sorted(v), np.int64) for r, v in sorted(send.items())}
        recv = {}
        for v in virt:
            recv.setdefault(int(owner[v]), []).append(v)
        self.recv = {r: np.array(sorted(v), np.int64) for r, v in sorted(recv.items())}
        self.peers = sorted(set(self.send) | set(self.recv))
        self.boundary = np.array(sorted({int(p) for lst in self.send.values() for p in lst}), np.int64)

    def to_local(self, gids):
        return np.array([self.local[int(g)] for g in gids], np.int64)

    def cut(self, arrays, n_all):
        """This share's part of whole-domain patch arrays (U, bx, by, bz,
        concatenated over all patches in global order, patch sizes n_all)."""
        n_all = np.asarray(n_all, np.int64).reshape(-1, 3)
        nx, ny, nz = n_all[:, 0], n_all[:, 1], n_all[:, 2]
        per = [5 * nx * ny * nz, (nx + 1) * ny * nz, nx * (ny + 1) * nz, nx * ny * (nz + 1)]
        out = []
        for a, s in zip(arrays, per):
            off = np.concatenate([[0], np.cumsum(s)])
            out.append(np.concatenate([a[off[g]:off[g + 1]] for g in self.ids]))
        return out


# ---------------------------------------------------------------- the loop

class ShardRunner:
    """One process's side of the lock-step loop, over an engine with
    sweep(t_end) -> patch updates, times() -> local patch times,
    pack(local ids) -> (values, meta), unpack(local ids, values, meta) and
    package_len(local ids)."""

    def __init__(self, engine, plan: RankPlan):
        self.engine = engine
        self.plan = plan
        self._t = np.asarray(engine.times(), np.float64).copy()

    def sweep(self, t_end):
        return int(self.engine.sweep(t_end))

    def outbox(self):
        """{peer: (global ids, values, meta)} for every boundary patch
        updated since the last call (its time moved)."""
        t = np.asarray(self.engine.times(), np.float64)
        moved = t != self._t
        self._t = t.copy()
        out = {}
        for peer, lst in self.plan.send.items():
            gids = np.array([g for g in lst if moved[self.plan.local[int(g)]]], np.int64)
            if gids.size:
                vals, meta = self.engine.pack(self.plan.to_local(gids))
                out[peer] = (gids, vals, meta)
            else:
                out[peer] = (gids, None, None)
        return out

    def inbox(self, peer, gids, vals, meta):
        if len(gids) == 0:
            return
        expect = set(self.plan.recv.get(peer, np.zeros(0, np.int64)).tolist())
        if not set(int(g) for g in gids) <= expect:
            raise RuntimeError("rank %d: package from %d for patches it does not hold" % (self.plan.rank, peer))
        loc = self.plan.to_local(gids)
        self.engine.unpack(loc, vals, meta)
        m = meta.cpu().numpy() if hasattr(meta, "cpu") else np.asarray(meta)
        self._t[loc] = np.asarray(m, np.float64).reshape(-1, 3)[:, 0]

    def not_done(self, t_end):
        t = np.asarray(self.engine.times(), np.float64)
        return int(np.sum((t < t_end) & (self.plan.owned == 1)))


class ShardDeadlock(RuntimeError):
    pass


def run_local(runners, t_end, max_rounds=1 << 30):
    """Several processes' shares advanced in one process (one transport-free
    loop): sweep every share, hand every package to its receiver, repeat
    until every owned patch reached t_end.  Returns the number of rounds."""
    for rnd in range(max_rounds):
        updates = sum(r.sweep(t_end) for r in runners)
        outs = [r.outbox() for r in runners]
        for src, out in enumerate(outs):
            for peer, (gids, vals, meta) in out.items():
                runners[peer].inbox(src, gids, vals, meta)
        if sum(r.not_done(t_end) for r in runners) == 0:
            return rnd + 1
        if updates == 0:
            raise ShardDeadlock("no process has a ready patch but some are behind t_end")
    return max_rounds


def run_distributed(runner, t_end, device="cpu", group=None, max_rounds=1 << 30):
    """This process's side of the loop over torch.distributed: per round one
    sweep, then point-to-point exchanges with each peer -- first the list of
    patches coming (a fixed-size int64 header: count, then global indices),
    then their values and meta -- and one all-reduce of (patches behind
    t_end, updates) for the end test.  `device` is where the transport wants
    its tensors ("cpu" for gloo, "cuda" for nccl).  Returns the rounds."""
    import torch
    import torch.distributed as dist
    plan = runner.plan
    eng = runner.engine
    for rnd in range(max_rounds):
        updates = runner.sweep(t_end)
        out = runner.outbox()
        reqs, hin = [], {}
        for peer in plan.peers:
            ns = len(plan.send.get(peer, ()))
            if ns:
                gids = out[peer][0]
                h = torch.full((ns + 1,), -1, dtype=torch.int64)
                h[0] = len(gids)
                h[1:1 + len(gids)] = torch.from_numpy(gids)
                reqs.append(dist.isend(h.to(device), peer, group=group))
            nr = len(plan.recv.get(peer, ()))
            if nr:
                hin[peer] = torch.empty(nr + 1, dtype=torch.int64, device=device)
                reqs.append(dist.irecv(hin[peer], peer, group=group))
        for q in reqs:
            q.wait()
        reqs, bufs = [], {}
        for peer in plan.peers:
            if peer in out and len(out[peer][0]):
                _, vals, meta = out[peer]
                reqs.append(dist.isend(torch.as_tensor(vals).to(device).contiguous(), peer, group=group))
                reqs.append(dist.isend(torch.as_tensor(meta).to(device).contiguous(), peer, group=group))
            if peer in hin:
                k = int(hin[peer][0].item())
                if k:
                    gids = hin[peer][1:1 + k].cpu().numpy()
                    nvals = eng.package_len(plan.to_local(gids))
                    v = torch.empty(nvals, dtype=eng.torch_dtype, device=device)
                    m = torch.empty((k, 3), dtype=torch.float64, device=device)
                    reqs.append(dist.irecv(v, peer, group=group))
                    reqs.append(dist.irecv(m, peer, group=group))
                    bufs[peer] = (gids, v, m)
        for q in reqs:
            q.wait()
        for peer, (gids, v, m) in bufs.items():
            runner.inbox(peer, gids, eng.from_transport(v), eng.from_transport(m))
        tot = torch.tensor([runner.not_done(t_end), updates], dtype=torch.int64, device=device)
        dist.all_reduce(tot, group=group)
        if int(tot[0]) == 0:
            return rnd + 1
        if int(tot[1]) == 0:
            raise ShardDeadlock("no process has a ready patch but some are behind t_end")
    return max_rounds


class DispatchEngine:
    """A share advanced by the CUDA library: a context of the share's
    patches with the virtual ones marked (dsp_params.owned), local steps,
    sweeps; packages stay on the device."""

    def __init__(self, plan: RankPlan, base_cells, box_len=(1.0, 1.0, 1.0), **kw):
        import torch
        from .dispatch import Dispatch
        kw.setdefault("time_mode", 1)
        self.g = Dispatch(plan.n, plan.lo, base_cells=base_cells, box_len=box_len, owned=plan.owned, **kw)
        self.torch_dtype = torch.float32 if self.g.precision == 1 else torch.float64

    def set_state(self, arrays):
        self.g.set_state(*arrays)

    def sweep(self, t_end):
        return self.g.advance(t_end=t_end, max_sweeps=1)["patch_updates"]

    def times(self):
        return self.g.times()[0]

    def pack(self, loc):
        return self.g.pack(loc, device=True)

    def unpack(self, loc, vals, meta):
        self.g.unpack(loc, vals.cuda(), meta.cuda())

    def package_len(self, loc):
        return self.g.package_len(loc)

    def from_transport(self, t):
        return t

    def close(self):
        self.g.close()
