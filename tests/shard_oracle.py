"""The oracle as a share's engine for the sharding driver (test
infrastructure): the same methods as shard.DispatchEngine, over an oracle
context whose virtual patches are marked (Sec. 3 C)."""
import numpy as np

from oracle import Oracle


class OracleEngine:
    def __init__(self, plan, base_cells, box_len=(1.0, 1.0, 1.0), **kw):
        import torch
        kw.setdefault("time_mode", 1)
        self.o = Oracle(plan.n, plan.lo, base_cells=base_cells, box_len=box_len, **kw)
        self.o.set_owned(plan.owned)
        self.torch_dtype = torch.float64
        n = np.asarray(plan.n, np.int64)
        nx, ny, nz = n[:, 0], n[:, 1], n[:, 2]
        self.per = np.stack([5 * nx * ny * nz, (nx + 1) * ny * nz, nx * (ny + 1) * nz, nx * ny * (nz + 1)], axis=1)

    def set_state(self, arrays):
        self.o.set_state(*arrays)

    def sweep(self, t_end):
        before = self.o.stats()["patch_updates"]
        self.o.advance(t_end=t_end, max_sweeps=1)
        return self.o.stats()["patch_updates"] - before

    def times(self):
        return self.o.get_times()[0]

    def package_len(self, loc):
        return int(self.per[np.asarray(loc, np.int64)].sum())

    def pack(self, loc):
        vals, metas = [], []
        for k in loc:
            arrays, meta = self.o.newest(int(k))
            vals.extend(arrays)
            metas.append(meta)
        return np.concatenate(vals), np.stack(metas)

    def unpack(self, loc, vals, meta):
        vals = np.asarray(vals, np.float64)
        meta = np.asarray(meta, np.float64).reshape(-1, 3)
        off = 0
        for j, k in enumerate(loc):
            parts = []
            for s in self.per[int(k)]:
                parts.append(vals[off:off + s])
                off += s
            self.o.push(int(k), parts, meta[j])
        assert off == vals.size

    def from_transport(self, t):
        return t.numpy()

    def schedule(self):
        return self.o.schedule()

    def state(self):
        return self.o.get_state()
