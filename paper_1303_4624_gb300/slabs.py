"""Domain decomposition of a periodic grid into slabs (argument marshalling and
message routing only; every population moves through the library's kernels).

The grid is split along its slowest axis (z for D3Q95, y for D2Q33).  Each slab
is a context made by ``lbm_create_slab`` whose state carries R ghost planes on
each side (include/lbm.h describes the layout and the halo messages).  One step
of the decomposed grid is: every slab takes one ``lbm_step``, then every slab
packs its two outgoing messages and every slab unpacks the two it receives.

``SlabGrid`` holds all slabs of a grid on the current device (one process; the
messages move by device-to-device copies); ``exchange_halos`` moves one slab's
messages between processes with ``torch.distributed`` point-to-point calls, and
is written against pack / unpack callables so that the same routing serves any
transport.
"""
from __future__ import annotations

import numpy as np

from . import lbm as L

UP, DOWN = 1, 2      # message tags: towards higher / lower coordinates


def split_axis(model):
    """Index of the split axis in an x-fastest dims triple (2: z, 1: y)."""
    return 2 if L.lbm_model_info(model)["D"] == 3 else 1


def local_fields(fields_global, axis, start, count, ghost):
    """The planes start - ghost .. start + count + ghost - 1 (periodic) of global
    field arrays shaped [..., Nz, Ny, Nx]; axis is 2 (z) or 1 (y) of (x, y, z)."""
    arr_axis = -1 - axis
    n = fields_global.shape[arr_axis]
    idx = np.arange(start - ghost, start + count + ghost) % n
    return np.take(fields_global, idx, axis=arr_axis)


def interior(arr, axis, ghost):
    """The interior planes of a slab-local array shaped [..., Nz, Ny, Nx]."""
    arr_axis = arr.ndim - 1 - axis
    sl = [slice(None)] * arr.ndim
    sl[arr_axis] = slice(ghost, arr.shape[arr_axis] - ghost)
    return arr[tuple(sl)]


def exchange_halos(pack, unpack, bufs, rank, world, group=None):
    """One halo exchange of one slab between processes (rank r's upper neighbour is
    r + 1, periodic).  pack(face, buf) writes the message for the neighbour across
    face into buf, unpack(face, buf) stores the message received across face;
    bufs = (send_up, send_down, recv_below, recv_above), torch tensors on the
    transport's device.  With one process the slab is its own neighbour."""
    import torch.distributed as dist
    send_up, send_down, recv_below, recv_above = bufs
    pack(1, send_up)
    pack(0, send_down)
    if world == 1:
        unpack(0, send_up)
        unpack(1, send_down)
        return
    above, below = (rank + 1) % world, (rank - 1) % world
    ops = [dist.P2POp(dist.isend, send_up, above, group, UP),
           dist.P2POp(dist.isend, send_down, below, group, DOWN),
           dist.P2POp(dist.irecv, recv_below, below, group, UP),
           dist.P2POp(dist.irecv, recv_above, above, group, DOWN)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    unpack(0, recv_below)
    unpack(1, recv_above)


class SlabGrid:
    """All slabs of one periodic grid on the current device.

    splits: the interior plane counts of the slabs along the split axis, in order
    (their sum is the grid's extent there; each at least the stencil reach)."""

    def __init__(self, model, dims, omega, storage, splits, stream=None):
        import torch
        self.model, self.storage = model, storage
        self.dims = tuple(int(d) for d in dims)
        self.axis = split_axis(model)
        if sum(splits) != self.dims[self.axis]:
            raise ValueError("the slabs' planes must add up to the grid's extent")
        self.splits = [int(s) for s in splits]
        self.starts = list(np.cumsum([0] + self.splits[:-1]))
        self.info = L.lbm_model_info(model)
        self.ctxs = []
        for n in self.splits:
            d = list(self.dims)
            d[self.axis] = n
            self.ctxs.append(L.lbm_create_slab(model, d, omega, storage, stream))
        h = L.lbm_halo_info(self.ctxs[0])
        self.ghost = h["ghost"]
        nb = h["face_bytes"]
        self.up = [torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in self.ctxs]
        self.down = [torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in self.ctxs]

    def close(self):
        for c in self.ctxs:
            L.lbm_destroy(c)
        self.ctxs = []

    def init(self, rho, U, T):
        """Global fields (rho [Nz, Ny, Nx], U [D, ...], T, lattice units)."""
        for c, s0, n in zip(self.ctxs, self.starts, self.splits):
            L.lbm_init(c, np.ascontiguousarray(local_fields(rho, self.axis, s0, n, self.ghost)),
                       np.ascontiguousarray(local_fields(U, self.axis, s0, n, self.ghost)),
                       np.ascontiguousarray(local_fields(T, self.axis, s0, n, self.ghost)))

    def exchange(self):
        k = len(self.ctxs)
        for s, c in enumerate(self.ctxs):
            L.lbm_halo_pack(c, 1, self.up[s])
            L.lbm_halo_pack(c, 0, self.down[s])
        for s, c in enumerate(self.ctxs):
            L.lbm_halo_unpack(c, 0, self.up[(s - 1) % k])
            L.lbm_halo_unpack(c, 1, self.down[(s + 1) % k])

    def step(self, n=1):
        for _ in range(n):
            for c in self.ctxs:
                L.lbm_step(c, 1)
            self.exchange()

    def raw(self):
        """The stored state of the whole grid [Q, Nz, Ny, Nx] (interior planes)."""
        parts = []
        for c, n in zip(self.ctxs, self.splits):
            d = list(self.dims)
            d[self.axis] = n + 2 * self.ghost
            h = np.zeros((self.info["Q"], d[2], d[1], d[0]), dtype=L.STORAGE_DTYPE[L.STORAGES[self.storage]])
            L.lbm_get_raw(c, h)
            parts.append(interior(h, self.axis, self.ghost))
        return np.concatenate(parts, axis=3 - self.axis)

    def moments(self):
        """rho, U, T of the whole grid (interior planes)."""
        D = self.info["D"]
        out = []
        for c, n in zip(self.ctxs, self.splits):
            d = list(self.dims)
            d[self.axis] = n + 2 * self.ghost
            shape = (d[2], d[1], d[0])
            r, u, t = np.zeros(shape), np.zeros((D,) + shape), np.zeros(shape)
            L.lbm_moments(c, r, u, t)
            out.append((interior(r, self.axis, self.ghost), interior(u, self.axis, self.ghost),
                        interior(t, self.axis, self.ghost)))
        ax = 2 - self.axis
        return (np.concatenate([o[0] for o in out], axis=ax),
                np.concatenate([o[1] for o in out], axis=ax + 1),
                np.concatenate([o[2] for o in out], axis=ax))
