"""Domain decomposition on the CPU: the library's halo plan (lbm_halo_plan, host
code) drives a numpy pack / unpack around the FP64 oracle's step, and a grid split
into slabs must reproduce the undivided oracle run.  The comparison allows 1e-13:
the oracle forms the moments with a BLAS product whose summation order depends on
the array's size, so slab and undivided runs round differently at the 1e-15
level, while a wrong or missing halo segment moves populations by ~1e-2 (the
fields carry 1e-2 noise).

* One process, several uneven slabs (the message routing of SlabGrid).
* Two gloo ranks, one slab each, the messages through torch.distributed
  point-to-point calls (exchange_halos, the routing a multi-process run uses).
"""
import os
import socket

import numpy as np
import pytest

from oracle import lbm as olbm
from oracle.model import get_model
from paper_1303_4624_gb300 import slabs
from paper_1303_4624_gb300 import workloads as W

lbm = pytest.importorskip("paper_1303_4624_gb300.lbm")


def to_library_order(mdl, lib_e, S):
    """Oracle direction order -> the library's (the halo plan indexes the latter)."""
    pos = {tuple(v): j for j, v in enumerate(mdl.e.tolist())}
    return S[[pos[tuple(v)] for v in lib_e.tolist()]]


def np_pack(S, axis, plan):
    """Message of the (direction, local plane) segments of S [Q, Nz, Ny, Nx]."""
    if axis == 2:
        return np.stack([S[i, p] for i, p in plan]).reshape(-1)
    return np.stack([S[i, 0, p] for i, p in plan]).reshape(-1)


def np_unpack(S, axis, plan, msg):
    plane = S.shape[2] * S.shape[3] if axis == 2 else S.shape[3]
    for j, (i, p) in enumerate(plan):
        seg = msg[j * plane:(j + 1) * plane]
        if axis == 2:
            S[i, p] = seg.reshape(S.shape[2], S.shape[3])
        else:
            S[i, 0, p] = seg


class OracleSlab:
    """One slab advanced by the oracle; state in the library's direction order."""

    def __init__(self, model, fields, start, count, omega):
        self.mdl = get_model(model)
        self.info = lbm.lbm_model_info(model)
        self.axis = 2 if self.mdl.D == 3 else 1
        self.R = self.info["reach"]
        self.n, self.omega = count, omega
        loc = [slabs.local_fields(a, self.axis, start, count, self.R)
               for a in (fields.rho, fields.U, fields.theta * self.mdl.T0)]
        S = olbm.init_populations(self.mdl, *loc)
        self.perm = [ {tuple(v): j for j, v in enumerate(self.mdl.e.tolist())}[tuple(v)]
                      for v in self.info["e"].tolist()]
        self.inv = np.argsort(self.perm)
        self.S = S[self.perm]
        self.plans = {(f, s): lbm.lbm_halo_plan(model, count, f, s) for f in (0, 1) for s in (0, 1)}

    def step(self):
        self.S = olbm.step(self.mdl, self.S[self.inv], self.omega)[self.perm]

    def pack(self, face):
        return np_pack(self.S, self.axis, self.plans[(face, 1)])

    def unpack(self, face, msg):
        np_unpack(self.S, self.axis, self.plans[(face, 0)], msg)

    def interior(self):
        return slabs.interior(self.S, self.axis, self.R)


def global_run(model, fields, omega, steps):
    mdl = get_model(model)
    info = lbm.lbm_model_info(model)
    S = olbm.init_populations(mdl, fields.rho, fields.U, fields.theta * mdl.T0)
    S = olbm.run(mdl, S, omega, steps)
    return to_library_order(mdl, info["e"], S)


CASES = [("D3Q95", (6, 5, 18), [5, 6, 7]), ("D3Q95", (7, 4, 10), [10]),
         ("D2Q33", (9, 13, 1), [4, 5, 4])]


@pytest.mark.parametrize("model,dims,splits", CASES)
def test_halo_plan_reproduces_the_undivided_grid(model, dims, splits):
    """Slabs of uneven thickness (one slab: its own neighbour across the periodic
    seam), 6 steps: every interior population matches the undivided run (to the
    rounding bound above)."""
    D = 3 if model == "D3Q95" else 2
    axis = 2 if D == 3 else 1
    fields = W.riemann_planar(D, *dims, dims[0] // 2, (1.0, 1.0), (0.6, 0.75), seed=5, noise=1e-2)
    omega, steps = 1.7, 6
    starts = np.cumsum([0] + splits[:-1])
    sl = [OracleSlab(model, fields, s0, n, omega) for s0, n in zip(starts, splits)]
    k = len(sl)
    for _ in range(steps):
        for s in sl:
            s.step()
        up = [s.pack(1) for s in sl]
        down = [s.pack(0) for s in sl]
        for i, s in enumerate(sl):
            s.unpack(0, up[(i - 1) % k])
            s.unpack(1, down[(i + 1) % k])
    got = np.concatenate([s.interior() for s in sl], axis=3 - axis)
    ref = global_run(model, fields, omega, steps)
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


def test_halo_plan_sizes_and_refusals():
    """102 plane-populations per face for D3Q95 (sum of the positive z components),
    26 for D2Q33 (y); send and receive lists pair up; slabs thinner than the reach
    are refused."""
    for model, n in (("D3Q95", 102), ("D2Q33", 26)):
        e = lbm.lbm_model_info(model)["e"]
        comp = e[:, 2] if model == "D3Q95" else e[:, 1]
        assert comp[comp > 0].sum() == n
        for face in (0, 1):
            s = lbm.lbm_halo_plan(model, 7, face, 1)
            r = lbm.lbm_halo_plan(model, 9, 1 - face, 0)     # the neighbour's receive list
            assert s.shape == (n, 2) and np.array_equal(s[:, 0], r[:, 0])
    with pytest.raises(lbm.LbmError):
        lbm.lbm_halo_plan("D3Q95", 4, 0, 1)


# ---------------------------------------------------------------- two gloo ranks

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q, model, dims, splits, steps):
    import torch
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        D = 3 if model == "D3Q95" else 2
        fields = W.riemann_planar(D, *dims, dims[0] // 2, (1.0, 1.0), (0.6, 0.75), seed=8,
                                  noise=1e-2)
        starts = np.cumsum([0] + splits[:-1])
        me = OracleSlab(model, fields, starts[rank], splits[rank], 1.6)
        nmsg = me.plans[(0, 1)].shape[0] * (dims[0] * dims[1] if D == 3 else dims[0])
        bufs = tuple(torch.zeros(nmsg, dtype=torch.float64) for _ in range(4))

        def pack(face, buf):
            buf.copy_(torch.from_numpy(me.pack(face)))

        def unpack(face, buf):
            me.unpack(face, buf.numpy())

        for _ in range(steps):
            me.step()
            slabs.exchange_halos(pack, unpack, bufs, rank, world)
        q.put((rank, me.interior()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("model,dims,splits", [("D3Q95", (5, 4, 13), [6, 7]),
                                               ("D2Q33", (8, 10, 1), [4, 6])])
def test_two_gloo_ranks_reproduce_the_undivided_grid(model, dims, splits):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    steps = 5
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q, model, dims, splits, steps))
             for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    axis = 2 if model == "D3Q95" else 1
    got = np.concatenate([out[0], out[1]], axis=3 - axis)
    D = 3 if model == "D3Q95" else 2
    fields = W.riemann_planar(D, *dims, dims[0] // 2, (1.0, 1.0), (0.6, 0.75), seed=8, noise=1e-2)
    ref = global_run(model, fields, 1.6, steps)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
