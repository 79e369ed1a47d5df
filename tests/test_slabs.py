"""z-slab decomposition (paper_2510_18968_b300/slabs.py) on the CPU.

The halo plan is checked directly (every halo layer is filled from its
owner, exactly once); then gloo ranks (world size 2 and 4, spawned
processes) each step their slab of a small grid with the oracle as the
stepper and exchange halos through torch.distributed after every step, and
the owned layers must equal a single-rank oracle run of the whole grid bit
for bit, on a periodic grid (WENO5 Alfven cube) and an outflow grid (MC2
cylindrical explosion), including slabs thinner than the halo (4 ranks)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2510_18968_b300 import slabs as S


@pytest.mark.parametrize("nz,world,H,periodic", [(16, 2, 6, True), (16, 4, 6, True),
                                                 (16, 2, 6, False), (16, 4, 6, False),
                                                 (12, 3, 9, True), (7, 3, 6, False)])
def test_exchange_plan_fills_every_halo_layer_from_its_owner(nz, world, H, periodic):
    slabs, plan = S.exchange_plan(nz, world, H, periodic)
    assert sum(s.z1 - s.z0 for s in slabs) == nz
    for d in slabs:
        filled = {}
        for (src, dst), runs in plan.items():
            if dst != d.rank:
                continue
            s = slabs[src]
            for ks, kd, n in runs:
                for q in range(n):
                    # the source layer is owned by the source rank and is the
                    # same global layer as the destination's halo layer
                    lo, hi = s.local_owned()
                    assert lo <= ks + q < hi
                    assert s.global_layer(ks + q) == d.global_layer(kd + q)
                    assert kd + q not in filled
                    filled[kd + q] = src
        lo, hi = d.local_owned()
        halo = [k for k in range(d.nz_local) if not lo <= k < hi]
        assert sorted(filled) == halo
        # the halo is H deep on every cut face, clipped at a domain face
        assert d.lo == (H if periodic else min(H, d.z0))
        assert d.hi == (H if periodic else min(H, nz - d.z1))


def test_halo_depth_per_scheme():
    assert S.halo_layers(dict(imex=0)) == 6
    assert S.halo_layers(dict(imex=3)) == 9
    assert S.halo_layers(dict(imex=0, qflux_mode=2)) == 9
    assert S.halo_layers(dict(imex=1, qflux_mode=2)) == 13


# --------------------------------------------------- gloo ranks, oracle

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload(name):
    import workloads as W
    if name == "alfven":
        # a longer periodic z-extent so that the slabs are 4-8 layers thick
        return _stretch_z(W.alfven_diag(n=8, sigma=1e3), 16)
    return W.cyl_blast(n=16, nz=16, L=1.5)


def _stretch_z(wl, nz):
    """The periodic Alfven wave on an 8 x 8 x nz grid (z period nz dz)."""
    import workloads as W
    P = dict(wl.params)
    n = (P["n"][0], P["n"][1], nz)
    dx = P["dx"]
    X, Y, Z = W.cell_centres(n, P["x0"], dx)
    tp = 2 * np.pi
    prim = np.zeros((14,) + X.shape)
    prim[0] = 1.0 + 0.1 * np.sin(tp * (X + Y))
    prim[1] = 1.0
    prim[2] = 0.1 * np.sin(tp * Z * 8 / nz)
    prim[3] = 0.1 * np.cos(tp * (X + Z * 8 / nz))
    prim[8] = 1.0
    prim[9] = 0.1 * np.cos(tp * Z * 8 / nz)
    prim[10] = 0.1 * np.sin(tp * (Y + Z * 8 / nz))
    v, B = prim[2:5], prim[8:11]
    prim[5:8] = -np.cross(v, B, axis=0)
    P["n"] = n
    return W.Workload("alfven_z", P, prim, wl.dt, 3)


class OracleStepper:
    """The oracle as a slab stepper (test infrastructure): the state is the
    conserved and primitive arrays of the slab's extended range."""

    def __init__(self, params, metric, cons, prim):
        import oracle
        self.oracle = oracle
        self.P, self.m, self.cons, self.prim = params, metric, cons, prim
        self.plane = prim.shape[2] * prim.shape[3]

    def layer_bytes(self):
        return 28 * 8 * self.plane

    def new_buffer(self, nbytes):
        import torch
        return torch.empty(nbytes, dtype=torch.uint8)

    def get_layers(self, k0, n, buf):
        a = buf.numpy().view(np.float64)
        a[:14 * n * self.plane] = self.cons[:, k0:k0 + n].ravel()
        a[14 * n * self.plane:] = self.prim[:, k0:k0 + n].ravel()

    def set_layers(self, k0, n, buf):
        a = buf.numpy().view(np.float64)
        self.cons[:, k0:k0 + n] = a[:14 * n * self.plane].reshape(14, n, *self.prim.shape[2:])
        self.prim[:, k0:k0 + n] = a[14 * n * self.plane:].reshape(14, n, *self.prim.shape[2:])

    def step(self, dt):
        st, _ = self.oracle.step(self.P, self.m, self.cons, self.prim, dt, 1)
        assert st == 0


def _oracle_slab(wl, slab):
    import oracle
    P = S.slab_params(wl.params, slab)
    prim = S.slab_arrays(slab, wl.prim)
    a, b, g, K = wl.metric_arrays()
    m = oracle.Metric(S.slab_arrays(slab, a).ravel(), S.slab_arrays(slab, b).reshape(3, -1),
                      S.slab_arrays(slab, g).reshape(6, -1), S.slab_arrays(slab, K).reshape(6, -1))
    cons = oracle.prim2con_grid(P, m, prim)
    return OracleStepper(P, m, cons, prim)


def _rank(rank, world, port, name, nsteps, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = _workload(name)
    nz = wl.params["n"][2]
    H = S.halo_layers(wl.params)
    periodic = wl.params["bc"][2] == 0
    slab = S.make_slab(nz, world, rank, H, periodic)
    st = _oracle_slab(wl, slab)
    ex = S.DistExchange(st, nz, H, periodic)
    for _ in range(nsteps):
        st.step(wl.dt)
        ex.exchange()
    lo, hi = slab.local_owned()
    out[rank] = (slab.z0, slab.z1, st.cons[:, lo:hi].copy(), st.prim[:, lo:hi].copy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name", ["alfven", "blast"])
@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_reproduce_the_single_rank_run_bit_for_bit(name, world):
    import oracle
    nsteps = 3
    wl = _workload(name)
    a, b, g, K = wl.metric_arrays()
    m = oracle.Metric(a.ravel(), b.reshape(3, -1), g.reshape(6, -1), K.reshape(6, -1))
    prim = np.ascontiguousarray(wl.prim.copy())
    cons = oracle.prim2con_grid(wl.params, m, prim)
    for _ in range(nsteps):
        oracle.step(wl.params, m, cons, prim, wl.dt, 1)
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), name, nsteps, out), nprocs=world, join=True)
        res = dict(out)
    covered = 0
    for r in range(world):
        z0, z1, c, p = res[r]
        assert np.array_equal(c, cons[:, z0:z1]), (r, np.abs(c - cons[:, z0:z1]).max())
        assert np.array_equal(p, prim[:, z0:z1]), r
        covered += z1 - z0
    assert covered == wl.params["n"][2]
