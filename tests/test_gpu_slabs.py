"""z-slab decomposition through the C ABI on one GPU: several handles, one
per slab of the grid (each with its halo), stepped one after the other and
exchanging halos by device copies after every step (LocalExchange; no kernel
waits for another), must reproduce one handle over the whole grid bit for
bit in the owned layers: FP64 and mixed paths, periodic and outflow grids,
curved metric with a conductivity profile, Gauss's-law charge, another IMEX
scheme, and slabs thinner than the halo."""
import numpy as np
import pytest

import workloads as W
from paper_2510_18968_b300 import slabs as S
from tests.helpers import make_solver

pytestmark = pytest.mark.gpu


def _with(wl, **p):
    wl.params.update(p)
    return wl


CASES = {
    "blast_mc2": lambda: W.cyl_blast(n=32, nz=24),
    "alfven_weno5": lambda: W.alfven_diag(n=16, sigma=1e4),
    "star_weno5": lambda: W.lane_emden_star(n=20),
    "blast_gauss": lambda: _with(W.cyl_blast(n=24, nz=24), qflux_mode=2),
    "blast_ssp3433": lambda: _with(W.cyl_blast(n=24, nz=24), imex=3),
}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,world", [("blast_mc2", 2), ("blast_mc2", 3), ("alfven_weno5", 2),
                                        ("alfven_weno5", 4), ("star_weno5", 2),
                                        ("blast_gauss", 2), ("blast_ssp3433", 3)])
def test_slab_handles_reproduce_the_whole_grid_bit_for_bit(name, world, precision):
    import torch
    import paper_2510_18968_b300 as R
    wl = CASES[name]()
    wl.params["precision"] = precision
    nsteps = 4
    ref = make_solver(wl)
    ref.step(wl.dt, nsteps)
    cons, prim = ref.get_cons(), ref.get_prims()
    ref.close()
    nz = wl.params["n"][2]
    H = S.halo_layers(wl.params)
    periodic = wl.params["bc"][2] == 0
    metric = wl.metric_arrays() if wl.alpha is not None else None
    slabs = [S.make_slab(nz, world, r, H, periodic) for r in range(world)]
    solvers = [S.slab_solver(R, wl.params, wl.prim, metric, wl.sigma_profile, sl)
               for sl in slabs]
    ex = S.LocalExchange([S.SolverStepper(s) for s in solvers], nz, H, periodic)
    for _ in range(nsteps):
        for s in solvers:
            s.step(wl.dt, 1, sync=False)
        ex.exchange()
    torch.cuda.synchronize()
    for sl, s in zip(slabs, solvers):
        lo, hi = sl.local_owned()
        c, p = s.get_cons(), s.get_prims()
        assert np.array_equal(c[:, lo:hi], cons[:, sl.z0:sl.z1]), (name, sl.rank)
        assert np.array_equal(p[:, lo:hi], prim[:, sl.z0:sl.z1]), (name, sl.rank)
        s.close()


def test_state_layers_round_trip_and_bad_ranges():
    import torch
    import paper_2510_18968_b300 as R
    wl = W.cyl_blast(n=16, nz=8)
    for precision in (0, 1):
        wl.params["precision"] = precision
        s = make_solver(wl)
        s.step(wl.dt, 2)
        lb = s.state_layer_bytes()
        assert lb == 16 * 16 * (14 * 8 + 14 * (4 if precision else 8) + (32 if precision else 0))
        host = np.zeros(3 * lb, np.uint8)
        s.get_state_layers(2, 3, host)
        dev = torch.empty(3 * lb, dtype=torch.uint8, device="cuda")
        s.get_state_layers(2, 3, dev)
        assert np.array_equal(dev.cpu().numpy(), host)
        cons, prim = s.get_cons(), s.get_prims()
        s.set_state_layers(2, 3, dev)
        assert np.array_equal(s.get_cons(), cons) and np.array_equal(s.get_prims(), prim)
        for k0, nk in ((-1, 2), (7, 2), (0, 0)):
            with pytest.raises((R.RMHDError, ValueError)):
                s.get_state_layers(k0, nk, torch.empty(max(nk, 1) * lb, dtype=torch.uint8,
                                                       device="cuda"))
        s.close()
