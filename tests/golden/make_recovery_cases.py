"""Write tests/golden/recovery_hard_cases.npz: stage-1 recovery inputs on
which the paper's iteration fails although a root exists (magnetised blast
front of the 256^2 cylindrical explosion, step 17, sigma = 1e3); the stored
set was picked where a damped 4D Newton on (p, v_i) stalls too.  Calls only
the oracle and the input generators."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def main():
    wl = W.cyl_blast(n=256, nz=1)
    a, b, g, K = wl.metric_arrays()
    m = oracle.Metric(a.ravel(), b.reshape(3, -1), g.reshape(6, -1), K.reshape(6, -1))
    prim = np.ascontiguousarray(wl.prim.copy())
    cons = oracle.prim2con_grid(wl.params, m, prim)
    oracle.step(wl.params, m, cons, prim, wl.dt, 17)
    c, p = cons.reshape(14, -1), prim.reshape(14, -1)
    P = oracle.make_params(**dict(wl.params, c2p_maxit=100))
    gam = 1.0 - 1.0 / np.sqrt(2.0)
    c_imp = gam * wl.dt
    # cells whose stage-1 recovery needs the pressure-bracket fallback
    # (status 4): the paper iteration fails there
    st = np.zeros(c.shape[1], int)
    its = np.zeros(c.shape[1], int)
    for i in range(c.shape[1]):
        _, _, its[i], st[i] = oracle.con2prim(P, c[:, i], 1, c_imp, wl.params["sigma0"], p[:, i])
    pick = np.where(st == 4)[0][:16]
    assert len(pick) > 0
    np.savez(os.path.join(HERE, "recovery_hard_cases.npz"), cons=c[:, pick], guess=p[:, pick],
             c=c_imp, sigma=wl.params["sigma0"], gamma_eos=wl.params["gamma_eos"],
             iters=its[pick])
    print("cells", pick, "iterations", its[pick], "statuses", np.bincount(st))


if __name__ == "__main__" and len(sys.argv) == 1:
    main()


def blast_step23():
    """Write tests/golden/recovery_blast_step23.npz: the stage-1 recovery
    inputs (U^n, guess P^n) of step 23 of the 256^2 cylindrical explosion
    (sigma = 1e3) at the four blast-front cells where the Newton solve of the
    velocity equations at the guess pressure does not converge from the
    guess velocity, so that the pressure bracket must start its velocity
    solves from rest."""
    wl = W.cyl_blast(n=256, nz=1)
    a, b, g, K = wl.metric_arrays()
    m = oracle.Metric(a.ravel(), b.reshape(3, -1), g.reshape(6, -1), K.reshape(6, -1))
    prim = np.ascontiguousarray(wl.prim.copy())
    cons = oracle.prim2con_grid(wl.params, m, prim)
    oracle.step(wl.params, m, cons, prim, wl.dt, 22)
    c, p = cons.reshape(14, -1), prim.reshape(14, -1)
    pick = np.array([26227, 26252, 39283, 39308])   # (x, y) = (115|140, 102|153)
    np.savez(os.path.join(HERE, "recovery_blast_step23.npz"), cons=c[:, pick], guess=p[:, pick],
             c=1.0 - 1.0 / np.sqrt(2.0), dt=wl.dt, sigma=wl.params["sigma0"],
             gamma_eos=wl.params["gamma_eos"], cells=pick)
    print("blast step 23 cells", pick)


if __name__ == "__main__" and len(sys.argv) > 1 and sys.argv[1] == "blast23":
    blast_step23()
