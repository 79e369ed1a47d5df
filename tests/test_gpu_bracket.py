"""The pressure bracket at the end of the recovery's fallback chain, run the
way the step's deferred passes run it: one warp per point, the velocity
solves' forward-difference columns and line-search step lengths evaluated
on the warp's lanes side by side.  Against the same chain in one thread per
point (the same decisions -- root or none, the same statuses -- and the same
root to rounding: the two compiled forms may fuse a candidate's arithmetic
differently) and against the oracle's recovery (the same root to 1e-10, or
no root and the same atmosphere reset).  Points: the magnetised blast-front states of
tests/golden on which the paper iteration and the 4D Newton stall, and the
same states with tau lowered until some have no root (seeded, fixed
factors)."""
import ctypes
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(__file__)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA is not available on a GPU test run")
    return torch


def _points():
    d = np.load(os.path.join(HERE, "golden", "recovery_hard_cases.npz"))
    cons, guess = [d["cons"]], [d["guess"]]
    # tau x 0.98 and above: a root; x 0.95 and below: none
    for f in (2.0, 1.1, 0.98, 0.97, 0.96, 0.95, 0.5, 0.1):
        c = d["cons"].copy()
        c[4] *= f        # tau
        cons.append(c)
        guess.append(d["guess"])
    return (np.ascontiguousarray(np.concatenate(cons, axis=1)),
            np.ascontiguousarray(np.concatenate(guess, axis=1)),
            float(d["c"]), float(d["sigma"]), float(d["gamma_eos"]))


def _run(torch, P, cons, guess, sigma, c, one_warp):
    import paper_2510_18968_b300 as R
    L = R.load()
    n = cons.shape[1]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    dc, dg, ds = dev(cons), dev(guess), dev(np.full(n, sigma))
    prim = torch.empty((14, n), dtype=torch.float64, device="cuda")
    status = torch.empty(n, dtype=torch.int32, device="cuda")
    rc = L.rmhd_test_bracket_points(ctypes.byref(P), n, ctypes.c_void_p(dc.data_ptr()),
                                    ctypes.c_void_p(dg.data_ptr()), ctypes.c_void_p(ds.data_ptr()),
                                    1, c, one_warp, ctypes.c_void_p(prim.data_ptr()),
                                    ctypes.c_void_p(status.data_ptr()), None)
    assert rc == 0
    torch.cuda.synchronize()
    return prim.cpu().numpy(), status.cpu().numpy()


def test_bracket_on_a_warp_makes_the_one_thread_decisions(torch_cuda):
    import paper_2510_18968_b300 as R
    torch = torch_cuda
    cons, guess, c, sigma, gam = _points()
    P = R.make_params(gamma_eos=gam)
    pw, sw = _run(torch, P, cons, guess, sigma, c, 1)
    pt, st = _run(torch, P, cons, guess, sigma, c, 0)
    assert np.array_equal(sw, st)
    scale = np.abs(pt).max(axis=1, keepdims=True) + 1e-300
    diff = (np.abs(pw - pt) / scale).max()
    print("warp vs thread: largest difference relative to the field's scale", diff)
    assert diff <= 1e-12, diff
    OP = oracle.make_params(gamma_eos=gam)
    outcomes = set()
    for i in range(cons.shape[1]):
        ref, _, _, so = oracle.con2prim(OP, cons[:, i], 1, c, sigma, guess[:, i])
        outcomes.add(so)
        if so in (0, 1, 4):
            # a root: the bracket finds it
            assert sw[i] == 4, (i, so, sw[i])
            assert np.allclose(pw[:, i], ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max()), i
        else:
            # no root (2) or density below the floor (3): the same reset
            assert sw[i] == so, (i, so, sw[i])
            assert np.allclose(pw[:, i], ref, rtol=1e-12, atol=1e-300), i
    # both kinds of point are present
    assert 4 in outcomes and 2 in outcomes, outcomes
