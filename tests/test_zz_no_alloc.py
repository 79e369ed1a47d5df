"""GPU test of rmhd_con2prim_points_noalloc, the recovery entry point that
allocates no device memory (for callers that size their device memory once
and may not allocate later, or cannot pay for cudaMalloc in a time-critical
loop).  It must give what rmhd_con2prim_points gives, call after call, while
its built-in work list is reused.  Kept in its own file, collected last."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _inputs(seed, n):
    from tests.test_gpu_parity import _random_recovery_inputs
    d = _random_recovery_inputs(n, seed, True, (1e-2, 1e5))
    # append the blast-front states on which the paper iteration fails, so
    # the work list is certainly used
    h = np.load(os.path.join(HERE, "golden", "recovery_hard_cases.npz"))
    k = h["cons"].shape[1]
    cin = np.concatenate([d["cin"], h["cons"]], axis=1)
    guess = np.concatenate([d["guess"], h["guess"]], axis=1)
    alpha = np.concatenate([d["alpha"], np.ones(k)])
    g6 = np.concatenate([d["g6"], np.tile(np.array([[1.0], [0], [0], [1], [0], [1]]), (1, k))],
                        axis=1)
    # the hard cases use sigma = 1e3 at c = gamma dt; express it through sigma
    sig_h = np.full(k, float(h["sigma"]) * float(h["c"]) / d["c"])
    sigma = np.concatenate([d["sigma"], sig_h])
    return cin, guess, alpha, g6, sigma, d["c"]


def test_noalloc_recovery_matches_the_allocating_entry_point():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    import paper_2510_18968_b300 as R

    P = dict(gamma_eos=4.0 / 3.0, rho_atmo=1e-14)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()

    def outputs(n):
        return (torch.empty((14, n), dtype=torch.float64, device="cuda"),
                torch.empty((14, n), dtype=torch.float64, device="cuda"),
                torch.empty(n, dtype=torch.int32, device="cuda"),
                torch.empty(n, dtype=torch.int32, device="cuda"))

    # a first call loads the kernels' code onto the device (the driver may
    # allocate for that); the device-memory check below starts after it
    cin, guess, alpha, g6, sigma, c = _inputs(500, 64)
    R.con2prim_points(P, dev(cin), dev(guess), dev(alpha), dev(g6), dev(sigma), 1, c,
                      out=outputs(alpha.size), noalloc=True)
    torch.cuda.synchronize()
    for call, seed in enumerate((501, 502)):
        cin, guess, alpha, g6, sigma, c = _inputs(seed, 4000)
        n = alpha.size
        args = (dev(cin), dev(guess), dev(alpha), dev(g6), dev(sigma), 1, c)
        ref = R.con2prim_points(P, *args)
        out = outputs(n)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        got = R.con2prim_points(P, *args, out=out, noalloc=True)
        torch.cuda.synchronize()
        # the call allocated no device memory (cudaMemGetInfo unchanged)
        assert torch.cuda.mem_get_info()[0] == free_before, call
        rp, rc, ri, rs = [x.cpu().numpy() for x in ref]
        gp, gc, gi, gs = [x.cpu().numpy() for x in got]
        assert (rs == 1).sum() + (rs == 4).sum() > 0, "no point used the work list"
        assert np.array_equal(gs, rs), call
        scale = np.abs(rp).max(axis=0) + 1e-300
        assert (np.abs(gp - rp) / scale).max() < 1e-12, call
        cscale = np.abs(rc).max(axis=0) + 1e-300
        assert (np.abs(gc - rc) / cscale).max() < 1e-12, call
        # iteration counts are telemetry; they agree where the paper
        # iteration converged in the first pass
        first = rs == 0
        assert np.array_equal(gi[first], ri[first]), call


def test_noalloc_rejects_more_points_than_its_work_list():
    torch = pytest.importorskip("torch")
    import paper_2510_18968_b300 as R

    L = R.load()
    n = 65536 + 1
    z = torch.zeros(14 * n, dtype=torch.float64, device="cuda")
    o = torch.zeros(14 * n, dtype=torch.float64, device="cuda")
    iz = torch.zeros(n, dtype=torch.int32, device="cuda")
    P = R.make_params()
    rc = L.rmhd_con2prim_points_noalloc(
        __import__("ctypes").byref(P), n, z.data_ptr(), z.data_ptr(), z.data_ptr(),
        z.data_ptr(), z.data_ptr(), 1, 0.1, o.data_ptr(), o.data_ptr(), iz.data_ptr(),
        iz.data_ptr(), None)
    assert rc == R.RMHD_EINVAL
    assert b"65536" in L.rmhd_last_error(None)
