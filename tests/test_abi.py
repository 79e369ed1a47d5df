"""CPU checks of the C ABI library: it loads, exports every function that
include/rmhd.h declares, its parameter struct matches the binding, and
argument checking happens before any device work."""
import ctypes
import os
import re

import pytest

import paper_2510_18968_b300 as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rmhd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rmhd_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    L = R.load()
    names = _declared()
    assert "rmhd_step" in names and "rmhd_create" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(R.EXPORTS) | set(names)


def test_param_struct_size_matches():
    L = R.load()
    size = ctypes.sizeof(R.Params)
    buf = (ctypes.c_ubyte * (size + 64))(*([0xAB] * (size + 64)))
    L.rmhd_default_params(ctypes.cast(buf, ctypes.POINTER(R.Params)))
    assert all(b == 0xAB for b in bytes(buf)[size:]), "C struct larger than the binding's"
    p = R.make_params()
    assert tuple(p.n) == (1, 1, 1) and p.gamma_eos == 2.0 and p.c2p_tol == 1e-14
    assert p.imex == 0


@pytest.mark.parametrize("bad", [dict(n=(0, 1, 1)), dict(dx=(0.0, 1, 1)), dict(gamma_eos=1.0),
                                 dict(recon=7), dict(sigma0=-1.0), dict(bc=(5, 0, 0)),
                                 dict(precision=3), dict(qflux_mode=9), dict(c2p_tol=0.0),
                                 dict(n=(2, 1, 1), bc=(0, 0, 0)),
                                 # padded cells beyond 2^31 (the 32-bit index limit)
                                 dict(n=(1300, 1300, 1300)), dict(sigma_model=4),
                                 dict(c2p_maxit=0), dict(c2p_wmax=1.0),
                                 dict(c2p_first_pass=-1), dict(n=(-4, 1, 1)),
                                 dict(imex=4), dict(imex=-1)])
def test_create_rejects_bad_params_without_touching_the_device(bad):
    with pytest.raises(R.RMHDError) as e:
        R.Solver(R.make_params(**bad))
    assert e.value.code == R.RMHD_EINVAL
