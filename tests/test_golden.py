"""Worked-example values printed in the paper (tests/golden/paper_values.txt)
against the input generators' closed forms."""
import os

import pytest

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_values.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, val, tol = line.split()[:3]
            out[name] = (float(val), float(tol))
    return out


G = _golden()


def _check(name, got):
    val, tol = G[name]
    assert abs(got - val) <= tol * abs(val), (name, got, val)


def test_alfven_speed_worked_example():
    _check("alfven_vA_worked_example", W.alfven_speed(1.0, 1.0, 2.0, 1.1547, 1.0))


def test_tov_pressures():
    K, rho_c = 100.0, 1.28e-3
    p_max = K * rho_c ** 2                # polytrope p = K rho^Gamma, Gamma = 2
    _check("tov_P_max", p_max)
    _check("tov_P_cut", 0.04 * p_max)     # the generator's cut-off fraction
    _check("tov_beta", 2.0 * p_max / 4.3e-8 ** 2)


def test_star_generator_field_normalisation():
    import numpy as np
    wl = W.lane_emden_star(n=16)
    B = wl.prim[8:11]
    assert abs(np.sqrt((B * B).sum(axis=0)).max() - 1e-3) < 1e-15
