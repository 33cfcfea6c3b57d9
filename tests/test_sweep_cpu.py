"""Host-side pieces of the sweep driver: the saturated liquid's c_p used to
turn the paper's Jakob numbers into wall superheats, checked against the FP64
oracle's equation of state (its dp/drho and T dp/dT at the Maxwell liquid
density) and against a finite-difference c_p of the oracle's pressure."""
import numpy as np
import pytest


def test_liquid_cp_matches_the_oracle_eos():
    from oracle import eos
    from paper_1812_10375_gb300 import build, hlb, sweep
    build.build()
    p = hlb.default_params(8, 8)
    cp = sweep.liquid_cp(p)
    pr = eos.PR()
    T = 0.86 * pr.Tc
    rl, rv, _ = eos.coexistence(T, pr)
    tdpdt = eos.T_dp_dT(rl, T, pr)
    ref = p.cv + tdpdt ** 2 / (T * rl ** 2 * eos.dp_drho(rl, T, pr))
    assert cp == pytest.approx(ref, rel=1e-9)
    # the same thermodynamic identity with both derivatives taken by central
    # differences of the oracle's pressure (Eq. 28)
    h = 1e-6 * T
    dpdT = (eos.pressure(rl, T + h, pr) - eos.pressure(rl, T - h, pr)) / (2 * h)
    d = 1e-6 * rl
    dpdr = (eos.pressure(rl + d, T, pr) - eos.pressure(rl - d, T, pr)) / (2 * d)
    assert cp == pytest.approx(p.cv + T * dpdT ** 2 / (rl ** 2 * dpdr), rel=1e-6)
    assert 2.0 * p.cv < cp < 3.0 * p.cv
