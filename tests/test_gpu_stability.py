"""Stability range of the double shear layer (Sec. III.B) on the GPU: the mean kinetic energy history that
decides stability matches the FP64 oracle step for step, the search's bracket is tight and reproducible,
and at Re = 1e4 the recursive regularization is more stable than the standard projection on D2Q9."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1704_04413_gb300 import stability as S
from paper_1704_04413_gb300 import workloads as wl

from gpu_util import lib

pytestmark = pytest.mark.gpu


def test_kinetic_energy_history_matches_oracle_through_the_divergence():
    """D2Q9 RR-4 (f^(0) at order 4), L = 128, Re = 1e5, M0 = 0.2: <u^2>(t) / <u^2>(0) every 100 steps, GPU
    FP64 against the oracle, until the run diverges; both cross the criterion at the same check."""
    m = lib()
    L, mach, re = 128, 0.2, 1e5
    V, cx, cy, w, cs2 = m.lbm_lattice_info("D2Q9")
    u0 = mach * math.sqrt(cs2)
    nu = u0 * L / re
    fl = wl.double_shear_layer(L, u0)
    ctx = m.lbm_create(m.make_params("D2Q9", L, L, nu=nu, collision="rr", hermite_order=4, reg_order=4, storage="f64"))
    p = orc.params("D2Q9", L, L, orc.tau_from_nu(cs2, nu), collision="rr", hermite_order=4, reg_order=4)
    try:
        m.lbm_init(ctx, fl.rho, fl.ux, fl.uy, None, fl.grad_u)
        f = orc.init(p, fl.rho, fl.ux, fl.uy, None, fl.grad_u)
        g0 = m.lbm_diagnostics(ctx)[0]
        o0 = orc.diagnostics(*orc.moments(p, f)[:3])[0]
        assert abs(g0 - o0) <= 1e-13 * o0
        cross_g = cross_o = None
        for t in range(100, S.steps_to(L, mach, math.sqrt(cs2)) + 1, 100):
            m.lbm_step(ctx, 100)
            f = orc.step(p, f, 100)
            g = m.lbm_diagnostics(ctx, raise_unstable=False)[0] / g0
            o = orc.diagnostics(*orc.moments(p, f)[:3])[0] / o0
            if cross_g is None and cross_o is None:
                assert abs(g - o) <= 1e-6, (t, g, o)  # until the divergence the two runs are the same run
            if cross_g is None and not g < 1.0:
                cross_g = t
            if cross_o is None and not o < 1.0:
                cross_o = t
            if cross_g is not None and cross_o is not None:
                break
        assert cross_g is not None and cross_o is not None and cross_g > 1000
        assert abs(cross_g - cross_o) <= 200
    finally:
        m.lbm_destroy(ctx)


def test_search_bracket_is_tight_and_reproducible():
    a, b = S.max_mach("D2Q9", "pr", [1e4], reg_order=2)[1e4]
    assert b is not None and 0.0 < a < b and b - a == pytest.approx(0.01)
    assert S.run_group("D2Q9", "pr", 2, 128, [(a, 1e4), (b, 1e4)]) == [True, False]


def test_recursive_regularization_extends_the_low_re_range_on_d2q9():
    out = S.stability_map(reynolds=(1e4,), lattices=("D2Q9",), variants=("pr2", "rr4"))["D2Q9"]
    assert out["rr4"][1e4][0] > out["pr2"][1e4][0] + 0.1


OPERATING_POINTS = [("D2Q9", 0.2, 4), ("D2V17", 0.35, 3), ("D2V37", 0.57, 4)]


@pytest.mark.parametrize("lattice,mach,nmax", OPERATING_POINTS)
def test_recursive_regularization_at_the_papers_re_3e4_operating_points(lattice, mach, nmax):
    """Sec. III.B runs the L = 128 double shear layer at Re = 3e4 with M0 = 0.2 (D2Q9), 0.35 (D2V17) and
    0.57 (D2V37) and finds the RR runs correct and more stable than PR.  RR with a1 from finite
    differences (Sec. II.E's second option) is stable up to 2 t_c at every order on every lattice; RR
    with the projected a1 is stable at every order on D2Q9 and D2V17 and diverges on D2V37 at this Mach
    number (its measured limit there is about 0.5, while PR's is about 0.73)."""
    fd = {n: S.run_group(lattice, "rr", n, 128, [(mach, 3e4)], a1_source=1)[0] for n in range(3, nmax + 1)}
    proj = {n: S.run_group(lattice, "rr", n, 128, [(mach, 3e4)])[0] for n in range(3, nmax + 1)}
    assert all(fd.values()), fd
    if lattice != "D2V37":
        assert all(proj.values()), proj
    else:
        assert not any(proj.values()), proj


def test_finite_difference_rr_outlasts_pr_at_high_reynolds_on_d2q9():
    """D2Q9, L = 128, M0 = 0.2 at Re = 1e5 and 1e6: standard PR-2 and RR with the projected a1 diverge
    before 2 t_c, RR-4 with a1 from finite differences stays stable (Sec. III.B's claim that RR extends
    the stable range over PR holds for this variant at every Reynolds number measured)."""
    for re in (1e5, 1e6):
        assert S.run_group("D2Q9", "rr", 4, 128, [(0.2, re)], a1_source=1) == [True]
        assert S.run_group("D2Q9", "pr", 2, 128, [(0.2, re)]) == [False]
        assert S.run_group("D2Q9", "rr", 4, 128, [(0.2, re)]) == [False]


def test_kinetic_energy_history_matches_oracle_at_re_3e4():
    """D2Q9 RR-4 at the Re = 3e4, M0 = 0.2 operating point, FP32 storage: <u^2>(t) / <u^2>(0) every 100
    steps for 600 steps, GPU against the FP64 oracle."""
    m = lib()
    L, mach, re = 128, 0.2, 3e4
    V, cx, cy, w, cs2 = m.lbm_lattice_info("D2Q9")
    u0 = mach * math.sqrt(cs2)
    nu = u0 * L / re
    fl = wl.double_shear_layer(L, u0)
    ctx = m.lbm_create(m.make_params("D2Q9", L, L, nu=nu, collision="rr", hermite_order=4, reg_order=4, storage="f32"))
    p = orc.params("D2Q9", L, L, orc.tau_from_nu(cs2, nu), collision="rr", hermite_order=4, reg_order=4)
    try:
        m.lbm_init(ctx, fl.rho, fl.ux, fl.uy, None, fl.grad_u)
        f = orc.init(p, fl.rho, fl.ux, fl.uy, None, fl.grad_u)
        g0 = m.lbm_diagnostics(ctx)[0]
        o0 = orc.diagnostics(*orc.moments(p, f)[:3])[0]
        for t in range(100, 601, 100):
            m.lbm_step(ctx, 100)
            f = orc.step(p, f, 100)
            g = m.lbm_diagnostics(ctx)[0] / g0
            o = orc.diagnostics(*orc.moments(p, f)[:3])[0] / o0
            assert abs(g - o) <= 1e-5, (t, g, o)
            assert g < 1.0
    finally:
        m.lbm_destroy(ctx)
