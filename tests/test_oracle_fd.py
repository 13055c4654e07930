"""Oracle: a1 by finite differences (Sec. II.E: a1^(2), a1^(3) "by projection ... or using finite
differences"), pinned by: on a Chapman-Enskog state built from given gradients the finite-difference
collision with the same gradients equals the projection collision (same prefactor, sign and tau); the
whole scheme still decays a shear wave at nu k^2 and an isobaric temperature wave at alpha k^2, with
second-order convergence in the grid spacing; the option is refused outside RR."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1704_04413_gb300 import workloads as wl


@pytest.mark.parametrize("lat,ho", [("D2Q9", 2), ("D2Q9", 4), ("D2V17", 3), ("D2V37", 4)])
def test_fd_equals_projection_on_a_chapman_enskog_state(lat, ho):
    rng = np.random.default_rng(3)
    g = rng.normal(0, 0.02, 4)  # d ux/dx, d ux/dy, d uy/dx, d uy/dy
    rho, ux, uy = (np.array([[v]]) for v in (1.02, 0.04, -0.03))
    grad = g.reshape(4, 1, 1)
    tau = 0.7
    pp = orc.params(lat, 1, 1, tau, collision="rr", hermite_order=ho)
    f = orc.init(pp, rho, ux, uy, None, grad)[:, 0, 0]  # f^(0) + f^(1) with a1^(2) = -tau rho cs^2 S
    proj = orc.collide(pp, f)
    fd = orc.collide_fd(orc.params(lat, 1, 1, tau, collision="rr", hermite_order=ho, a1_source=1), f,
                        np.concatenate([g, [0.0, 0.0]]))
    assert np.allclose(fd, proj, rtol=0, atol=1e-15)


def test_fd_thermal_without_temperature_gradient_equals_projection_at_rest():
    """Thermal D2V37 with u = 0 and a uniform temperature: the projected and the finite-difference a1^(3)
    estimates both carry no temperature-gradient term."""
    g = np.array([0.01, -0.02, 0.015, -0.005])
    rho, z, th = np.array([[0.98]]), np.array([[0.0]]), np.array([[1.04]])
    pp = orc.params("D2V37", 1, 1, 0.7, collision="rr", hermite_order=4, thermal=True)
    f = orc.init(pp, rho, z, z, th, g.reshape(4, 1, 1))[:, 0, 0]
    proj = orc.collide(pp, f)
    fd = orc.collide_fd(orc.params("D2V37", 1, 1, 0.7, collision="rr", hermite_order=4, thermal=True, a1_source=1),
                        f, np.concatenate([g, [0.0, 0.0]]))
    assert np.allclose(fd, proj, rtol=0, atol=1e-14)


def shear_rate(lat, ho, ny, src, tau=0.8):
    cs2 = orc.lattice(lat).cs2
    fl = wl.shear_wave(2, ny, 1e-3)
    k = 2 * np.pi / ny
    p = orc.params(lat, 2, ny, tau, collision="rr", hermite_order=ho, a1_source=src)
    f = orc.init(p, fl.rho, fl.ux, fl.uy, None, fl.grad_u)
    a0 = np.abs(orc.moments(p, f)[1]).max()
    n = int(0.5 / (cs2 * (tau - 0.5) * k * k))
    f = orc.step(p, f, n)
    return np.log(a0 / np.abs(orc.moments(p, f)[1]).max()) / n / (cs2 * (tau - 0.5) * k * k)


@pytest.mark.parametrize("lat,ho", [("D2Q9", 2), ("D2V17", 3), ("D2V37", 4)])
def test_fd_shear_wave_decay_converges_at_second_order(lat, ho):
    e32, e64 = abs(shear_rate(lat, ho, 32, 1) - 1), abs(shear_rate(lat, ho, 64, 1) - 1)
    assert e32 < 0.07 and e64 < 0.02
    assert 3.0 < e32 / e64 < 5.0


def temp_rate(nx, tau3):
    cs2 = orc.lattice("D2V37").cs2
    k = 2 * np.pi / nx
    x = np.arange(nx) + 0.5
    th = np.tile(1 + 0.01 * np.sin(k * x), (2, 1))
    p = orc.params("D2V37", nx, 2, 0.8, collision="rr", hermite_order=4, thermal=True, tau3=tau3, a1_source=1)
    f = orc.init(p, 1 / th, 0 * th, 0 * th, th)
    ts, amps = [], []
    for t in range(0, 601, 20):
        if t:
            f = orc.step(p, f, 20)
        T = orc.moments(p, f)[3]
        ts.append(t)
        amps.append(2 * np.mean((T - T.mean()) * np.sin(k * x)[None, :]))
    ts, amps = np.array(ts), np.array(amps)
    return -np.polyfit(ts[ts >= 100], np.log(amps[ts >= 100]), 1)[0] / (cs2 * (tau3 - 0.5) * k * k)


def test_fd_temperature_wave_decays_with_the_heat_conductivity():
    e32, e64 = abs(temp_rate(32, 0.6) - 1), abs(temp_rate(64, 0.6) - 1)
    assert e64 < 0.025 and 3.0 < e32 / e64 < 5.0
    assert temp_rate(64, 1.0) == pytest.approx(1.0, abs=0.01)


def test_fd_option_is_rr_only():
    f = np.full(9, 1.0 / 9)
    with pytest.raises(ValueError):
        orc.collide(orc.params("D2Q9", 1, 1, 0.8, collision="rr", a1_source=1), f)  # needs gradients
    with pytest.raises(ValueError):
        orc.collide_fd(orc.params("D2Q9", 1, 1, 0.8, collision="pr", a1_source=1), f, np.zeros(6))
    with pytest.raises(ValueError):
        orc.step(orc.params("D2Q9", 4, 4, 0.8, collision="bgk", a1_source=1), np.ones((9, 4, 4)) / 9)
