"""Oracle: one relaxation time per Hermite order (Eq. GenRegCollision with tau_{n,alpha} -> tau_n, Sec. II.B),
pinned by what the kinetic theory fixes: equal times reduce to the single-time collision; the order-3 time
alone sets the thermal diffusivity, alpha = cs^2 (tau_3 - 1/2) (Pr = (tau_2 - 1/2) / (tau_3 - 1/2)),
measured from the decay of an isobaric temperature wave; the order-2 time alone sets the viscosity; mass,
momentum and energy stay conserved."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1704_04413_gb300 import workloads as wl


def cell(lat, thermal, seed):
    """One cell's populations: a perturbed equilibrium at random (rho, u, theta)."""
    rng = np.random.default_rng(seed)
    rho = np.array([[1.0 + 0.05 * rng.standard_normal()]])
    ux, uy = (np.array([[0.05 * rng.standard_normal()]]) for _ in range(2))
    th = np.array([[1.0 + 0.05 * rng.standard_normal()]]) if thermal else None
    p = orc.params(lat, 1, 1, 0.8, collision="rr", hermite_order=4 if lat != "D2V17" else 3, thermal=thermal)
    f = orc.init(p, rho, ux, uy, th)[:, 0, 0]
    return f * (1.0 + 0.02 * rng.uniform(-1, 1, size=f.size))


CASES = [("D2Q9", False), ("D2V17", False), ("D2V37", False), ("D2V37", True)]


@pytest.mark.parametrize("lat,thermal", CASES)
@pytest.mark.parametrize("coll", ["pr", "rr"])
def test_equal_times_reduce_to_the_single_time_collision(lat, thermal, coll):
    f = cell(lat, thermal, 1)
    ho = 4 if lat != "D2V17" else 3
    one = orc.collide(orc.params(lat, 1, 1, 0.7, collision=coll, hermite_order=ho, thermal=thermal), f)
    per = orc.collide(orc.params(lat, 1, 1, 0.7, collision=coll, hermite_order=ho, thermal=thermal, tau3=0.7,
                                 tau4=0.7), f)
    assert np.allclose(per, one, rtol=0, atol=1e-15)


@pytest.mark.parametrize("lat,thermal", CASES)
@pytest.mark.parametrize("coll", ["pr", "rr"])
def test_conservation_with_per_order_times(lat, thermal, coll):
    L = orc.lattice(lat)
    f = cell(lat, thermal, 2)
    ho = 4 if lat != "D2V17" else 3
    g = orc.collide(orc.params(lat, 1, 1, 0.7, collision=coll, hermite_order=ho, thermal=thermal, tau3=0.55,
                               tau4=1.3), f)
    cx, cy = np.array(L.cx, float), np.array(L.cy, float)
    for w in (np.ones_like(cx), cx, cy) + ((cx * cx + cy * cy,) if thermal else ()):
        assert abs(np.dot(w, g) - np.dot(w, f)) <= 1e-14 * max(1.0, abs(np.dot(w, f)))


def test_times_other_than_tau_change_the_collision_only_through_their_order():
    f = cell("D2V37", True, 3)
    base = orc.params("D2V37", 1, 1, 0.8, collision="pr", hermite_order=4, thermal=True)
    a = orc.collide(base, f)
    b = orc.collide(orc.params("D2V37", 1, 1, 0.8, collision="pr", hermite_order=4, thermal=True, tau4=1.2), f)
    # the difference is a pure fourth-order Hermite component: its moments of order <= 3 vanish
    L = orc.lattice("D2V37")
    cx, cy = np.array(L.cx, float), np.array(L.cy, float)
    d = b - a
    assert np.abs(d).max() > 1e-6
    for k in range(4):
        for l in range(4 - k):
            assert abs(np.dot(cx ** k * cy ** l, d)) < 1e-14


def test_bgk_rejects_per_order_times():
    f = cell("D2Q9", False, 4)
    with pytest.raises(ValueError):
        orc.collide(orc.params("D2Q9", 1, 1, 0.8, collision="bgk", tau3=0.9), f)


def wave_rate(coll, tau2, tau3, nx=64, steps=600):
    """Decay rate of the isobaric temperature wave theta = 1 + 0.01 sin(k x), rho theta = 1, u = 0, on thermal
    D2V37, fitted to log |amplitude| over t in [100, steps]."""
    k = 2 * np.pi / nx
    x = np.arange(nx) + 0.5
    th = np.tile(1 + 0.01 * np.sin(k * x), (2, 1))
    p = orc.params("D2V37", nx, 2, tau2, collision=coll, hermite_order=4, thermal=True, tau3=tau3)
    f = orc.init(p, 1.0 / th, np.zeros_like(th), np.zeros_like(th), th)
    ts, amps = [], []
    for t in range(0, steps + 1, 20):
        if t:
            f = orc.step(p, f, 20)
        T = orc.moments(p, f)[3]
        ts.append(t)
        amps.append(2 * np.mean((T - T.mean()) * np.sin(k * x)[None, :]))
    ts, amps = np.array(ts), np.array(amps)
    sel = ts >= 100
    return -np.polyfit(ts[sel], np.log(amps[sel]), 1)[0], k


@pytest.mark.parametrize("coll", ["pr", "rr"])
@pytest.mark.parametrize("tau3", [0.6, 1.0])
def test_temperature_wave_decays_with_the_order3_time(coll, tau3):
    cs2 = orc.lattice("D2V37").cs2
    rate, k = wave_rate(coll, 0.8, tau3)
    assert rate == pytest.approx(cs2 * (tau3 - 0.5) * k * k, rel=0.02)


def test_shear_wave_decay_ignores_the_order3_time():
    """Thermal D2V37 RR shear wave: the decay rate is nu k^2 with nu = cs^2 (tau_2 - 1/2) whatever tau_3 (the
    two rates agree to 1 %, where the same two tau_3 change the temperature wave's rate 3-fold)."""
    cs2 = orc.lattice("D2V37").cs2
    nx, ny, tau2 = 2, 64, 0.8
    fl = wl.shear_wave(nx, ny, 1e-3)
    rates = []
    for tau3 in (0.6, 1.2):
        p = orc.params("D2V37", nx, ny, tau2, collision="rr", hermite_order=4, thermal=True, tau3=tau3)
        f = orc.init(p, fl.rho, fl.ux, fl.uy, np.ones_like(fl.rho), fl.grad_u)
        a0 = np.abs(orc.moments(p, f)[1]).max()
        f = orc.step(p, f, 400)
        rates.append(np.log(a0 / np.abs(orc.moments(p, f)[1]).max()) / 400)
    k = 2 * np.pi / ny
    assert rates[0] == pytest.approx(rates[1], rel=1e-2)
    assert rates[0] == pytest.approx(cs2 * (tau2 - 0.5) * k * k, rel=0.03)
