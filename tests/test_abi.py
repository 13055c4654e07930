"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/lbm.h declares, describes the lattices of Tab. I like
the oracle does, and rejects invalid parameters before touching the device."""
import os
import re

import numpy as np
import pytest

from oracle import oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbm():
    from paper_1704_04413_gb300 import build as b
    b.build()
    from paper_1704_04413_gb300 import lbm as m
    m.load()
    return m


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(lbm3?_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lbm):
    lib = lbm.load()
    decl = declared_functions()
    assert decl, "no declarations found"
    for name in decl:
        assert hasattr(lib, name), name
    assert set(lbm.EXPORTED) <= decl
    assert set(lbm.EXPORTED3) <= decl


@pytest.mark.parametrize("name", ["D2Q9", "D2V17", "D2V37"])
def test_lattice_info_matches_oracle(lbm, name):
    V, cx, cy, w, cs2 = lbm.lbm_lattice_info(name)
    L = orc.lattice(name)
    assert V == L.V
    assert abs(cs2 - L.cs2) < 1e-15 * L.cs2 * 10
    lib = {(a, b): ww for a, b, ww in zip(cx, cy, w)}
    ora = {(a, b): ww for a, b, ww in zip(L.cx, L.cy, L.w)}
    assert set(lib) == set(ora)
    for k in lib:
        assert abs(lib[k] - ora[k]) < 1e-16


def test_invalid_parameters_are_rejected_on_host(lbm):
    bad = [
        dict(lattice="D2Q9", hermite_order=5),
        dict(lattice="D2V17", hermite_order=4),
        dict(lattice="D2Q9", reg_order=1),
        dict(lattice="D2Q9", thermal=True),
        dict(lattice="D2Q9", tau=0.5),
        dict(lattice="D2Q9", tau=0.0, nu=-1.0),
        dict(lattice="D2Q9", nx=0),
        dict(lattice="D2Q9", store_scale=3.0, storage="f16"),
        dict(lattice="D2Q9", bc_x=7),
        dict(lattice="D2Q9", tau3=0.5),                    # per-order time must exceed 1/2
        dict(lattice="D2Q9", tau4=-1.0),
        dict(lattice="D2Q9", collision="bgk", tau3=0.9),   # one time per order needs PR or RR
        dict(lattice="D2Q9", collision="pr", a1_source=1),  # finite-difference a1 is an RR option
        dict(lattice="D2Q9", a1_source=2),
    ]
    for kw in bad:
        kw.setdefault("tau", 0.8)
        p = lbm.make_params(**kw)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create(p)
        assert e.value.code == lbm.EINVAL, kw
    p = lbm.make_params("D2Q9", tau=0.8)
    p.compute = lbm.F64  # F64 compute with F32 storage is not a supported pair
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create(p)


def test_strerror(lbm):
    assert lbm.lbm_strerror(lbm.EINVAL) == "invalid argument"
    assert lbm.lbm_strerror(-99) == "unknown status"


def test_batch_rejects_invalid_sets_on_host(lbm):
    base = lbm.make_params("D2Q9", 32, 32, tau=0.7, storage="f16")
    other = lbm.make_params("D2V17", 32, 32, tau=0.7, storage="f32")  # different storage
    with pytest.raises(lbm.LbmError):
        lbm.lbm_batch_create([base, other])
    with pytest.raises(lbm.LbmError):
        lbm.lbm_batch_create([lbm.make_params("D2V37", 32, 32, tau=0.7, hermite_order=4, storage="f16")])
    with pytest.raises(lbm.LbmError):
        lbm.lbm_batch_create([base] * 65)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_batch_create([lbm.make_params("D2Q9", 32, 32, tau=0.7, storage="f64")])
    with pytest.raises(lbm.LbmError):
        lbm.lbm_batch_create([lbm.make_params("D2Q9", 32, 32, tau=0.7, storage="f16", a1_source=1)])


@pytest.mark.parametrize("name", ["D3Q19", "D3Q27", "D3V39", "D3Q103"])
def test_3d_lattice_info_matches_oracle(lbm, name):
    from oracle import lbm3d
    V, cx, cy, cz, w, cs2 = lbm.lbm3_lattice_info(name)
    L = lbm3d.lattice(name)
    assert V == L.V and abs(cs2 - L.cs2) < 1e-15
    lib = {(a, b, c): ww for a, b, c, ww in zip(cx, cy, cz, w)}
    ora = {tuple(int(v) for v in xi): ww for xi, ww in zip(L.xi, L.w)}
    assert set(lib) == set(ora)
    for k in lib:
        assert abs(lib[k] - ora[k]) < 1e-16


def test_3d_invalid_parameters_are_rejected_on_host(lbm):
    bad = [dict(lattice="D3Q19", hermite_order=4), dict(lattice="D3Q27", reg_order=7),
           dict(lattice="D3Q19", tau=0.5), dict(lattice="D3Q19", nz=0), dict(lattice="D3Q19", bc=(0, 0, 3)),
           dict(lattice="D3Q103", storage=9), dict(lattice=42)]
    for kw in bad:
        kw.setdefault("tau", 0.8)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm3_create(lbm.make_params3(**kw))
        assert e.value.code == lbm.EINVAL, kw
