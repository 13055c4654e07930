"""The allocation-free conservation sums (lbm_conservation_noalloc) against lbm_conservation.

That entry point serves callers that cannot allocate device memory when they
need the sums (their device memory belongs to another allocator, or their loop
forbids allocation): it takes caller-owned device buffers and keeps its scratch
in a static device array.  This file is collected last so that a failure here
comes after every other test has run.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1704_04413_gb300 import workloads as wl

from gpu_util import Ctx, lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,storage", [("D2Q9", "f64"), ("D2V37", "f32"), ("D2V17", "f32")])
def test_noalloc_sums_match_context_sums_on_two_calls(name, storage):
    import torch
    m = lib()
    nx, ny = 300, 77
    Lt = orc.lattice(name)
    u0, nu, _ = wl.shear_layer_params(nx, np.sqrt(Lt.cs2), 0.1, 3e4)
    fl = wl.double_shear_layer(nx, u0, ny=ny)
    neq = {"D2Q9": 2, "D2V17": 3, "D2V37": 4}[name]
    stream = torch.cuda.current_stream()
    with Ctx(name, nx, ny, orc.tau_from_nu(Lt.cs2, nu), "rr", neq, 0, storage) as c:
        c.init(fl)
        out = torch.zeros(4, dtype=torch.float64, device="cuda")
        for call in range(2):  # two calls in a row, state advanced in between
            c.step(7)
            ref = m.lbm_conservation(c.ctx)
            f64 = torch.empty((c.V, ny, nx), dtype=torch.float64, device="cuda")
            m.lbm_get_populations(c.ctx, f64)  # decoded populations, exact for f64 and f32 storage
            f = f64 if storage == "f64" else f64.to(torch.float32)
            out.fill_(float("nan"))
            m.lbm_conservation_noalloc(name, storage, f, nx, ny, nx, out, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got)), call
            assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)) <= 1e-12, (call, got, ref)


def test_noalloc_rejects_grids_beyond_its_static_scratch():
    import torch
    m = lib()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    f = torch.zeros(16, dtype=torch.float32, device="cuda")
    # raw addresses: the binding passes them through and the library refuses the size before any launch
    with pytest.raises(m.LbmError) as e:
        m.lbm_conservation_noalloc("D2Q9", "f32", f.data_ptr(), 4097, 4096, 4097, out.data_ptr())
    assert e.value.code == m.EINVAL


@pytest.mark.parametrize("name,storage", [("D2Q9", "f16"), ("D2V17", "bf16"), ("D2V37", "i16"), ("D2V37", "f16")])
def test_noalloc_shifted_storage_sums_on_two_calls(name, storage):
    """Shifted 16-bit storage (the only formats that use rho0 and the scale): stored values
    g_i = s (f_i / w_i - rho0) written on the host with a non-unit rho0 and s, decoded sums
    f_i = w_i (rho0 + g_i / s) added in FP64 on the host as the expected value, two calls in a row
    on different data, rows padded (pitch > nx)."""
    import torch
    m = lib()
    V, cx, cy, w, _ = m.lbm_lattice_info(name)
    nx, ny, pitch, rho0, s = 203, 41, 208, 1.25, 4.0
    stream = torch.cuda.current_stream()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(7)
    for call in range(2):
        g = rng.uniform(-0.9, 0.9, size=(V, ny, pitch))
        if storage == "i16":
            q = np.round(g * 32768.0).astype(np.int16)
            gv = q.astype(np.float64) / 32768.0
            dev = torch.from_numpy(q).cuda()
        else:
            tdt = torch.float16 if storage == "f16" else torch.bfloat16
            t = torch.from_numpy(g).to(tdt)
            gv = t.to(torch.float64).numpy()
            dev = t.cuda()
        fdec = np.asarray(w)[:, None, None] * (rho0 + gv[:, :, :nx] / s)
        c = [np.ones(V), np.asarray(cx, float), np.asarray(cy, float),
             0.5 * (np.asarray(cx, float) ** 2 + np.asarray(cy, float) ** 2)]
        terms = [ck[:, None, None] * fdec for ck in c]
        ref = np.array([t_.sum() for t_ in terms])
        scale = np.array([np.abs(t_).sum() for t_ in terms])
        out.fill_(float("nan"))
        m.lbm_conservation_noalloc(name, storage, dev, nx, ny, pitch, out, rho0=rho0, store_scale=s,
                                   stream=stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), (call, got, ref)


def test_noalloc_rejects_bad_scale_and_host_buffers():
    """A scale that is not a power of two, and host buffers passed as raw addresses, return LBM_EINVAL
    before any launch; mismatched tensors are refused by the binding.  Every buffer here is large enough
    for the call, so nothing would be read out of bounds even if a check were missing."""
    import torch
    m = lib()
    nx, ny = 16, 8
    V = m.lbm_lattice_info("D2Q9")[0]
    f = torch.zeros(V * ny * nx, dtype=torch.float16, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(m.LbmError) as e:
        m.lbm_conservation_noalloc("D2Q9", "f16", f, nx, ny, nx, out, store_scale=3.0)
    assert e.value.code == m.EINVAL
    fh = torch.zeros(V * ny * nx, dtype=torch.float16).pin_memory()
    oh = torch.zeros(4, dtype=torch.float64).pin_memory()
    with pytest.raises(m.LbmError) as e:
        m.lbm_conservation_noalloc("D2Q9", "f16", fh.data_ptr(), nx, ny, nx, out.data_ptr())
    assert e.value.code == m.EINVAL
    with pytest.raises(m.LbmError) as e:
        m.lbm_conservation_noalloc("D2Q9", "f16", f.data_ptr(), nx, ny, nx, oh.data_ptr())
    assert e.value.code == m.EINVAL
    with pytest.raises(TypeError):
        m.lbm_conservation_noalloc("D2Q9", "f32", f, nx, ny, nx, out)  # 2-byte elements for FP32 storage
    with pytest.raises(ValueError):
        m.lbm_conservation_noalloc("D2Q9", "f16", f, nx, ny + 1, nx, out)  # buffer shorter than V ny pitch
    with pytest.raises(TypeError):
        m.lbm_conservation_noalloc("D2Q9", "f16", f, nx, ny, nx, out.to(torch.float32))
    with pytest.raises(TypeError):
        m.lbm_conservation_noalloc("D2Q9", "f16", f.cpu(), nx, ny, nx, out)
