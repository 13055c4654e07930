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
    with pytest.raises(m.LbmError) as e:
        m.lbm_conservation_noalloc("D2Q9", "f32", f, 4097, 4096, 4097, out)
    assert e.value.code == m.EINVAL
