"""Helpers of the GPU tests: contexts on cuda:0 through the C ABI, the
velocity-order permutation between the library and the oracle, and error norms."""
import numpy as np

from oracle import oracle as orc


def lib():
    from paper_1704_04413_gb300 import lbm
    lbm.load()
    return lbm


def stream():
    import torch
    torch.cuda.set_device(0)
    return torch.cuda.current_stream().cuda_stream


def perm(name):
    """Index array P with f_lib = f_oracle[P] (matched by velocity vector)."""
    V, cx, cy, _, _ = lib().lbm_lattice_info(name)
    L = orc.lattice(name)
    idx = {(int(a), int(b)): k for k, (a, b) in enumerate(zip(L.cx, L.cy))}
    return np.array([idx[(int(a), int(b))] for a, b in zip(cx, cy)])


class Ctx:
    """A library context; closes on exit."""

    def __init__(self, name, nx, ny, tau, coll="rr", neq=2, nreg=0, storage="f32", thermal=False,
                 bcx=0, bcy=0, rho0=0.0, scale=0.0, tau3=0.0, tau4=0.0, a1_source=0):
        m = lib()
        self.m = m
        self.name, self.nx, self.ny = name, nx, ny
        self.V = m.lbm_lattice_info(name)[0]
        self.P = perm(name)
        p = m.make_params(name, nx, ny, tau=tau, collision=coll, hermite_order=neq, reg_order=nreg,
                          thermal=thermal, bc_x=bcx, bc_y=bcy, storage=storage, rho0=rho0, store_scale=scale,
                          stream=stream(), tau3=tau3, tau4=tau4, a1_source=a1_source)
        self.ctx = m.lbm_create(p)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.m.lbm_destroy(self.ctx)

    def set_oracle_f(self, f_orc):
        self.m.lbm_set_populations(self.ctx, np.ascontiguousarray(f_orc[self.P]))

    def get_oracle_f(self):
        g = np.empty((self.V, self.ny, self.nx))
        self.m.lbm_get_populations(self.ctx, g)
        out = np.empty_like(g)
        out[self.P] = g
        return out

    def init(self, fl, theta=None, grad=True):
        self.m.lbm_init(self.ctx, fl.rho, fl.ux, fl.uy, theta, fl.grad_u if grad else None)

    def step(self, n=1):
        self.m.lbm_step(self.ctx, n)

    def moments(self):
        a = [np.empty((self.ny, self.nx)) for _ in range(4)]
        self.m.lbm_moments(self.ctx, *a)
        return a


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def pop_rel(got, ref, w):
    """Per-population error of one collision, relative to the population's own magnitude or to its
    equilibrium scale w_i (lattice weight at unit density), whichever is larger.  A population the
    collision drives close to zero keeps the absolute resolution of its natural scale."""
    w = np.asarray(w).reshape((-1,) + (1,) * (np.ndim(ref) - 1))
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), w)))


def stored(f, storage):
    """The populations a context holds after lbm_set_populations of FP64 values f: rounded to FP32 for FP32
    storage.  One collision is compared from that input, so the per-collision bound measures the
    collision's arithmetic; the FP32 representation of the input is a storage effect (alone it moves
    D2V17 PR-3's fast populations by up to 2.4e-6 relative through the third-order projection)."""
    return f.astype(np.float32).astype(np.float64) if storage == "f32" else f


def coll_errors(got, ref, w):
    """(pop_rel, plain relative error max |got - ref| / |ref| over the populations with |ref| >= w_i / 10).
    The second is the per-collision bound read literally, where it is well defined; the first extends it
    to populations the collision drives toward zero (whose absolute FP32 resolution is that of w_i)."""
    w = np.asarray(w).reshape((-1,) + (1,) * (np.ndim(ref) - 1))
    big = np.abs(ref) >= np.broadcast_to(w, ref.shape) / 10.0
    e_big = float(np.max(np.abs(got - ref)[big] / np.abs(ref)[big])) if big.any() else 0.0
    return pop_rel(got, ref, w), e_big


def assert_coll(got, ref, w, tol, tol_big=None):
    """Per-collision parity at `tol`: relative to max(|f_i|, w_i) everywhere, and relative to |f_i| itself
    on every population with |f_i| >= w_i / 10 (at tol_big where a mode's FP32 evaluation is known to need
    more; default tol)."""
    tol_big = tol if tol_big is None else tol_big
    e_pop, e_big = coll_errors(got, ref, w)
    assert e_pop <= tol and e_big <= tol_big, "pop_rel %.3e, max_rel(|f| >= w/10) %.3e, tol %.1e / %.1e" % (
        e_pop, e_big, tol, tol_big)
