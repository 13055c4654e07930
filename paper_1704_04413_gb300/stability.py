"""Stability range of the double shear layer (Sec. III.B): the largest Mach number M0 = u0 / cs for which a
simulation on an L x L grid stays stable up to t = 2 t_c (t_c = L / u0), for Reynolds numbers in
[1e4, 1e6].  A run counts as stable when the mean kinetic energy never exceeds its initial value,
<u^2>(t) < <u^2>(0) for t <= 2 t_c, and as unstable when it does or a value stops being finite.  M0^max is
resolved to dm = 0.01.

The search brackets M0^max for every Reynolds number at once: each round runs `points` Mach numbers inside
every current bracket as independent instances (one batched launch per step on D2Q9 / D2V17, one context
per instance on D2V37), checks <u^2> every `check` steps through lbm_diagnostics, and keeps, per Reynolds
number, the largest stable M0 below the smallest unstable one.  The equilibrium is expanded to the
lattice's maximal order (4 on D2Q9, 3 on D2V17, 4 on D2V37) as in Sec. III.B.  Every step runs in the
library's kernels; this module only schedules runs and reads the FP64 diagnostics.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import lbm
from . import workloads as wl

MAX_ORDER = {"D2Q9": 4, "D2V17": 3, "D2V37": 4}


def steps_to(L: int, mach: float, cs: float, convective_times: float = 2.0) -> int:
    """Steps of `convective_times` t_c = L / (M0 cs)."""
    return int(math.ceil(convective_times * L / (mach * cs)))


class _Group:
    """Independent shear-layer instances stepped together: a batch where the lattice allows, else a list of
    contexts advanced one after the other on the same stream."""

    def __init__(self, lattice, collision, reg_order, L, machs_res, storage, stream, a1_source=0):
        V, cx, cy, w, cs2 = lbm.lbm_lattice_info(lattice)
        self.cs = math.sqrt(cs2)
        self.params, fields = [], []
        for mach, re in machs_res:
            u0 = mach * self.cs
            nu = u0 * L / re
            self.params.append(lbm.make_params(lattice, L, L, nu=nu, collision=collision,
                                               hermite_order=MAX_ORDER[lattice], reg_order=reg_order,
                                               storage=storage, stream=stream, a1_source=a1_source))
            fields.append(wl.double_shear_layer(L, u0))
        self.batch = None
        if lattice in ("D2Q9", "D2V17") and storage != "f64" and a1_source == 0:
            self.batch = lbm.lbm_batch_create(self.params)
            self.ctxs = [lbm.lbm_batch_context(self.batch, i) for i in range(len(self.params))]
        else:
            self.ctxs = [lbm.lbm_create(p) for p in self.params]
        for c, fl in zip(self.ctxs, fields):
            lbm.lbm_init(c, fl.rho, fl.ux, fl.uy, None, fl.grad_u)

    def step(self, n):
        if self.batch is not None:
            lbm.lbm_batch_step(self.batch, n)
        else:
            for c in self.ctxs:
                lbm.lbm_step(c, n)

    def close(self):
        if self.batch is not None:
            lbm.lbm_batch_destroy(self.batch)
        else:
            for c in self.ctxs:
                lbm.lbm_destroy(c)


def _mean_u2(ctx):
    d = lbm.lbm_diagnostics(ctx, raise_unstable=False)
    return float(d[0]) if np.isfinite(d).all() else math.inf


def run_group(lattice, collision, reg_order, L, machs_res, storage="f32", check=20, stream=None, a1_source=0):
    """Stability verdicts of instances (M0, Re): True when <u^2> stays below its initial value up to 2 t_c.
    a1_source = 1: RR with a1 from finite differences of the fields (Sec. II.E) instead of the projection."""
    g = _Group(lattice, collision, reg_order, L, machs_res, storage, stream, a1_source)
    try:
        ends = [steps_to(L, m, g.cs) for m, _ in machs_res]
        e0 = [_mean_u2(c) for c in g.ctxs]
        stable = [True] * len(g.ctxs)
        active = list(range(len(g.ctxs)))
        t = 0
        while active:
            n = min([check] + [ends[i] - t for i in active])
            g.step(n)
            t += n
            still = []
            for i in active:
                if _mean_u2(g.ctxs[i]) >= e0[i]:
                    stable[i] = False
                elif t < ends[i]:
                    still.append(i)
            active = still
        return stable
    finally:
        g.close()


def max_mach(lattice, collision, reynolds, reg_order=0, L=128, lo=0.0, hi=1.5, dm=0.01, points=None,
             storage="f32", check=20, stream=None, max_instances=64, a1_source=0):
    """M0^max per Reynolds number: dict Re -> (largest stable M0 below the smallest unstable one, smallest
    unstable M0), to dm.  0.0 as the first value means no tested Mach number was stable; None as the second
    means every tested one was."""
    reynolds = list(reynolds)
    if points is None:
        points = max(2, min(15, max_instances // max(1, len(reynolds)) - 1))
    tried = {re: {} for re in reynolds}  # M0 -> verdict

    def bracket(re):
        unstable = [m for m, ok in tried[re].items() if not ok]
        b = min(unstable + [hi])
        a = max([m for m, ok in tried[re].items() if ok and m < b] + [lo])
        return a, b

    while True:
        jobs = []
        for re in reynolds:
            a, b = bracket(re)
            if b - a <= dm + 1e-9:
                continue
            cand = {round(round((a + (b - a) * k / (points + 1)) / dm) * dm, 6) for k in range(1, points + 1)}
            jobs += [(m, re) for m in sorted(cand) if a < m < b and m not in tried[re]]
        if not jobs:
            break
        for k in range(0, len(jobs), max_instances):
            chunk = jobs[k:k + max_instances]
            verdicts = run_group(lattice, collision, reg_order, L, chunk, storage, check, stream, a1_source) \
                if a1_source else run_group(lattice, collision, reg_order, L, chunk, storage, check, stream)
            for (m, re), ok in zip(chunk, verdicts):
                tried[re][m] = ok
    out = {}
    for re in reynolds:
        a, b = bracket(re)
        out[re] = (a, None if b >= hi else b)
    return out


def stability_map(reynolds=(1e4, 3e4, 1e5, 1e6), L=128, lattices=("D2Q9", "D2V17", "D2V37"), storage="f32", check=20,
                  stream=None, variants=None):
    """M0^max per lattice, collision variant and Reynolds number.  Variants (default all): "bgk", "pr<N>" for
    the projection at every order N from 2 to the lattice maximum (PR-2 is the standard second-order
    projection; PR at the maximal order is the projection onto the lattice's whole Hermite basis, BGK
    itself on the complete D2Q9 basis) and "rr<N>" for the recursive regularization at every order from 3
    to the maximum ("rr2" would repeat "pr2"); "rrfd<N>" is RR-N with a1 from finite differences of the
    fields instead of the projection (Sec. II.E allows both).  "pr_best", "rr_projection_best" and
    "rr_fd_best" are the most stable order of each family, "rr_best" the most stable RR of either kind."""
    out = {}
    for lat in lattices:
        t0 = time.perf_counter()
        nmax = MAX_ORDER[lat]
        names = variants or (["bgk"] + ["pr%d" % n for n in range(2, nmax + 1)] +
                             ["rr%d" % n for n in range(3, nmax + 1)] + ["rrfd%d" % n for n in range(3, nmax + 1)])
        res = {}
        for v in names:
            fd = v.startswith("rrfd")
            coll, order = (v, 0) if v == "bgk" else (v[:2], int(v[4:] if fd else v[2:]))
            if order > nmax:
                continue
            res[v] = max_mach(lat, coll, reynolds, reg_order=order, L=L, storage=storage, check=check,
                              stream=stream, a1_source=1 if fd else 0)
        for fam, keys in (("pr_best", [k for k in res if k.startswith("pr")]),
                          ("rr_projection_best", [k for k in res if k.startswith("rr") and not k.startswith("rrfd")]),
                          ("rr_fd_best", [k for k in res if k.startswith("rrfd")]),
                          ("rr_best", [k for k in res if k.startswith("rr")])):
            if keys:
                res[fam] = {re: max(res[k][re][0] for k in keys) for re in reynolds}
        res["seconds"] = round(time.perf_counter() - t0, 2)
        out[lat] = res
    return out
