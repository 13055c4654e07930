"""Host logic of the stability-range search (Sec. III.B: M0^max to 0.01): the bracket search against
verdict functions with known thresholds, no GPU (the runs are replaced by the verdict function)."""
import pytest

from paper_1704_04413_gb300 import stability as S


def fake_runs(monkeypatch, threshold, holes=()):
    calls = []

    def run_group(lattice, collision, reg_order, L, machs_res, storage="f32", check=20, stream=None):
        calls.append(list(machs_res))
        assert len(machs_res) <= 64
        return [m < threshold[re] and round(m, 6) not in holes for m, re in machs_res]

    monkeypatch.setattr(S, "run_group", run_group)
    return calls


@pytest.mark.parametrize("t1,t2", [(0.237, 0.61), (0.005, 1.6), (0.3, 0.3001), (1.2, 0.02)])
def test_brackets_the_threshold_to_the_grid(monkeypatch, t1, t2):
    thr = {1e4: t1, 1e6: t2}
    calls = fake_runs(monkeypatch, thr)
    out = S.max_mach("D2Q9", "rr", [1e4, 1e6], reg_order=4)
    for re, t in thr.items():
        a, b = out[re]
        stable_grid = [k / 100 for k in range(1, 150) if k / 100 < t]
        want_a = max(stable_grid) if stable_grid else 0.0
        assert a == pytest.approx(want_a)
        if t >= 1.5:
            assert b is None  # every tested Mach number was stable
        else:
            assert b == pytest.approx(want_a + 0.01)
    assert len(calls) <= 6  # a few rounds of parallel runs, not a sequential bisection


def test_an_unstable_point_below_the_threshold_caps_the_result(monkeypatch):
    # one isolated unstable Mach number below the smooth threshold: the search keeps the lowest unstable one
    thr = {3e4: 0.5}
    fake_runs(monkeypatch, thr, holes={0.1, 0.11, 0.12, 0.13, 0.14, 0.15, 0.16, 0.17, 0.18, 0.19, 0.2})
    a, b = S.max_mach("D2Q9", "rr", [3e4], reg_order=4)[3e4]
    assert b is not None and b <= 0.2 + 1e-9
    assert a < b and b - a <= 0.01 + 1e-9


def test_step_counts_cover_two_convective_times():
    cs = 3 ** -0.5
    assert S.steps_to(128, 0.2, cs) == 2218  # 2 L / (M0 cs)
    assert S.steps_to(128, 0.2, cs, convective_times=1.0) == 1109
