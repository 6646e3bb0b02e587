"""Accuracy-versus-time sweeps (Sec. 3, time to solution against error).

CPU: the Pareto front keeps exactly the non-dominated cases.  GPU: on the
Kirkwood sphere (closed-form reference) the error falls with mesh refinement
at fixed solver settings, and the front runs from fast/coarse to
slow/accurate with a case below 0.3% error.
"""
import pytest

from paper_1309_4018_b300.pareto import Case, pareto_front


def test_front_is_the_non_dominated_set():
    pts = [(1.0, 0.5), (2.0, 0.1), (1.5, 0.6), (3.0, 0.1), (2.5, 0.05), (0.5, 0.9), (2.6, 0.2)]
    cases = [Case(str(i), {}, 0, t, 0.0, e, 0) for i, (t, e) in enumerate(pts)]
    front = pareto_front(cases)
    got = [(c.time_s, c.rel_error) for c in front]
    dominated = {p for p in pts if any(q[0] <= p[0] and q[1] <= p[1] and q != p for q in pts)}
    assert set(got) == set(pts) - dominated
    assert [t for t, _ in got] == sorted(t for t, _ in got)
    assert [e for _, e in got] == sorted((e for _, e in got), reverse=True)


@pytest.mark.gpu
def test_sphere_sweep():
    from gpu_util import ctx
    from oracle.closed_forms import kirkwood_energy
    from paper_1309_4018_b300.pareto import sweep
    from synth.configs import sphere_problem
    cases = []
    for level in (3, 4, 5, 6):
        d = sphere_problem(level=level, charges="both")
        for theta, P in ((0.6, 4), (0.5, 6)):
            cases.append((f"L{level} theta{theta} P{P}", d, dict(precision="mixed", theta=theta, P=P, ncrit=100,
                                                                  gmres_tol=1e-6)))
    ch = sphere_problem(level=3, charges="both")["charges"]
    ref = kirkwood_energy(4.0, 4.0, 80.0, 0.125, ch["xyz"], ch["q"])
    res = sweep(cases, ref, ctx())
    by = {c.label: c for c in res}
    for theta, P in ((0.6, 4), (0.5, 6)):
        errs = [by[f"L{l} theta{theta} P{P}"].rel_error for l in (3, 4, 5, 6)]
        assert all(a > b for a, b in zip(errs, errs[1:])), errs
    front = pareto_front(res)
    assert len(front) >= 2 and front[-1].rel_error < 3e-3
