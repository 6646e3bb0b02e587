"""Convergence study (Sec. 3 "Richardson extrapolation", Eqs. rich_extr, observed_order).

CPU: the two formulas recover the exponent and the limit of an exact power
law.  GPU: the 512/2,048/8,192-panel Kirkwood spheres solved by the library
converge at order one in the panel area and extrapolate to the closed form
within 1e-4 (the paper: order 1.013, Sec. 3.1); the synthetic protein meshed
at three grid spacings converges at an order near one.
"""
import numpy as np
import pytest

from paper_1309_4018_b300.richardson import extrapolate, observed_order


def test_formulas_on_a_power_law():
    for p, r, fstar, c in ((1.0, 4.0, -41.2, 3.0), (2.0, 2.0, 10.0, -0.5), (1.37, 1.5, 0.3, 2.2)):
        h = [1.0, 1.0 / r, 1.0 / r ** 2]
        f3, f2, f1 = (fstar + c * x ** p for x in h)
        assert abs(observed_order(f1, f2, f3, r) - p) < 1e-9
        assert abs(extrapolate(f1, f2, r, p) - fstar) < 1e-9 * max(1.0, abs(fstar))


@pytest.mark.gpu
def test_kirkwood_sphere_study():
    from gpu_util import ctx
    from oracle.closed_forms import kirkwood_energy
    from paper_1309_4018_b300.richardson import study
    from synth.configs import sphere_problem
    probs = [sphere_problem(level=l, charges="both") for l in (3, 4, 5)]
    st = study(probs, 4.0, ctx(), precision="fp64", theta=0.4, P=10, ncrit=100, gmres_tol=1e-10)
    d = probs[-1]
    ex = kirkwood_energy(4.0, 4.0, 80.0, 0.125, d["charges"]["xyz"], d["charges"]["q"])
    assert 0.9 < st.order < 1.1
    assert abs(st.extrapolated - ex) < 1e-4 * abs(ex)
    assert abs(st.energies[-1] - ex) > abs(st.extrapolated - ex)


@pytest.mark.gpu
def test_protein_study():
    """Nested refinements of the synthetic protein's surface (9.9k, 39.6k, 158k panels).

    Its charges sit 1.2-2 A under the surface, closer than these panels
    resolve, so the sequence is not yet in the asymptotic range (the study
    reports the observed order, or NaN when the differences change sign); the
    energies stay within a 0.5% band and the two precisions agree.
    """
    from gpu_util import ctx
    from paper_1309_4018_b300.richardson import study
    from synth.configs import protein_refinements
    probs = protein_refinements(levels=2)
    st = study(probs, 4.0, ctx(), precision="mixed", gmres_tol=1e-6)
    assert st.panels[1] == 4 * st.panels[0] and st.panels[2] == 4 * st.panels[1]
    e = np.array(st.energies)
    assert np.all(np.abs(e - e[-1]) < 5e-3 * abs(e[-1]))
    st64 = study(probs[:2], 4.0, ctx(), precision="fp64", gmres_tol=1e-8)
    assert np.allclose(st64.energies, e[:2], rtol=1e-6)
