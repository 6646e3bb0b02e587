"""Pins of the oracle treecode matvec (Sec. 2.3): theta -> 0 is the dense operator,
and the truncation error falls with the expansion order P."""
import numpy as np

from oracle import formulation as F
from oracle.dense import operator_matrix
from oracle.treecode import TreecodeOracle
from synth.configs import layered_sphere_problem, sphere_problem


def _rel(out, y, pr, rows):
    num = den = 0.0
    for (s, side), v in out.items():
        ref = y[F.row_slice(pr, s, side)][rows[s]]
        num += ((v - ref) ** 2).sum()
        den += (ref ** 2).sum()
    return np.sqrt(num / den)


def test_theta0_equals_dense():
    pr = sphere_problem(level=3, charges="both")
    A = operator_matrix(pr)
    x = np.random.default_rng(0).normal(size=A.shape[0])
    tc = TreecodeOracle(pr, dict(theta=0.0, ncrit=30))
    rows = {0: np.arange(0, 512, 5)}
    assert _rel(tc.matvec(x, rows), A @ x, pr, rows) < 1e-14


def test_error_falls_with_order():
    pr = layered_sphere_problem(level=3, charges="both")
    A = operator_matrix(pr)
    x = np.random.default_rng(1).normal(size=A.shape[0])
    y = A @ x
    rows = {0: np.arange(0, 512, 17), 1: np.arange(0, 512, 17)}
    errs = []
    for P in (1, 3, 5):
        tc = TreecodeOracle(pr, dict(theta=0.5, ncrit=20, P=P))
        errs.append(_rel(tc.matvec(x, rows), y, pr, rows))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 1e-3
