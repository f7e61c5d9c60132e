"""Pins of the oracle on family D (Burgers boundary-condition regime): linear rows, so the
projection is the normal-equations formula, reached by one Newton step."""
import numpy as np

from oracle import problems, solve
from paper_2607_00095_b300 import synthetic
from tests import pins_1d


def test_family_d_is_the_linear_projection():
    nx, nt, B = 9, 4, 3
    uh, pr = synthetic.gen_burgers_bc(81, B, nx, nt)
    S = problems.structure_bc(nx, nt)
    b = problems.rhs_bc(nx, nt, pr)
    u, lam, st = solve.project(S, b, uh.reshape(B, -1), tol_kkt=1e-13)
    assert (st["status"] == 0).all() and (st["iters"] <= 1).all()
    A = S.dense_A()
    for s in range(B):
        ue, le = pins_1d.linear_projection(A, b[s], uh[s].ravel())
        np.testing.assert_allclose(u[s], ue, rtol=0, atol=1e-12)
        np.testing.assert_allclose(lam[s], le, rtol=0, atol=1e-10)
    # the rows, written out from the definitions
    w = u.reshape(B, nt, nx)
    dx = 1.0 / (nx - 1)
    np.testing.assert_allclose(w[:, :, 0], np.repeat(pr[:, :1], nt, axis=1), atol=1e-13)
    np.testing.assert_allclose(dx * w.sum(axis=2), np.repeat(pr[:, 1:], nt, axis=1), atol=1e-13)
    np.testing.assert_allclose(w[:, :, -1], w[:, :, -2], atol=1e-13)
