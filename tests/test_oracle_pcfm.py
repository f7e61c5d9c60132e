"""Pins of the oracle's PCFM sampling loop (Sampling section, Eqs. 1-3) against results
derived independently of the loop code."""
import numpy as np

from oracle import pcfm, problems, solve
from paper_2607_00095_b300 import synthetic
from tests import pins_1d


def _linear_rows(nx, nt, params):
    """IC and mass rows of family A as a dense affine system A u = b."""
    S = problems.structure_1d("A", nx, nt)
    b = problems.rhs_1d("A", nx, nt, params[None])[0]
    rows = [r for r in range(S.m) if S.row_type[r] in (problems.ROW_IC, problems.ROW_MASS)
            and S.active[r]]
    A = np.zeros((len(rows), S.n))
    for j, r in enumerate(rows):
        A[j, S.a_col[S.a_ptr[r]:S.a_ptr[r + 1]]] = S.a_val[S.a_ptr[r]:S.a_ptr[r + 1]]
    return A, b[rows]


def test_affine_projection_closed_form_recursion():
    """With an affine projection P y + q the loop has a closed form: u_hat_1 at step k is
    tau_k u_1^(k-1) + (1 - tau_k) x1 + sigma0 (1 - tau_k)^2 xi (the u0 terms cancel), so
    u_1^(k) = Pi(x1) + sigma0 c_k P xi with c_0 = 1, c_k = tau_k c_(k-1) + (1 - tau_k)^2."""
    nx, nt, N, s0 = 8, 4, 6, 0.7
    u0, x1, xi, pr = synthetic.gen_pcfm(41, 1, nx, nt, "A")
    A, b = _linear_rows(nx, nt, pr[0])
    proj = lambda y: (pins_1d.linear_projection(A, b, y[0])[0][None], None, None)
    u, _, _ = pcfm.sample(proj, u0, x1, xi, N, s0)
    P = np.eye(A.shape[1]) - A.T @ np.linalg.solve(A @ A.T, A)
    c = 1.0
    for k in range(1, N):
        t = k / N
        c = t * c + (1 - t) ** 2
    expect = pins_1d.linear_projection(A, b, x1[0])[0] + s0 * c * (P @ xi[0])
    np.testing.assert_allclose(u[0], expect, rtol=0, atol=1e-12 * np.abs(expect).max())


def test_single_step_is_one_projection():
    nx, nt = 8, 4
    u0, x1, xi, pr = synthetic.gen_pcfm(42, 2, nx, nt, "A")
    proj = lambda y: solve.project_1d("A", nx, nt, pr, y, tol_kkt=1e-13)[:3]
    u, _, _ = pcfm.sample(proj, u0, x1, xi, 1, 0.4)
    ue, _ = pins_1d.family_a_closed_form(nx, nt, pr, x1 + 0.4 * xi)
    np.testing.assert_allclose(u, ue, rtol=0, atol=1e-12)


def test_no_perturbation_lands_on_the_projection_of_the_data():
    """sigma0 = 0: every candidate lies on the segment from x1 to Pi(x1), whose nearest
    feasible point is Pi(x1) (family A: unique, closed form)."""
    nx, nt = 16, 5
    u0, x1, xi, pr = synthetic.gen_pcfm(43, 3, nx, nt, "A")
    proj = lambda y: solve.project_1d("A", nx, nt, pr, y, tol_kkt=1e-13)[:3]
    u, _, st = pcfm.sample(proj, u0, x1, xi, 5, 0.0)
    assert (st["status"] == 0).all()
    ue, _ = pins_1d.family_a_closed_form(nx, nt, pr, x1)
    np.testing.assert_allclose(u, ue, rtol=0, atol=1e-11)
