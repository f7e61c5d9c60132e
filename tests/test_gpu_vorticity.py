"""GPU parity of the 2-D vorticity constraints (Navier-Stokes problem: IC, total vorticity,
enstrophy per frame) through vorticity_problem against the oracle and the closed form."""
import numpy as np
import pytest

from oracle import problems, solve
from paper_2607_00095_b300 import synthetic, vorticity_problem
from tests import gpu_helpers as H
from tests import pins_1d

pytestmark = pytest.mark.gpu
FLOOR = -1e300


@pytest.mark.parametrize("N,nt,B,seed", [(4, 5, 3, 62), (16, 6, 4, 63)])
def test_vorticity_against_dense_oracle(N, nt, B, seed):
    uh, pr = synthetic.gen_vorticity(seed, B, N, nt)
    p = vorticity_problem(N, nt)
    u, lam, st, d = H.run_gpu(p, uh, pr)
    assert (st["status"] == 0).all() and st["h_inf"].max() <= H.H_TOL
    ue, le, so, S, _ = solve.project_1d("A", N * N, nt, pr, uh, energy_floor=FLOOR)
    assert (so["status"] == 0).all()
    H.assert_u_close(u, ue)
    H.assert_lam_close(S, lam, le)


def test_vorticity_full_size_closed_form_and_conservation():
    """The Navier-Stokes sizes (16 x 16, 50 frames), B = 512."""
    w = synthetic.WORKLOADS["vorticity_2d"]
    B, N, nt = w["B"], w["N"], w["nt"]
    uh, pr = synthetic.gen_vorticity(w["seed"], B, N, nt)
    p = vorticity_problem(N, nt)
    u, lam, st, d = H.run_gpu(p, uh, pr)
    assert (st["status"] == 0).all() and st["h_inf"].max() <= H.H_TOL
    ue, le = pins_1d.family_a_closed_form(N * N, nt, pr, uh, energy_floor=FLOOR)
    H.assert_u_close(u, ue)
    H.assert_lam_close(problems.structure_1d("A", N * N, nt), lam, le)
    wv = u.reshape(B, nt, N * N)
    w0 = pr[:, :N * N]
    # total vorticity per frame is the mass row (dx dy sum = mean here): the stopping test
    # bounds it by tol_kkt = 1e-10 (the iteration keeps u stationary, so the linear rows
    # converge with the nonlinear ones rather than in the first full step)
    np.testing.assert_allclose(wv.mean(axis=2), np.repeat(w0.mean(axis=1)[:, None], nt, axis=1),
                               atol=1e-10)
    np.testing.assert_allclose((wv * wv).mean(axis=2),
                               np.repeat((w0 * w0).mean(axis=1)[:, None], nt, axis=1),
                               rtol=1e-10)
