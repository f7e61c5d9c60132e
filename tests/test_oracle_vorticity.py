"""Pins of the oracle on the 2-D vorticity constraints (IC, total vorticity, enstrophy per
frame), which are family A's rows on a flattened frame with rate 0 and no energy floor."""
import numpy as np

from oracle import solve
from paper_2607_00095_b300 import synthetic
from tests import pins_1d

FLOOR = -1e300


def test_vorticity_rows_match_the_closed_form_and_conserve():
    N, nt, B = 4, 4, 3
    uh, pr = synthetic.gen_vorticity(61, B, N, nt)
    u, lam, st, S, b = solve.project_1d("A", N * N, nt, pr, uh, energy_floor=FLOOR, tol_kkt=1e-13)
    assert (st["status"] == 0).all()
    ue, le = pins_1d.family_a_closed_form(N * N, nt, pr, uh, energy_floor=FLOOR)
    np.testing.assert_allclose(u, ue, rtol=0, atol=1e-12)
    # the constraints of the Navier-Stokes problem, evaluated directly on the frames
    w = u.reshape(B, nt, N * N)
    w0 = pr[:, :N * N]
    np.testing.assert_allclose(w[:, 0], w0, atol=1e-13)
    np.testing.assert_allclose(w.mean(axis=2), np.repeat(w0.mean(axis=1)[:, None], nt, axis=1),
                               atol=1e-13)
    np.testing.assert_allclose((w * w).mean(axis=2),
                               np.repeat((w0 * w0).mean(axis=1)[:, None], nt, axis=1), atol=1e-12)
