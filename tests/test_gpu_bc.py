"""GPU parity of family D (Burgers boundary-condition regime: Dirichlet, mass and Neumann
rows per slice) against the oracle's dense Newton-KKT and the normal-equations formula."""
import numpy as np
import pytest
import torch

from oracle import problems, solve
from paper_2607_00095_b300 import Problem, _abi, decode_stats, synthetic
from tests import gpu_helpers as H


pytestmark = pytest.mark.gpu


def _oracle(nx, nt, pr, uh):
    S = problems.structure_bc(nx, nt)
    b = problems.rhs_bc(nx, nt, pr)
    u, lam, st = solve.project(S, b, uh.reshape(uh.shape[0], -1))
    return u, lam, st, S


@pytest.mark.parametrize("nx,nt,B,seed", [(9, 4, 3, 82), (4, 2, 2, 83), (101, 7, 4, 84),
                                          (128, 33, 5, 85)])
def test_bc_against_oracle(nx, nt, B, seed):
    uh, pr = synthetic.gen_burgers_bc(seed, B, nx, nt)
    p = Problem("D", nx, nt)
    u, lam, st, _, d = H.run_gpu(p, uh, pr)
    assert (st["status"] == 0).all() and st["h_inf"].max() <= 1e-12
    assert (st["iters"] == 1).all()
    ue, le, so, S = _oracle(nx, nt, pr, uh)
    assert (so["status"] == 0).all()
    H.assert_u_close(u, ue)
    H.assert_lam_close(S, lam, le)
    h, hinf = p.residual(d["u"], d["pr"])
    torch.cuda.synchronize()
    he = problems.eval_h(S, u, problems.rhs_bc(nx, nt, pr))
    np.testing.assert_allclose(h.cpu().numpy(), he, atol=1e-13)
    assert hinf.cpu().numpy().max() <= 1e-12


def test_bc_full_size_sampled():
    """The Burgers boundary-condition sizes: nx = nt = 101, B = 512 (odd nx)."""
    w = synthetic.WORKLOADS["burgers_bc_1d"]
    B, nx, nt = w["B"], w["nx"], w["nt"]
    uh, pr = synthetic.gen_burgers_bc(w["seed"], B, nx, nt)
    p = Problem("D", nx, nt)
    u, lam, st, _, d = H.run_gpu(p, uh, pr)
    assert (st["status"] == 0).all() and st["h_inf"].max() <= 1e-12
    pick = [0, 77, 511]
    ue, le, so, S = _oracle(nx, nt, pr[pick], uh[pick])
    H.assert_u_close(u[pick], ue)
    H.assert_lam_close(S, lam[pick], le)


def test_bc_edge_cases():
    nx, nt = 16, 3
    uh, pr = synthetic.gen_burgers_bc(86, 3, nx, nt)
    # sample 1: already feasible (no step); sample 2: a NaN
    ue, _, _, _ = _oracle(nx, nt, pr[1:2], uh[1:2])
    uh[1] = ue.reshape(nt, nx)
    uh[2, 1, 5] = np.nan
    p = Problem("D", nx, nt)
    u, lam, st, _, d = H.run_gpu(p, uh, pr, tol_kkt=1e-12)
    assert st["status"][0] == 0 and st["iters"][0] == 1
    assert st["status"][1] == 0 and st["iters"][1] == 0
    np.testing.assert_array_equal(u[1], uh[1].ravel())
    assert st["status"][2] == 3
    with pytest.raises(_abi.SnapError) as ei:
        p.backward(d["u"], d["u"], d["lam"], d["pr"])
    assert ei.value.code == 2
    with pytest.raises(_abi.SnapError):
        Problem("D", 3, 4)
