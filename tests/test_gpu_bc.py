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
    u, lam, st, d = H.run_gpu(p, uh, pr)
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
    u, lam, st, d = H.run_gpu(p, uh, pr)
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
    u, lam, st, d = H.run_gpu(p, uh, pr, tol_kkt=1e-12)
    assert st["status"][0] == 0 and st["iters"][0] == 1
    assert st["status"][1] == 0 and st["iters"][1] == 0
    np.testing.assert_array_equal(u[1], uh[1].ravel())
    assert st["status"][2] == 3
    with pytest.raises(_abi.SnapError):
        Problem("D", 3, 4)


def test_bc_adjoint_against_oracle_and_fd():
    nx, nt, B = 13, 4, 3
    uh, pr = synthetic.gen_burgers_bc(87, B, nx, nt)
    gbar = synthetic.gen_gbar(88, (B, nx * nt))
    p = Problem("D", nx, nt)
    u, lam, st, d = H.run_gpu(p, uh, pr)
    gh, gp = p.backward(H.to_dev(gbar), d["u"], d["lam"], d["pr"], stats=d["st"])
    torch.cuda.synchronize()
    gh, gp = gh.cpu().numpy(), gp.cpu().numpy()
    # the oracle's dense adjoint at the oracle's own solution of the same inputs
    S = problems.structure_bc(nx, nt)
    ue, le, so = solve.project(S, problems.rhs_bc(nx, nt, pr), uh.reshape(B, -1))
    assert (so["status"] == 0).all()
    a, bl = solve.adjoint(S, ue, le, gbar)
    np.testing.assert_allclose(gh, a, rtol=0, atol=1e-12 * np.abs(a).max())
    gpe = np.stack([bl[:, :nt].sum(axis=1), bl[:, nt:2 * nt].sum(axis=1)], axis=1)
    np.testing.assert_allclose(gp, gpe, rtol=1e-10, atol=1e-12)
    # central differences of L = gbar . u(u_hat, params)
    h = 1e-6

    def loss(prm, x):
        uu, _, _, _ = H.run_gpu(p, x, prm)
        return (uu * gbar).sum(axis=1)

    for j in range(2):
        pp, pm = pr.copy(), pr.copy()
        pp[:, j] += h
        pm[:, j] -= h
        np.testing.assert_allclose((loss(pp, uh) - loss(pm, uh)) / (2 * h), gp[:, j], rtol=1e-6,
                                   atol=1e-8)
    rng = np.random.default_rng(9)
    for _ in range(4):
        dr = rng.normal(size=uh.shape)
        fd = (loss(pr, uh + h * dr) - loss(pr, uh - h * dr)) / (2 * h)
        np.testing.assert_allclose(fd, (gh * dr.reshape(B, -1)).sum(axis=1), rtol=1e-6, atol=1e-8)
