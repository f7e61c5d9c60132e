"""GPU implicit-function adjoint of the 1-D projection against the oracle's dense adjoint
and central finite differences (h = 1e-6, relative 1e-5)."""
import numpy as np
import pytest
import torch

from oracle import solve
from paper_2607_00095_b300 import Problem, SnapProject, synthetic
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _setup(B, nx, nt, seed, family="B"):
    uh, pr = synthetic.gen_1d(seed, B, nx, nt, family)
    gbar = synthetic.gen_gbar(seed + 1, (B, nt * nx))
    return uh, pr, gbar


def test_backward_matches_oracle_dense_adjoint():
    B, nx, nt = 6, 128, 25
    uh, pr, gbar = _setup(B, nx, nt, 101)
    p = Problem("B", nx, nt)
    u, lam, st, d = H.run_gpu(p, uh, pr)
    assert (st["status"] == 0).all()
    gh, gp = p.backward(H.to_dev(gbar), d["u"], d["lam"], d["pr"], stats=d["st"])
    torch.cuda.synchronize()
    # the oracle's adjoint at the oracle's own solution of the same seeded inputs: nothing
    # on the oracle side comes from the GPU
    a, gpo = H.oracle_adjoint_1d("B", nx, nt, pr, uh, gbar)
    H.assert_adjoint_close(gh.cpu().numpy(), a)
    H.assert_adjoint_close(gp.cpu().numpy(), gpo)


def test_backward_full_size_sampled():
    """The differentiation workload at the bench's size and launch configuration (B = 512,
    128 x 100), 16 sampled samples against the oracle's dense adjoint at its own solution."""
    B, nx, nt = 512, 128, 100
    uh, pr = synthetic.gen_1d(1001, B, nx, nt, "B")
    gbar = synthetic.gen_gbar(1002, (B, nt * nx))
    p = Problem("B", nx, nt)
    u, lam, st, d = H.run_gpu(p, uh, pr)
    assert (st["status"] == 0).all()
    pick = np.sort(np.random.default_rng(17).choice(B, size=16, replace=False))
    a, gpo = H.oracle_adjoint_1d("B", nx, nt, pr[pick], uh[pick], gbar[pick])
    gh, gp = p.backward(H.to_dev(gbar), d["u"], d["lam"], d["pr"], stats=d["st"])
    torch.cuda.synchronize()
    H.assert_adjoint_close(gh.cpu().numpy()[pick], a)
    H.assert_adjoint_close(gp.cpu().numpy()[pick], gpo)


def test_backward_repeatable():
    """Two calls on the same inputs give the same bits (no state between calls)."""
    B, nx, nt = 8, 128, 40
    uh, pr, gbar = _setup(B, nx, nt, 111)
    p = Problem("B", nx, nt)
    u, lam, st, d = H.run_gpu(p, uh, pr)
    g1 = p.backward(H.to_dev(gbar), d["u"], d["lam"], d["pr"], stats=d["st"])
    g0 = p.backward(H.to_dev(gbar), d["u"], d["lam"], d["pr"], stats=d["st"])
    for x, y in zip(g1, g0):
        np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())


def test_backward_central_fd():
    """B = 4 as the differentiation workload states; every r and c_k, 32 u_hat directions."""
    B, nx, nt = 4, 128, 100
    uh, pr, gbar = _setup(B, nx, nt, 1001)
    gbar = synthetic.gen_gbar(1002, (B, nt * nx))
    p = Problem("B", nx, nt)
    opts = dict(tol_kkt=1e-13)
    u, lam, st, d = H.run_gpu(p, uh, pr, **opts)
    assert (st["status"] == 0).all()
    gh, gp = p.backward(H.to_dev(gbar), d["u"], d["lam"], d["pr"], stats=d["st"])
    gh = gh.cpu().numpy()
    gp = gp.cpu().numpy()
    h = 1e-6

    def loss(prm, x):
        uu, _, ss, _ = H.run_gpu(p, x, prm, **opts)
        assert (ss["status"] == 0).all()
        return (uu * gbar).sum(axis=1)

    cols = [nx] + [nx + 1 + k for k in range(1, nt)]          # r and c_1..c_{nt-1}
    for j in cols:
        pp, pm = pr.copy(), pr.copy()
        pp[:, j] += h
        pm[:, j] -= h
        fd = (loss(pp, uh) - loss(pm, uh)) / (2 * h)
        for s in range(B):
            assert abs(fd[s] - gp[s, j]) <= 1e-5 * max(1.0, abs(gp[s, j])), (j, s, fd[s], gp[s, j])
    rng = np.random.default_rng(3)
    for _ in range(32):
        dr = rng.normal(size=uh.shape)
        fd = (loss(pr, uh + h * dr) - loss(pr, uh - h * dr)) / (2 * h)
        an = (gh * dr.reshape(B, -1)).sum(axis=1)
        for s in range(B):
            assert abs(fd[s] - an[s]) <= 1e-5 * max(1.0, abs(an[s]))


def test_autograd_function_and_nan_for_failed_samples():
    B, nx, nt = 3, 64, 6
    uh, pr, gbar = _setup(B, nx, nt, 121)
    pr[1, nx + 1 + 3] = -1.0                     # sample 1 infeasible -> NaN gradients
    p = Problem("B", nx, nt)
    x = H.to_dev(uh.reshape(B, -1)).requires_grad_(True)
    th = H.to_dev(pr).requires_grad_(True)
    for _ in range(2):
        y = SnapProject.apply(x, th, p)
        (y * H.to_dev(gbar)).sum().backward()
        gx = x.grad.cpu().numpy()
        gt = th.grad.cpu().numpy()
        assert np.isnan(gx[1]).all() and np.isnan(gt[1]).all()
        assert np.isfinite(gx[[0, 2]]).all() and np.isfinite(gt[[0, 2]]).all()
        x.grad = None
        th.grad = None
