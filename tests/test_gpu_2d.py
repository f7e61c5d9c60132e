"""GPU parity of the 2-D family (divergence with central differences + kinetic energy)
against the oracle's dense Newton-KKT (small grids) and its FFT closed form (full size)."""
import numpy as np
import pytest
import torch

from oracle import closed_form, problems, solve
from paper_2607_00095_b300 import Problem, _abi, decode_stats, synthetic
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _gpu(N, nt, wh, pr, **kw):
    p = Problem("C", N, nt)
    u, lam, st, d = H.run_gpu(p, wh, pr, **kw)
    return p, u, lam, st, d


@pytest.mark.parametrize("N,nt,B,seed", [(8, 3, 2, 301), (16, 2, 2, 302), (4, 2, 1, 303),
                                          (6, 3, 2, 305), (10, 2, 1, 306), (12, 2, 2, 307)])
def test_2d_parity_dense_oracle(N, nt, B, seed):
    wh, pr = synthetic.gen_2d(seed, B, N, nt, kmax=max(1, min(8, N // 2 - 1)))
    p, u, lam, st, d = _gpu(N, nt, wh, pr)
    S = problems.structure_2d(N, nt)
    b = problems.rhs_2d(N, nt, pr)
    ue, le, so = solve.project(S, b, wh.reshape(B, -1))
    assert (so["status"] == 0).all()
    np.testing.assert_array_equal(st["status"], 0)
    H.assert_u_close(u, ue)
    H.assert_lam_close(S, lam, le)
    assert st["h_inf"].max() <= H.H_TOL and st["kkt_inf"].max() <= 1e-10


@pytest.mark.parametrize("N,nt,B,seed", [(64, 16, 64, 1003), (32, 8, 16, 304), (20, 3, 5, 308),
                                          (24, 4, 8, 309), (48, 3, 6, 310), (62, 2, 3, 311),
                                          (30, 2, 3, 312)])
def test_2d_full_size_against_closed_form(N, nt, B, seed):
    """The 2-D velocity workload (B=64, 64x64, 16 frames), the uneven mix's 2-D size, and
    sides that are not powers of two: class sizes M = N / 2 of 10 and 12 (the plain class
    products), 24 (the register-tiled products), 31 and 15 (odd)."""
    wh, pr = synthetic.gen_2d(seed, B, N, nt)
    p, u, lam, st, d = _gpu(N, nt, wh, pr)
    np.testing.assert_array_equal(st["status"], 0)
    wc, lc = closed_form.project_2d(wh, pr)
    H.assert_u_close(u, wc.reshape(B, -1))
    S = problems.structure_2d(N, nt)
    H.assert_lam_close(S, lam, lc)
    # residual from the written w, GPU entry point and host
    h, hinf = p.residual(d["u"], d["pr"])
    assert hinf.cpu().numpy().max() <= H.H_TOL
    he = problems.eval_h(S, u[:2], problems.rhs_2d(N, nt, pr[:2]))
    np.testing.assert_allclose(h.cpu().numpy()[:2], he, atol=1e-11)


@pytest.mark.parametrize("N", [8, 12])
def test_2d_adjoint_against_oracle_and_fd(N):
    nt, B = 3, 2
    wh, pr = synthetic.gen_2d(311, B, N, nt, kmax=3)
    gbar = synthetic.gen_gbar(312, (B, nt * 2 * N * N))
    p, u, lam, st, d = _gpu(N, nt, wh, pr, tol_kkt=1e-13)
    np.testing.assert_array_equal(st["status"], 0)
    gh, gp = p.backward(H.to_dev(gbar), d["u"], d["lam"], d["pr"], stats=d["st"])
    gh = gh.cpu().numpy()
    gp = gp.cpu().numpy()
    # the oracle's dense adjoint at the oracle's own solution of the same inputs
    S = problems.structure_2d(N, nt)
    ue, le, so = solve.project(S, problems.rhs_2d(N, nt, pr), wh.reshape(B, -1), tol_kkt=1e-13)
    assert (so["status"] == 0).all()
    a, bl = solve.adjoint(S, ue, le, gbar)
    gpo = problems.grad_params_2d(N, nt, pr, bl)
    H.assert_adjoint_close(gh, a)
    H.assert_adjoint_close(gp, gpo)
    h = 1e-6

    def loss(prm, x):
        _, uu, _, ss, _ = _gpu(N, nt, x, prm, tol_kkt=1e-13)
        return (uu * gbar).sum(axis=1)

    for j in range(2):
        pp, pm = pr.copy(), pr.copy()
        pp[:, j] += h
        pm[:, j] -= h
        fd = (loss(pp, wh) - loss(pm, wh)) / (2 * h)
        np.testing.assert_allclose(fd, gp[:, j], rtol=1e-5, atol=1e-7)
    rng = np.random.default_rng(5)
    for _ in range(8):
        dr = rng.normal(size=wh.shape)
        fd = (loss(pr, wh + h * dr) - loss(pr, wh - h * dr)) / (2 * h)
        an = (gh * dr.reshape(B, -1)).sum(axis=1)
        np.testing.assert_allclose(fd, an, rtol=1e-5, atol=1e-7)


def test_2d_edge_cases():
    N, nt, B = 8, 2, 3
    wh, pr = synthetic.gen_2d(321, B, N, nt, kmax=3)
    wh[1, 0, 0, 3, 3] = np.nan                  # non-finite target
    # sample 2: exactly divergence-free target (the noiseless field)
    wc, _ = closed_form.project_2d(wh[2:3], pr[2:3])
    wh[2] = wc[0] * 1.3
    p, u, lam, st, d = _gpu(N, nt, wh, pr)
    assert st["status"][0] == 0 and st["status"][2] == 0
    assert st["status"][1] == 3
    np.testing.assert_allclose(u[2], wc.reshape(1, -1)[0], rtol=0, atol=1e-12 * np.abs(wc).max())
    with pytest.raises(_abi.SnapError):
        Problem("C", 66, 2)                     # grid sides above 64
    with pytest.raises(_abi.SnapError):
        Problem("C", 7, 2)                      # odd grid side
    with pytest.raises(_abi.SnapError) as ei:
        p.project(d["uh"], d["pr"], u0=d["uh"] + 0.0)
    assert ei.value.code == 2
