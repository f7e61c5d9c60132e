"""Pins of the oracle against things other than itself (CPU only).

Each pin is chosen so that a plausible slip in the oracle (a dropped term in grad L or in
W, a wrong sign of J^T lam, a transposed block of K, a wrong pivot in LDL^T, a wrong row
in the family builders, a wrong chain rule in dh/dtheta) fails at least one of them.
"""
import os

import numpy as np
import pytest

from oracle import closed_form, problems, solve
from paper_2607_00095_b300 import synthetic
from tests import pins_1d

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _subset(S, keep):
    """Structure with only the rows where keep is True (test helper)."""
    keep = np.asarray(keep, bool)
    rows = np.nonzero(keep)[0]

    def sub(ptr, col, val):
        p = [0]
        c, v = [], []
        for r in rows:
            c.extend(col[ptr[r]:ptr[r + 1]]); v.extend(val[ptr[r]:ptr[r + 1]])
            p.append(len(c))
        return np.asarray(p, np.int32), np.asarray(c, np.int32), np.asarray(v, np.float64)

    ap, ac, av = sub(S.a_ptr, S.a_col, S.a_val)
    qp, qc, qv = sub(S.q_ptr, S.q_col, S.q_val)
    return problems.Structure(S.family, S.n, len(rows), ap, ac, av, qp, qc, qv,
                              S.active[rows].copy(), S.row_type[rows].copy(), dict(S.dims))


# ---------------------------------------------------------------------------------------
# dense LDL^T against library routines
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("N,seed", [(1, 0), (2, 1), (5, 2), (17, 3), (60, 4)])
def test_ldl_solve_and_inertia_match_numpy(N, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(N, N))
    A = A + A.T
    if N >= 5:
        A[0, 0] = 0.0                      # forces a 2x2 pivot on the first step
    rhs = rng.normal(size=N)
    x, inert, rc = solve.ldl_solve_dense(A, rhs)
    assert rc == 0
    np.testing.assert_allclose(x, np.linalg.solve(A, rhs), rtol=1e-9, atol=1e-10)
    ev = np.linalg.eigvalsh(A)
    assert inert == (int((ev > 0).sum()), int((ev < 0).sum()), 0)


def test_ldl_kkt_inertia_and_singular():
    rng = np.random.default_rng(7)
    n, m = 6, 3
    J = rng.normal(size=(m, n))
    K = np.block([[np.eye(n), J.T], [J, np.zeros((m, m))]])
    _, inert, rc = solve.ldl_solve_dense(K, rng.normal(size=n + m))
    assert rc == 0 and inert == (n, m, 0)
    J[2] = J[0] + J[1]                     # rank deficient J -> singular K
    K = np.block([[np.eye(n), J.T], [J, np.zeros((m, m))]])
    _, inert, _ = solve.ldl_solve_dense(K, rng.normal(size=n + m))
    assert inert[2] >= 1


# ---------------------------------------------------------------------------------------
# row builders
# ---------------------------------------------------------------------------------------

def test_toy_jacobian_matches_printed_appendix_c():
    ref = np.loadtxt(os.path.join(GOLDEN, "toy_jacobian_appC.txt"))
    S = problems.structure_toy(3, 3)
    np.testing.assert_array_equal(S.dense_A(), ref)
    assert S.dense_Q().sum() == 0


def test_family_rows_by_definition():
    nx, nt = 8, 3
    S = problems.structure_1d("B", nx, nt)
    assert S.m == nx + 3 * nt and S.n == nx * nt
    rng = np.random.default_rng(3)
    u = rng.normal(size=(1, S.n))
    uh, pr = synthetic.gen_1d(5, 1, nx, nt, "B")
    b = problems.rhs_1d("B", nx, nt, pr)
    h = problems.eval_h(S, u, b)[0]
    U = u.reshape(nt, nx)
    dx = 1.0 / nx
    g = pr[0, :nx]
    assert np.allclose(h[:nx], U[0] - g)
    assert np.allclose(h[nx:nx + nt], dx * U.sum(1) - dx * g.sum())
    E0 = dx * (g * g).sum()
    t = np.arange(nt) / (nt - 1)
    Ek = np.maximum(E0 * np.exp(-0.5 * t), (dx * g.sum()) ** 2 + 0.05)
    assert np.allclose(h[nx + nt:nx + 2 * nt], dx * (U * U).sum(1) - Ek)
    assert np.allclose(h[nx + 2 * nt:], U[:, 0] ** 2 + U[:, nx // 2] ** 2 - pr[0, nx + 1:])
    assert list(S.active[nx:nx + nt]) == [0] + [1] * (nt - 1)


def test_divergence_rows_by_definition_and_redundancy():
    N, nt = 6, 2
    S = problems.structure_2d(N, nt)
    rng = np.random.default_rng(4)
    w = rng.normal(size=(nt, 2, N, N))
    h = problems.eval_h(S, w.reshape(1, -1), problems.rhs_2d(N, nt, [[1.0, 0.2]]))[0]
    dx = 1.0 / N
    u, v = w[0, 0], w[0, 1]
    div = (np.roll(u, -1, 1) - np.roll(u, 1, 1) + np.roll(v, -1, 0) - np.roll(v, 1, 0)) / (2 * dx)
    np.testing.assert_allclose(h[:N * N], div.ravel(), atol=1e-12)
    # D has exactly four redundant rows per frame; the active rows are independent
    A = S.dense_A()[:N * N, :2 * N * N]
    assert np.linalg.matrix_rank(A) == N * N - 4
    act = S.active[:N * N].astype(bool)
    assert np.linalg.matrix_rank(A[act]) == N * N - 4


# ---------------------------------------------------------------------------------------
# generators: closed values
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("nx", [8, 32, 128])
def test_generator_closed_values(nx):
    nt = 5
    uh, pr = synthetic.gen_1d(11, 6, nx, nt, "B")
    dx = 1.0 / nx
    g = pr[:, :nx]
    np.testing.assert_allclose(dx * g.sum(1), 0.0, atol=1e-14)          # M = 0
    np.testing.assert_allclose(dx * (g * g).sum(1), 0.625, atol=1e-14)  # E0 = 1/2 + 1/8
    # c_k = g(0)^2 + g(1/2)^2 = 1/2 sin^2(phi) * 2 ... with g(0) = g(1/2) = 0.5 sin(phi)
    phi_sin = g[:, 0] / 0.5
    t = np.arange(nt) / (nt - 1)
    np.testing.assert_allclose(pr[:, nx + 1:], 0.5 * phi_sin[:, None] ** 2 * np.exp(-t)[None], atol=1e-14)


# ---------------------------------------------------------------------------------------
# projections against closed forms
# ---------------------------------------------------------------------------------------

def test_linear_only_projection_matches_normal_equations():
    nx, nt, B = 16, 6, 3
    S = problems.structure_1d("A", nx, nt)
    keep = S.row_type != problems.ROW_ENERGY
    SL = _subset(S, keep)
    uh, pr = synthetic.gen_1d(21, B, nx, nt, "A")
    b = problems.rhs_1d("A", nx, nt, pr)[:, keep]
    u, lam, st = solve.project(SL, b, uh.reshape(B, -1))
    assert (st["status"] == 0).all()
    A = SL.dense_A()
    act = SL.active.astype(bool)
    for s in range(B):
        ue, ye = pins_1d.linear_projection(A[act], b[s, act], uh[s].ravel())
        np.testing.assert_allclose(u[s], ue, rtol=0, atol=1e-13)
        np.testing.assert_allclose(lam[s, act], ye, rtol=1e-11, atol=1e-12)
        assert np.all(lam[s, ~act] == 0)
        # per slice k >= 1: u_k = u_hat_k - mean(u_hat_k) + M ; slice 0 = g
        U = u[s].reshape(nt, nx)
        np.testing.assert_allclose(U[0], pr[s, :nx], atol=1e-14)
        M = pr[s, :nx].mean()
        np.testing.assert_allclose(U[1:], uh[s, 1:] - uh[s, 1:].mean(1, keepdims=True) + M, atol=1e-13)


def test_linear_projection_random_dense_rows():
    rng = np.random.default_rng(9)
    n, m = 12, 5
    A = rng.normal(size=(m, n))
    rows = [(list(range(n)), list(A[r])) for r in range(m)]
    ap, ac, av = problems._csr(rows, m)
    qp, qc, qv = problems._csr([([], [])] * m, m)
    S = problems.Structure("rand", n, m, ap, ac, av, qp, qc, qv, np.ones(m, np.uint8),
                           np.zeros(m, np.int32))
    b = rng.normal(size=(1, m))
    uh = rng.normal(size=(1, n))
    u, lam, st = solve.project(S, b, uh)
    ue, ye = pins_1d.linear_projection(A, b[0], uh[0])
    np.testing.assert_allclose(u[0], ue, atol=1e-12)
    np.testing.assert_allclose(lam[0], ye, atol=1e-11)
    assert st["iters"][0] == 1


def test_family_a_matches_closed_form_small_1d_workload():
    w = synthetic.WORKLOADS["small_1d"]
    nx, nt, B = w["nx"], w["nt"], w["B"]
    uh, pr = synthetic.gen_1d(w["seed"], B, nx, nt, "A")
    ue, le = pins_1d.family_a_closed_form(nx, nt, pr, uh)
    # default stopping test ||F||_inf <= 1e-10: u is within ~ ||K^-1|| 1e-10 of the solution
    u, lam, st, S, b = solve.project_1d("A", nx, nt, pr, uh)
    assert (st["status"] == 0).all() and (st["kkt_inf"] <= 1e-10).all()
    np.testing.assert_allclose(u, ue, rtol=0, atol=1e-9)
    # converged to the rounding floor, u and lambda agree to ~1e-13 (u = W^-1 (u_hat - A^T lam)
    # with u kept stationary rounds to within a few hundred ulps of the closed form's arithmetic)
    u, lam, st, S, b = solve.project_1d("A", nx, nt, pr, uh, tol_kkt=1e-13)
    assert (st["status"] == 0).all()
    np.testing.assert_allclose(u, ue, rtol=0, atol=3e-13)
    # the primal-dual iteration (explicit start u0 = u_hat) reaches the same point
    u2, lam2, st2, _, _ = solve.project_1d("A", nx, nt, pr, uh, u0=uh, tol_kkt=1e-13)
    assert (st2["status"] == 0).all()
    np.testing.assert_allclose(u2, ue, rtol=0, atol=3e-13)
    np.testing.assert_allclose(lam2, le, rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(lam, le, rtol=1e-10, atol=1e-11)
    assert st["h_inf"].max() <= 1e-12


def _kkt_residual(S, b, uh, u, lam):
    A, Q = S.dense_A(), S.dense_Q()
    act = S.active.astype(bool)
    J = A + 2.0 * Q * u[None, :]
    grad = u - uh + J[act].T @ lam[act]
    h = A @ u + Q @ (u * u) - b
    W = np.eye(S.n) + np.diag(2.0 * (lam[act, None] * Q[act]).sum(0))
    return np.abs(grad).max(), np.abs(h).max(), J[act], W


def _sosc_min_eig(J, W):
    # smallest eigenvalue of W on null(J)
    _, s, vt = np.linalg.svd(J)
    rank = int((s > 1e-10 * s[0]).sum())
    Z = vt[rank:].T
    return np.linalg.eigvalsh(Z.T @ W @ Z).min()


@pytest.mark.parametrize("family,nx,nt,seed", [("A", 8, 4, 1), ("B", 8, 4, 2), ("B", 12, 5, 3)])
def test_kkt_stationarity_feasibility_sosc_tiny(family, nx, nt, seed):
    B = 3
    uh, pr = synthetic.gen_1d(seed, B, nx, nt, family, noise=0.3)
    u, lam, st, S, b = solve.project_1d(family, nx, nt, pr, uh)
    for s in range(B):
        assert st["status"][s] == 0
        g, h, J, W = _kkt_residual(S, b[s], uh[s].ravel(), u[s], lam[s])
        assert g <= 1e-10 and h <= 1e-10
        assert _sosc_min_eig(J, W) > 0


def test_family_b_reduces_to_family_a():
    nx, nt, B = 16, 6, 4
    uh, prA = synthetic.gen_1d(31, B, nx, nt, "A")
    ua, la = pins_1d.family_a_closed_form(nx, nt, prA, uh)
    UA = ua.reshape(B, nt, nx)
    c = UA[:, :, 0] ** 2 + UA[:, :, nx // 2] ** 2
    prB = np.concatenate([prA, c], axis=1)
    u, lam, st, S, b = solve.project_1d("B", nx, nt, prB, uh)
    assert (st["status"] == 0).all()
    np.testing.assert_allclose(u, ua, atol=1e-12)
    # multipliers at the rounding floor (at ||F||_inf <= 1e-10 they carry ~ cond * 1e-10)
    u, lam, st, S, b = solve.project_1d("B", nx, nt, prB, uh, tol_kkt=1e-13)
    assert (st["status"] == 0).all()
    np.testing.assert_allclose(lam[:, :nx + 2 * nt], la, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(lam[:, nx + 2 * nt:], 0.0, atol=1e-10)


def test_family_b_brute_force_nx4():
    nx, nt = 4, 2
    rng = np.random.default_rng(41)
    hits = 0
    for trial in range(6):
        g = np.array([0.3, 1.0, -0.2, -0.8]) + 0.1 * rng.normal(size=4)
        pr = np.concatenate([g, [0.5], [g[0] ** 2 + g[2] ** 2, 0.7 * (g[0] ** 2 + g[2] ** 2)]])[None]
        uh = np.concatenate([g, 0.8 * g + 0.05 * rng.normal(size=4)])[None]
        u, lam, st, S, b = solve.project_1d("B", nx, nt, pr, uh)
        assert st["status"][0] == 0
        dx = 0.25
        M = dx * g.sum()
        E = b[0, nx + nt + 1]
        mins = pins_1d.brute_force_b_nx4(uh[0, 4:], M, E, pr[0, -1])
        uo = u[0, 4:]
        fo = 0.5 * np.sum((uo - uh[0, 4:]) ** 2)
        # the oracle lands on a local minimum of the curve; usually the global one
        d = min(np.abs(U - uo).max() for _, U in mins)
        assert d < 1e-6
        assert fo >= mins[0][0] - 1e-12
        hits += abs(fo - mins[0][0]) < 1e-10
    assert hits >= 4


def test_split_components_equals_unsplit():
    nx, nt, B = 8, 5, 2
    uh, pr = synthetic.gen_1d(51, B, nx, nt, "B")
    u1, l1, s1, S, b = solve.project_1d("B", nx, nt, pr, uh)
    u0, l0, s0 = solve.project(S, b, uh.reshape(B, -1), split_components=0)
    assert (s0["status"] == 0).all()
    np.testing.assert_allclose(u1, u0, atol=1e-12)
    np.testing.assert_allclose(l1, l0, rtol=1e-8, atol=1e-10)
    nc, cv, cr = solve.components(S)
    assert nc == nx + (nt - 1)           # each IC row is its own component; one per slice k >= 1
    assert (cr[~S.active.astype(bool)] == -1).all()


def test_batch_permutation_exact():
    nx, nt, B = 8, 4, 5
    uh, pr = synthetic.gen_1d(61, B, nx, nt, "B")
    u, lam, st, _, _ = solve.project_1d("B", nx, nt, pr, uh)
    p = np.array([3, 0, 4, 1, 2])
    u2, lam2, st2, _, _ = solve.project_1d("B", nx, nt, pr[p], uh[p])
    assert np.array_equal(u2, u[p]) and np.array_equal(lam2, lam[p])


# ---------------------------------------------------------------------------------------
# 2-D: dense Newton-KKT against the FFT closed form
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("N", [6, 8, 12, 16])
def test_2d_dense_newton_matches_fft_closed_form(N):
    nt, B = 2, 2
    wh, pr = synthetic.gen_2d(71 + N, B, N, nt, kmax=min(8, N // 2 - 1))
    S = problems.structure_2d(N, nt)
    b = problems.rhs_2d(N, nt, pr)
    u, lam, st = solve.project(S, b, wh.reshape(B, -1))
    assert (st["status"] == 0).all()
    wc, lc = closed_form.project_2d(wh, pr)
    np.testing.assert_allclose(u, wc.reshape(B, -1), atol=1e-11)
    scale = np.abs(lc[:, :nt * N * N]).max()
    np.testing.assert_allclose(lam[:, :nt * N * N], lc[:, :nt * N * N], atol=1e-9 * scale)
    np.testing.assert_allclose(lam[:, nt * N * N:], lc[:, nt * N * N:], rtol=1e-9)
    assert np.all(lam[:, :nt * N * N][:, ~S.active[:nt * N * N].astype(bool)] == 0)


def test_2d_closed_form_properties_full_grid():
    N, nt, B = 64, 3, 2
    wh, pr = synthetic.gen_2d(81, B, N, nt)
    w, lam = closed_form.project_2d(wh, pr)
    S = problems.structure_2d(N, nt)
    h = problems.eval_h(S, w.reshape(B, -1), problems.rhs_2d(N, nt, pr))
    assert np.abs(h).max() < 1e-10
    # stationarity: w - w_hat + D^T lam_div + lam_K dx^2 w = 0
    A = None
    import scipy.sparse as sp
    A = sp.csr_matrix((S.a_val, S.a_col, S.a_ptr), shape=(S.m, S.n))
    dx = 1.0 / N
    for s in range(B):
        lk = np.repeat(lam[s, nt * N * N:], 2 * N * N)
        g = w[s].ravel() - wh[s].ravel() + A[:nt * N * N].T @ lam[s, :nt * N * N] + lk * dx * dx * w[s].ravel()
        assert np.abs(g).max() < 1e-10


# ---------------------------------------------------------------------------------------
# adjoint: central finite differences of the forward projection
# ---------------------------------------------------------------------------------------

def _fd_loss(family, nx, nt, pr, uh, gbar):
    u, _, st, _, _ = solve.project_1d(family, nx, nt, pr, uh, tol_kkt=1e-13)
    assert (st["status"] == 0).all()
    return float(np.sum(u * gbar.reshape(u.shape)))


def test_adjoint_matches_central_fd():
    family, nx, nt, B = "B", 16, 5, 4
    uh, pr = synthetic.gen_1d(91, B, nx, nt, family)
    gbar = synthetic.gen_gbar(92, (B, nt * nx))
    u, lam, st, S, b = solve.project_1d(family, nx, nt, pr, uh, tol_kkt=1e-13)
    a, gp, bl = solve.adjoint_1d(family, nx, nt, pr, u, lam, gbar)
    h = 1e-6
    rng = np.random.default_rng(93)
    # every parameter (g, r, c) of sample 0 and 1
    for s in (0, 1):
        for j in range(pr.shape[1]):
            pp, pm = pr.copy(), pr.copy()
            pp[s, j] += h; pm[s, j] -= h
            fd = (_fd_loss(family, nx, nt, pp, uh, gbar) - _fd_loss(family, nx, nt, pm, uh, gbar)) / (2 * h)
            assert abs(fd - gp[s, j]) <= 1e-5 * max(1.0, abs(gp[s, j])), (s, j, fd, gp[s, j])
    # random directions in u_hat
    for _ in range(8):
        d = rng.normal(size=uh.shape)
        fd = (_fd_loss(family, nx, nt, pr, uh + h * d, gbar) - _fd_loss(family, nx, nt, pr, uh - h * d, gbar)) / (2 * h)
        an = float(np.sum(a * d.reshape(a.shape)))
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an))


def test_adjoint_family_a_against_closed_form_fd():
    nx, nt, B = 32, 6, 2
    uh, pr = synthetic.gen_1d(95, B, nx, nt, "A")
    gbar = synthetic.gen_gbar(96, (B, nt * nx))
    u, lam, st, S, b = solve.project_1d("A", nx, nt, pr, uh, tol_kkt=1e-13)
    a, gp, bl = solve.adjoint_1d("A", nx, nt, pr, u, lam, gbar)
    h = 1e-6

    def loss(p, x):
        uc, _ = pins_1d.family_a_closed_form(nx, nt, p, x)
        return float(np.sum(uc * gbar))

    for j in (0, 5, nx):                                   # g_0, g_5, r
        pp, pm = pr.copy(), pr.copy()
        pp[:, j] += h; pm[:, j] -= h
        fd = (loss(pp, uh) - loss(pm, uh)) / (2 * h)
        assert abs(fd - gp[:, j].sum()) <= 1e-5 * max(1.0, abs(fd))
    rng = np.random.default_rng(97)
    d = rng.normal(size=uh.shape)
    fd = (loss(pr, uh + h * d) - loss(pr, uh - h * d)) / (2 * h)
    assert abs(fd - np.sum(a * d.reshape(a.shape))) <= 1e-5 * max(1.0, abs(fd))


@pytest.mark.parametrize("N", [6, 8, 16])
def test_adjoint_2d_grad_params_against_closed_form_fd(N):
    """dL/d(K0, r2) of the 2-D family: the oracle's dense adjoint at its own solution, mapped
    through grad_params_2d, against central differences of the FFT closed form (a different
    route to the same projection); also dL/dw_hat along random directions.  A slip in either
    derivative of K0 exp(-r2 t) (sign, the factor t, the factor K0) fails here."""
    nt, B = 3, 2
    wh, pr = synthetic.gen_2d(170 + N, B, N, nt, kmax=min(8, N // 2 - 1))
    pr = pr.copy()
    pr[:, 1] = [0.2, 0.7]                     # distinct decay rates per sample
    gbar = synthetic.gen_gbar(180 + N, (B, nt * 2 * N * N))
    S = problems.structure_2d(N, nt)
    u, lam, st = solve.project(S, problems.rhs_2d(N, nt, pr), wh.reshape(B, -1), tol_kkt=1e-13)
    assert (st["status"] == 0).all()
    a, bl = solve.adjoint(S, u, lam, gbar)
    gp = problems.grad_params_2d(N, nt, pr, bl)

    def loss(p, x):
        w, _ = closed_form.project_2d(x, p)
        return (w.reshape(B, -1) * gbar).sum(axis=1)

    h = 1e-6
    for j in range(2):
        pp, pm = pr.copy(), pr.copy()
        pp[:, j] += h; pm[:, j] -= h
        fd = (loss(pp, wh) - loss(pm, wh)) / (2 * h)
        np.testing.assert_allclose(gp[:, j], fd, rtol=1e-6, atol=1e-9)
        assert np.all(np.abs(gp[:, j]) > 1e-3)          # the check is not vacuous
    rng = np.random.default_rng(190 + N)
    for _ in range(3):
        d = rng.normal(size=wh.shape)
        fd = (loss(pr, wh + h * d) - loss(pr, wh - h * d)) / (2 * h)
        np.testing.assert_allclose((a * d.reshape(B, -1)).sum(axis=1), fd, rtol=1e-6, atol=1e-8)
