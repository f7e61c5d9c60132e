"""Family E -- Burgers with initial-condition, mass and Godunov flux rows.
TEST INFRASTRUCTURE ONLY: imported by tests/, smoke() and bench.py's CPU arms, never by the
CUDA library.

The constraint set of the Burgers IC regime (Appendix A, "IC, mass, Flux(k)"; the flux
residual of Appendix D, "Godunov's Flux Conservation"; the scaling study's Flux(1/5/10)):

  grid      x_i = i dx, i = 0..nx-1, dx = 1/(nx-1); t_k = k dt, k = 0..nt-1, dt = 1/(nt-1);
            neighbours are periodic (cell nx-1 is the left neighbour of cell 0);
  IC        u^0_i - g_i = 0                                          (nx rows)
  mass      dx sum_i u^k_i - M = 0,  M = dx sum_i g_i                 (nt rows, Riemann sum)
  flux      R^(k)_i = u^k_i - G(u^{k-1})_i = 0,  k = 1..K             (K nx rows)
            G(v)_i = v_i - (dt/dx) (F(v_i, v_{i+1}) - F(v_{i-1}, v_i))
  F(a, b)   the Godunov flux of f(u) = u^2/2: the minimum of f over [a, b] when a <= b, the
            maximum of f over [b, a] when a > b.

Row order: IC_0..IC_{nx-1}, mass_0..mass_{nt-1}, flux_1 (nx rows), ..., flux_K (nx rows).

Implied rows.  mass_0 follows from the IC rows, and with periodic neighbours the fluxes of
a step telescope, so mass_k (1 <= k <= K) follows from mass_{k-1} and the flux rows of
step k.  These K + 1 mass rows take no part in the solve (multiplier 0) but count in
||h||_inf.  The active rows then fix u^0..u^K completely (block lower-triangular in time
with identity diagonal blocks), and each later slice k > K only carries its mass row.

project() evaluates the KKT point by its definition: u^0 = g, u^k = G(u^{k-1}) for
k = 1..K, u^k = u_hat^k + (M/dx - sum u_hat^k)/nx for k > K; the multipliers solve the
stationarity equations u - u_hat + J^T lambda = 0 (dense solve with the transposed Jacobian
of the chain block; closed form on the mass slices).  newton_kkt() runs the Newton-KKT
iteration of Appendix B on the full system (small cases only) and reaches the same point.

Generalised Jacobian of F (the flux is piecewise quadratic; at a switch the branch taken by
these comparisons, in this order, is differentiated):
  a <= b:  a > 0  -> F = a^2/2 (dF/da = a);  b < 0 -> F = b^2/2 (dF/db = b);  else F = 0.
  a >  b:  a + b >= 0 -> F = a^2/2 (dF/da = a);  else F = b^2/2 (dF/db = b).
"""
import numpy as np

ROW_IC, ROW_MASS, ROW_FLUX = 0, 1, 9


def grid(nx, nt):
    dx = 1.0 / (nx - 1)
    dt = 1.0 / (nt - 1)
    return dx, dt, dt / dx


def godunov_flux(a, b):
    """F(a, b) for Burgers (elementwise)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    fa, fb = 0.5 * a * a, 0.5 * b * b
    # a <= b: min of the convex f over [a, b]: 0 if the interval holds 0, else the nearer end
    lo = np.where(a > 0, fa, np.where(b < 0, fb, 0.0))
    # a > b: max of f over [b, a]: the end with the larger |u|
    hi = np.maximum(fa, fb)
    return np.where(a <= b, lo, hi)


def flux_branch(a, b):
    """(ia, ib): 1 where the generalised derivative of F is taken from a^2/2 (ia) or b^2/2
    (ib); dF/da = ia a, dF/db = ib b, d2F/da2 = ia, d2F/db2 = ib."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    le = a <= b
    ia = np.where(le, a > 0, a + b >= 0)
    ib = np.where(le, (a <= 0) & (b < 0), a + b < 0)
    return ia.astype(np.float64), ib.astype(np.float64)


def godunov_step(v, c):
    """G(v) over the last axis, periodic neighbours, c = dt/dx."""
    v = np.asarray(v, np.float64)
    Fr = godunov_flux(v, np.roll(v, -1, axis=-1))        # F_{i+1/2}
    return v - c * (Fr - np.roll(Fr, 1, axis=-1))


def step_jacobian(v, c):
    """Dense dG/dv (nx x nx) at v (one slice)."""
    nx = v.shape[0]
    vr = np.roll(v, -1)
    ia, ib = flux_branch(v, vr)
    al, be = ia * v, ib * vr                             # dF_{i+1/2}/dv_i, dF_{i+1/2}/dv_{i+1}
    Jg = np.eye(nx)
    for i in range(nx):
        ip, im = (i + 1) % nx, (i - 1) % nx
        # G_i = v_i - c (F_{i+1/2} - F_{i-1/2})
        Jg[i, i] += -c * al[i]
        Jg[i, ip] += -c * be[i]
        Jg[i, im] += c * al[im]
        Jg[i, i] += c * be[im]
    return Jg


def sizes(nx, nt, K):
    n = nx * nt
    m = nx + nt + K * nx
    return n, m


def active_rows(nx, nt, K):
    _, m = sizes(nx, nt, K)
    act = np.ones(m, np.uint8)
    act[nx:nx + K + 1] = 0                               # mass_0 .. mass_K implied
    return act


def row_types(nx, nt, K):
    return np.concatenate([np.full(nx, ROW_IC), np.full(nt, ROW_MASS),
                           np.full(K * nx, ROW_FLUX)]).astype(np.int32)


def eval_h(nx, nt, K, g, u):
    """Every nominal row at u; g [B, nx], u [B, nt*nx] -> h [B, m]."""
    dx, _, c = grid(nx, nt)
    g = np.atleast_2d(np.asarray(g, np.float64))
    B = g.shape[0]
    U = np.asarray(u, np.float64).reshape(B, nt, nx)
    M = dx * g.sum(axis=1)
    h_ic = U[:, 0, :] - g
    h_mass = dx * U.sum(axis=2) - M[:, None]
    h_flux = [U[:, k, :] - godunov_step(U[:, k - 1, :], c) for k in range(1, K + 1)]
    return np.concatenate([h_ic, h_mass] + h_flux, axis=1)


def chain_jacobian(nx, nt, K, u_chain):
    """Jacobian of the IC and flux rows w.r.t. slices 0..K: square ((K+1) nx)."""
    _, _, c = grid(nx, nt)
    N = (K + 1) * nx
    J = np.zeros((N, N))
    J[:nx, :nx] = np.eye(nx)
    for k in range(1, K + 1):
        r = k * nx
        J[r:r + nx, k * nx:(k + 1) * nx] = np.eye(nx)
        J[r:r + nx, (k - 1) * nx:k * nx] = -step_jacobian(u_chain[k - 1], c)
    return J


def project(nx, nt, K, g, u_hat):
    """KKT point of every sample by definition.  g [B, nx], u_hat [B, nt*nx] ->
    (u [B, n], lam [B, m], stats dict)."""
    assert 1 <= K <= nt - 1
    dx, _, c = grid(nx, nt)
    g = np.atleast_2d(np.asarray(g, np.float64))
    B = g.shape[0]
    n, m = sizes(nx, nt, K)
    Uh = np.asarray(u_hat, np.float64).reshape(B, nt, nx)
    U = np.empty_like(Uh)
    lam = np.zeros((B, m))
    M = dx * g.sum(axis=1)
    for b in range(B):
        U[b, 0] = g[b]
        for k in range(1, K + 1):
            U[b, k] = godunov_step(U[b, k - 1], c)
        for k in range(K + 1, nt):
            U[b, k] = Uh[b, k] + (M[b] / dx - Uh[b, k].sum()) / nx
            lam[b, nx + k] = (Uh[b, k].sum() - M[b] / dx) / (nx * dx)
        J = chain_jacobian(nx, nt, K, U[b, :K + 1])
        rhs = (Uh[b, :K + 1] - U[b, :K + 1]).reshape(-1)
        lc = np.linalg.solve(J.T, rhs)
        lam[b, :nx] = lc[:nx]
        lam[b, nx + nt:] = lc[nx:]
    u = U.reshape(B, n)
    h = eval_h(nx, nt, K, g, u)
    stats = dict(h_inf=np.abs(h).max(axis=1), obj=0.5 * ((u - Uh.reshape(B, n)) ** 2).sum(axis=1))
    return u, lam, stats


def hess_lagrangian_diag(nx, nt, K, u, lam):
    """Diagonal of W = I + sum_r lam_r Hess h_r (one sample): only the flux rows are
    nonlinear, and their Hessians are diagonal (d2F/da2 = ia, d2F/db2 = ib)."""
    _, _, c = grid(nx, nt)
    U = u.reshape(nt, nx)
    W = np.ones((nt, nx))
    for k in range(1, K + 1):
        v = U[k - 1]
        ia, ib = flux_branch(v, np.roll(v, -1))
        lk = lam[nx + nt + (k - 1) * nx: nx + nt + k * nx]
        # R^(k)_i = u^k_i - v_i + c (F_{i+1/2} - F_{i-1/2});  F_{i+1/2} depends on (v_i, v_{i+1})
        for i in range(nx):
            ip, im = (i + 1) % nx, (i - 1) % nx
            W[k - 1, i] += c * lk[i] * ia[i] - c * lk[ip] * ia[i]
            W[k - 1, ip] += c * lk[i] * ib[i] - c * lk[ip] * ib[i]
    return W.reshape(-1)


def full_jacobian(nx, nt, K, u):
    """Dense Jacobian of every nominal row (one sample)."""
    n, m = sizes(nx, nt, K)
    dx, _, c = grid(nx, nt)
    U = u.reshape(nt, nx)
    J = np.zeros((m, n))
    J[:nx, :nx] = np.eye(nx)
    for k in range(nt):
        J[nx + k, k * nx:(k + 1) * nx] = dx
    for k in range(1, K + 1):
        r = nx + nt + (k - 1) * nx
        J[r:r + nx, k * nx:(k + 1) * nx] = np.eye(nx)
        J[r:r + nx, (k - 1) * nx:k * nx] = -step_jacobian(U[k - 1], c)
    return J


def newton_kkt(nx, nt, K, g, u_hat, tol=1e-10, max_iter=50, max_backtracks=30, c1=1e-4):
    """The Newton-KKT iteration of Appendix B on the full active system of one sample, from
    (u_hat, 0), merit 1/2 ||F||^2 with Armijo halving; dense solves.  Small cases only.
    Returns (u, lam, iters, converged)."""
    g = np.asarray(g, np.float64).reshape(-1)
    uh = np.asarray(u_hat, np.float64).reshape(-1)
    n, m = sizes(nx, nt, K)
    act = active_rows(nx, nt, K).astype(bool)
    u, lam = uh.copy(), np.zeros(m)

    def F_of(u, lam):
        h = eval_h(nx, nt, K, g[None], u[None])[0]
        J = full_jacobian(nx, nt, K, u)
        gl = u - uh + J[act].T @ lam[act]
        return np.concatenate([gl, h[act]]), J

    F, J = F_of(u, lam)
    for it in range(max_iter):
        if np.abs(F).max() <= tol:
            return u, lam, it, True
        Ja = J[act]
        W = np.diag(hess_lagrangian_diag(nx, nt, K, u, lam))
        ma = Ja.shape[0]
        Kkt = np.block([[W, Ja.T], [Ja, np.zeros((ma, ma))]])
        d = np.linalg.solve(Kkt, -F)
        du, dl = d[:n], d[n:]
        phi0 = 0.5 * F @ F
        t = 1.0
        for _ in range(max_backtracks + 1):
            un = u + t * du
            ln = lam.copy()
            ln[act] += t * dl
            Fn, Jn = F_of(un, ln)
            if 0.5 * Fn @ Fn <= (1 - 2 * c1 * t) * phi0:
                break
            t *= 0.5
        else:
            return u, lam, it, False
        u, lam, F, J = un, ln, Fn, Jn
    return u, lam, max_iter, bool(np.abs(F).max() <= tol)


def adjoint(nx, nt, K, g, u, gbar):
    """Implicit-function adjoint at the solution: K [a; b] = [gbar; 0].  On slices 0..K the
    active rows are square and invertible, so a = 0 there and J^T b = gbar; on a mass slice
    a = gbar - mean(gbar), b = sum(gbar) / (nx dx).  dL/dg = -b^T dh/dg = b_IC + dx sum of the
    active mass multipliers b (dM/dg_i = dx).  Returns (a [B, n], grad_g [B, nx], b [B, m])."""
    dx, _, _ = grid(nx, nt)
    g = np.atleast_2d(np.asarray(g, np.float64))
    B = g.shape[0]
    n, m = sizes(nx, nt, K)
    U = np.asarray(u, np.float64).reshape(B, nt, nx)
    G = np.asarray(gbar, np.float64).reshape(B, nt, nx)
    a = np.zeros((B, nt, nx))
    bl = np.zeros((B, m))
    gg = np.zeros((B, nx))
    for b in range(B):
        J = chain_jacobian(nx, nt, K, U[b, :K + 1])
        bc = np.linalg.solve(J.T, G[b, :K + 1].reshape(-1))
        bl[b, :nx] = bc[:nx]
        bl[b, nx + nt:] = bc[nx:]
        for k in range(K + 1, nt):
            bm = G[b, k].sum() / (nx * dx)
            bl[b, nx + k] = bm
            a[b, k] = G[b, k] - dx * bm
        gg[b] = bl[b, :nx] + dx * bl[b, nx + K + 1:nx + nt].sum()
    return a.reshape(B, n), gg, bl
