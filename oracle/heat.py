"""Heat equation with IC, mass, PDE-residual and energy-evolution rows (the paper's second
heat-equation constraint operator, Appendix A "Heat Equation Problems"; the energy-evolution
identity of the appendix "Energy Evolution Constraint") -- TEST INFRASTRUCTURE ONLY.

Discretisation (the paper gives no stencil or time scheme; the consistent reading of its rows):
  x_i = i dx on the periodic [0, 2 pi), dx = 2 pi / nx;  t_k = k dt, dt = 1 / (nt - 1).
  D2 v_i = (v_{i+1} - 2 v_i + v_{i-1}) / dx^2,  D+ v_i = (v_{i+1} - v_i) / dx  (periodic).
Rows, in this order (per sample, params = [g_0 .. g_{nx-1}, alpha]):
  IC      u^0_i - g_i                                                       nx rows
  mass    dx sum_i u^k_i - dx sum_i g_i                     k = 0..nt-1     nt rows
  PDE     (u^k_i - u^{k-1}_i) / dt - alpha/2 (D2 u^k + D2 u^{k-1})_i       (nt-1) nx rows
                                                            k = 1..nt-1, slice-major
  energy  (E^k - E^{k-1}) / dt + alpha dx ||D+ ubar^k||^2,  E^k = 1/2 dx ||u^k||^2,
          ubar^k = (u^k + u^{k-1}) / 2                      k = 1..nt-1     nt-1 rows
The PDE rows are the Crank-Nicolson residual of u_t = alpha u_xx; the energy rows are the
discrete d/dt 1/2 int u^2 + alpha int u_x^2 at the same midpoint.  Taking the inner product of
a PDE row block with dx ubar^k and summing by parts (periodic: <D2 v, v> = -||D+ v||^2) gives
exactly the energy row, and summing a PDE row block over i gives the mass difference of
slices k and k-1: both families of rows are implied by the IC and PDE rows (left out of the
solve, multiplier 0, counted in ||h||_inf, as the rows at t = 0 of the other families).
The active rows (IC + PDE) are linear, square (nt nx rows for nt nx unknowns) and
nonsingular (A = I - alpha dt / 2 D2 is symmetric positive definite), so the feasible set is
the single point u* = J^-1 b (the Crank-Nicolson solution from g) and the projection of
eq. (2) is that point for every u_hat; its multipliers solve the stationarity equations
J^T lambda = u_hat - u*.  project() writes this definition out with a sparse LU of J (library
primitive).  The dense Newton-KKT of kkt_dense.c on the same active rows reaches the same
point in one step (tests).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def grid(nx, nt):
    dx = 2.0 * np.pi / nx
    dt = 1.0 / (nt - 1)
    return dx, dt


def sizes(nx, nt):
    """(variables, nominal rows, parameters) per sample."""
    return nx * nt, nx + nt + (nt - 1) * nx + (nt - 1), nx + 1


def offsets(nx, nt):
    """Row offsets of the four row types in the nominal order."""
    ic, mass = 0, nx
    pde = mass + nt
    energy = pde + (nt - 1) * nx
    return ic, mass, pde, energy


def active_rows(nx, nt):
    _, m, _ = sizes(nx, nt)
    ic, mass, pde, energy = offsets(nx, nt)
    a = np.zeros(m, np.uint8)
    a[ic:mass] = 1
    a[pde:energy] = 1
    return a


def _d2(v, dx):
    return (np.roll(v, -1, axis=-1) - 2.0 * v + np.roll(v, 1, axis=-1)) / (dx * dx)


def _dplus(v, dx):
    return (np.roll(v, -1, axis=-1) - v) / dx


def eval_h(nx, nt, params, u):
    """h(u) for every nominal row; params [B, nx+1], u [B, nt*nx] -> [B, m]."""
    params = np.atleast_2d(np.asarray(params, np.float64))
    B = params.shape[0]
    dx, dt = grid(nx, nt)
    g, alpha = params[:, :nx], params[:, nx]
    U = np.asarray(u, np.float64).reshape(B, nt, nx)
    h_ic = U[:, 0, :] - g
    h_mass = dx * U.sum(axis=2) - dx * g.sum(axis=1)[:, None]
    cur, prev = U[:, 1:, :], U[:, :-1, :]
    h_pde = (cur - prev) / dt - 0.5 * alpha[:, None, None] * (_d2(cur, dx) + _d2(prev, dx))
    E = 0.5 * dx * (U * U).sum(axis=2)
    ubar = 0.5 * (cur + prev)
    h_en = (E[:, 1:] - E[:, :-1]) / dt + alpha[:, None] * dx * (_dplus(ubar, dx) ** 2).sum(axis=2)
    return np.concatenate([h_ic, h_mass, h_pde.reshape(B, -1), h_en], axis=1)


def jacobian_active(nx, nt, alpha):
    """Sparse Jacobian of the active rows (IC, then PDE rows k = 1..nt-1) w.r.t. u, in the
    active-row order; square (nt nx)."""
    dx, dt = grid(nx, nt)
    n = nx * nt
    rows, cols, vals = [], [], []
    for i in range(nx):
        rows.append(i); cols.append(i); vals.append(1.0)
    c = 0.5 * alpha / (dx * dx)
    for k in range(1, nt):
        for i in range(nx):
            r = k * nx + i
            for (kk, sgn) in ((k, 1.0), (k - 1, -1.0)):
                base = kk * nx
                # (u^k - u^{k-1}) / dt  and  -alpha/2 D2 of both slices
                rows.append(r); cols.append(base + i); vals.append(sgn / dt + 2.0 * c)
                rows.append(r); cols.append(base + (i + 1) % nx); vals.append(-c)
                rows.append(r); cols.append(base + (i - 1) % nx); vals.append(-c)
    return sp.csc_matrix((vals, (rows, cols)), shape=(n, n))


def project(nx, nt, params, u_hat):
    """The projection by definition: u = J^-1 b (the single feasible point), lambda on the
    active rows from J^T lambda = u_hat - u.  Returns (u [B, n], lam [B, m], stats)."""
    params = np.atleast_2d(np.asarray(params, np.float64))
    B = params.shape[0]
    n, m, _ = sizes(nx, nt)
    u_hat = np.asarray(u_hat, np.float64).reshape(B, n)
    act = active_rows(nx, nt).astype(bool)
    u = np.zeros((B, n))
    lam = np.zeros((B, m))
    for b in range(B):
        J = jacobian_active(nx, nt, params[b, nx])
        lu = spla.splu(J)
        rhs = np.zeros(n)
        rhs[:nx] = params[b, :nx]
        u[b] = lu.solve(rhs)
        lam_act = lu.solve(u_hat[b] - u[b], trans="T")
        lam[b, act] = lam_act
    h = eval_h(nx, nt, params, u)
    stats = dict(status=np.zeros(B, np.int64), h_inf=np.abs(h).max(axis=1))
    return u, lam, stats


def adjoint(nx, nt, params, u, gbar):
    """Implicit-function adjoint at the solution: K [a; b] = [gbar; 0] with the square active
    J gives a = 0 (dL/du_hat = 0: the projection does not depend on u_hat) and J^T b = gbar.
    dL/dtheta = -b^T dh/dtheta: dL/dg = b_IC (h_IC = u^0 - g); dL/dalpha =
    sum_k b_PDE^k . 1/2 D2 (u^k + u^{k-1}).  Returns (a [B, n], grad_params [B, nx+1])."""
    params = np.atleast_2d(np.asarray(params, np.float64))
    B = params.shape[0]
    n, _, npar = sizes(nx, nt)
    dx, _ = grid(nx, nt)
    gbar = np.asarray(gbar, np.float64).reshape(B, n)
    U = np.asarray(u, np.float64).reshape(B, nt, nx)
    a = np.zeros((B, n))
    gp = np.zeros((B, npar))
    for b in range(B):
        J = jacobian_active(nx, nt, params[b, nx])
        bl = spla.splu(J).solve(gbar[b], trans="T")
        gp[b, :nx] = bl[:nx]
        bp = bl[nx:].reshape(nt - 1, nx)
        gp[b, nx] = np.sum(bp * 0.5 * (_d2(U[b, 1:], dx) + _d2(U[b, :-1], dx)))
    return a, gp


def cn_mode_solution(nx, nt, alpha, p, phase):
    """Closed form for a single Fourier mode g_i = sin(2 pi p i / nx + phase): every
    Crank-Nicolson step multiplies it by (1 - s) / (1 + s), s = 2 alpha dt / dx^2
    sin^2(pi p / nx) (the symbols of I -+ alpha dt / 2 D2 on that mode)."""
    dx, dt = grid(nx, nt)
    s = 2.0 * alpha * dt / (dx * dx) * np.sin(np.pi * p / nx) ** 2
    rho = (1.0 - s) / (1.0 + s)
    x = np.arange(nx) * dx
    g = np.sin(p * x + phase)
    return (rho ** np.arange(nt))[:, None] * g[None, :]
