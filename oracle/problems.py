"""Constraint rows of each problem family, for the oracle -- TEST INFRASTRUCTURE ONLY.

Every row has the form  h_r(u) = sum_j A_rj u_j + sum_j Q_rj u_j^2 - b_r(theta), so the
oracle's dense Newton-KKT solver (kkt_dense.c) needs only (A, Q, b, active).

Families and their sources:
  "A"   initial condition, per-step mass, per-step energy on a periodic 1-D space-time
        grid.  Constraint types of Table I (Dirichlet IC "Au - b", global mass
        "int u dx - C"); Riemann-sum discretisation of Appendix D ("Discretization":
        m(t_k) ~ sum_i u_i^k dx); the energy is the per-step invariant
        dx * sum_i u_i^2 = E_k with E_k = max(E0 exp(-r t_k), M^2 + floor),
        E0 = dx sum g^2, M = dx sum g (no 1/2: the workload's definition; Appendix A
        defines E(t) with a 1/2, see the readings list).
  "B"   "A" plus the nonlinear two-sided boundary invariant u(0,t)^2 + u(1/2,t)^2 = c(t).
  "C"   2-D velocity (u, v) on a periodic N x N grid per frame: discrete divergence with
        2nd-order central differences, and kinetic energy 1/2 dx^2 sum(u^2+v^2) = K0 exp(-r2 t).
  "toy" the worked example of Appendix C: IC rows, then left-Riemann mass differences
        sum_{i=1}^{Nx-1} u_i^(k) - sum_{i=1}^{Nx-1} u_i^(1) for k = 2..Nt (first step omitted).

Variable order (Appendix C's flattening, x fastest within a time slice):
  1-D: u[k * nx + i], k = time index, i = space index.
  2-D: w[f * 2N^2 + c * N^2 + j * N + i], c = 0 (u) or 1 (v), j = y index, i = x index.

Row order (nominal, all rows, including the ones implied by others):
  1-D: IC_0..IC_{nx-1}, mass_0..mass_{nt-1}, energy_0..energy_{nt-1}, [boundary_0..].
  2-D: div[f][j][i] for all frames, then energy_0..energy_{nt-1}.

Rows implied by other rows take no part in the solve (active = 0, multiplier 0), but
still count in ||h||_inf:
  1-D: mass_0, energy_0, boundary_0 are fixed by the IC rows (Appendix C also omits the
       first-step mass row).
  2-D: central differences on an even periodic grid leave four redundant divergence rows
       per frame, one per parity class (i mod 2, j mod 2); the rows at cells
       (0,0), (1,0), (0,1), (1,1) are the ones left out.
"""
from dataclasses import dataclass, field

import numpy as np

ROW_IC, ROW_MASS, ROW_ENERGY, ROW_BOUNDARY, ROW_DIV, ROW_KE, ROW_TOYMASS = range(7)
ROW_DIRICHLET, ROW_NEUMANN = 7, 8
ROW_TYPE_NAMES = {ROW_IC: "ic", ROW_MASS: "mass", ROW_ENERGY: "energy",
                  ROW_BOUNDARY: "boundary", ROW_DIV: "div", ROW_KE: "kinetic_energy",
                  ROW_TOYMASS: "mass", ROW_DIRICHLET: "dirichlet", ROW_NEUMANN: "neumann",
                  9: "flux"}


@dataclass
class Structure:
    family: str
    n: int                      # variables per sample
    m: int                      # nominal rows per sample
    a_ptr: np.ndarray
    a_col: np.ndarray
    a_val: np.ndarray
    q_ptr: np.ndarray
    q_col: np.ndarray
    q_val: np.ndarray
    active: np.ndarray          # uint8 [m]
    row_type: np.ndarray        # int [m]
    dims: dict = field(default_factory=dict)

    def dense_A(self):
        A = np.zeros((self.m, self.n))
        for r in range(self.m):
            for p in range(self.a_ptr[r], self.a_ptr[r + 1]):
                A[r, self.a_col[p]] += self.a_val[p]
        return A

    def dense_Q(self):
        Q = np.zeros((self.m, self.n))
        for r in range(self.m):
            for p in range(self.q_ptr[r], self.q_ptr[r + 1]):
                Q[r, self.q_col[p]] += self.q_val[p]
        return Q


def _csr(rows, m):
    """rows: list (length m) of (cols, vals) -> CSR arrays."""
    ptr = np.zeros(m + 1, dtype=np.int32)
    cols, vals = [], []
    for r in range(m):
        c, v = rows[r]
        ptr[r + 1] = ptr[r] + len(c)
        cols.append(np.asarray(c, dtype=np.int32))
        vals.append(np.asarray(v, dtype=np.float64))
    col = np.concatenate(cols) if cols else np.zeros(0, np.int32)
    val = np.concatenate(vals) if vals else np.zeros(0)
    return ptr, col.astype(np.int32), val.astype(np.float64)


def time_grid(nt):
    """t_k = k / (nt - 1), k = 0..nt-1, on t in [0, 1] (the workloads' dt = 1/(nt-1))."""
    return np.arange(nt, dtype=np.float64) / (nt - 1)


# ----------------------------------------------------------------------------------------
# 1-D families A and B
# ----------------------------------------------------------------------------------------

def structure_1d(family, nx, nt):
    """Rows of families "A" (IC, mass, energy) and "B" (+ boundary invariant)."""
    assert family in ("A", "B")
    assert nx >= 4 and nx % 2 == 0 and nt >= 2
    dx = 1.0 / nx
    ih = nx // 2
    empty = ([], [])
    arows, qrows, types, active = [], [], [], []
    for i in range(nx):                                   # IC: u(x_i, 0) - g_i
        arows.append(([i], [1.0])); qrows.append(empty)
        types.append(ROW_IC); active.append(1)
    for k in range(nt):                                   # mass: dx sum_i u_{k,i} - M
        arows.append((list(range(k * nx, (k + 1) * nx)), [dx] * nx)); qrows.append(empty)
        types.append(ROW_MASS); active.append(1 if k > 0 else 0)
    for k in range(nt):                                   # energy: dx sum_i u_{k,i}^2 - E_k
        arows.append(empty); qrows.append((list(range(k * nx, (k + 1) * nx)), [dx] * nx))
        types.append(ROW_ENERGY); active.append(1 if k > 0 else 0)
    if family == "B":
        for k in range(nt):                               # u_{k,0}^2 + u_{k,nx/2}^2 - c_k
            arows.append(empty); qrows.append(([k * nx, k * nx + ih], [1.0, 1.0]))
            types.append(ROW_BOUNDARY); active.append(1 if k > 0 else 0)
    m = len(types)
    ap, ac, av = _csr(arows, m)
    qp, qc, qv = _csr(qrows, m)
    return Structure(family, nx * nt, m, ap, ac, av, qp, qc, qv,
                     np.asarray(active, np.uint8), np.asarray(types, np.int32),
                     dict(nx=nx, nt=nt))


def n_params_1d(family, nx, nt):
    """params = [g_0..g_{nx-1}, r, (c_0..c_{nt-1} for family B)]."""
    return nx + 1 + (nt if family == "B" else 0)


def rhs_1d(family, nx, nt, params, energy_floor=0.05):
    """b(theta) for every nominal row; params [B, n_params] -> b [B, m]."""
    params = np.atleast_2d(np.asarray(params, np.float64))
    Bn = params.shape[0]
    dx = 1.0 / nx
    t = time_grid(nt)
    g = params[:, :nx]
    r = params[:, nx]
    M = dx * g.sum(axis=1)
    E0 = dx * (g * g).sum(axis=1)
    Ek = np.maximum(E0[:, None] * np.exp(-r[:, None] * t[None, :]), (M * M + energy_floor)[:, None])
    parts = [g, np.repeat(M[:, None], nt, axis=1), Ek]
    if family == "B":
        parts.append(params[:, nx + 1:nx + 1 + nt])
    b = np.concatenate(parts, axis=1)
    assert b.shape == (Bn, nx + (3 if family == "B" else 2) * nt)
    return b


def grad_params_1d(family, nx, nt, params, badj, energy_floor=0.05):
    """dL/dtheta = -badj^T dh/dtheta = badj^T db/dtheta (h = ... - b), per sample.

    Only active rows carry a nonzero multiplier adjoint; badj [B, m] is the lambda-part of
    the adjoint solution K [a; badj] = [gbar; 0].  At the max() in E_k the exp branch is
    taken when E0 exp(-r t_k) >= M^2 + floor.
    """
    params = np.atleast_2d(np.asarray(params, np.float64))
    badj = np.atleast_2d(np.asarray(badj, np.float64))
    dx = 1.0 / nx
    t = time_grid(nt)
    g = params[:, :nx]
    r = params[:, nx]
    M = dx * g.sum(axis=1)
    E0 = dx * (g * g).sum(axis=1)
    b_ic = badj[:, :nx]
    b_m = badj[:, nx:nx + nt]
    b_e = badj[:, nx + nt:nx + 2 * nt]
    expo = np.exp(-r[:, None] * t[None, :])
    exp_branch = E0[:, None] * expo >= (M * M + energy_floor)[:, None]
    out = np.zeros_like(params)
    # d b_IC,i / d g_i = 1 ; d M / d g_i = dx
    out[:, :nx] = b_ic + dx * b_m.sum(axis=1)[:, None]
    # energy rows: exp branch  dE_k/dg_i = 2 dx g_i exp(-r t_k), dE_k/dr = -t_k E0 exp(-r t_k)
    #              floor branch dE_k/dg_i = 2 M dx
    we = np.where(exp_branch, b_e * expo, 0.0).sum(axis=1)
    wf = np.where(exp_branch, 0.0, b_e).sum(axis=1)
    out[:, :nx] += 2.0 * dx * g * we[:, None] + (2.0 * M * dx * wf)[:, None]
    out[:, nx] = np.where(exp_branch, -b_e * t[None, :] * E0[:, None] * expo, 0.0).sum(axis=1)
    if family == "B":
        out[:, nx + 1:nx + 1 + nt] = badj[:, nx + 2 * nt:nx + 3 * nt]
    return out


# ----------------------------------------------------------------------------------------
# 2-D family C
# ----------------------------------------------------------------------------------------

DROPPED_CELLS_2D = ((0, 0), (1, 0), (0, 1), (1, 1))     # (i, j), one per parity class


def structure_bc(nx, nt):
    """Boundary-condition regime of the Burgers problem (Appendix A, discretisation of
    Appendix D): x_i = i dx on [0, 1], dx = 1 / (nx - 1); per slice k a Dirichlet row
    u_{k,0} - u_L, a mass row dx sum_i u_{k,i} - m0 (Riemann sum) and a Neumann row
    u_{k,nx-1} - u_{k,nx-2}; rows grouped by type, all active."""
    assert nx >= 4 and nt >= 1
    dx = 1.0 / (nx - 1)
    empty = ([], [])
    arows, qrows, types = [], [], []
    for k in range(nt):
        arows.append(([k * nx], [1.0])); qrows.append(empty); types.append(ROW_DIRICHLET)
    for k in range(nt):
        arows.append((list(range(k * nx, (k + 1) * nx)), [dx] * nx)); qrows.append(empty)
        types.append(ROW_MASS)
    for k in range(nt):
        arows.append(([k * nx + nx - 2, k * nx + nx - 1], [-1.0, 1.0])); qrows.append(empty)
        types.append(ROW_NEUMANN)
    m = len(types)
    ap, ac, av = _csr(arows, m)
    qp, qc, qv = _csr(qrows, m)
    return Structure("D", nx * nt, m, ap, ac, av, qp, qc, qv, np.ones(m, np.uint8),
                     np.asarray(types, np.int32), dict(nx=nx, nt=nt))


def rhs_bc(nx, nt, params):
    """b for every row: params [B, 2] = (u_L, m0) -> b [B, 3 nt]."""
    params = np.atleast_2d(np.asarray(params, np.float64))
    Bn = params.shape[0]
    return np.concatenate([np.repeat(params[:, 0:1], nt, axis=1),
                           np.repeat(params[:, 1:2], nt, axis=1), np.zeros((Bn, nt))], axis=1)


def structure_2d(N, nt):
    """Rows of family "C": divergence (central differences) and kinetic energy per frame."""
    assert N >= 4 and N % 2 == 0 and nt >= 2
    dx = 1.0 / N
    nf = 2 * N * N
    inv2dx = 1.0 / (2.0 * dx)
    empty = ([], [])
    arows, qrows, types, active = [], [], [], []
    for f in range(nt):
        base = f * nf
        for j in range(N):
            for i in range(N):
                cols = [base + j * N + (i + 1) % N, base + j * N + (i - 1) % N,
                        base + N * N + ((j + 1) % N) * N + i, base + N * N + ((j - 1) % N) * N + i]
                vals = [inv2dx, -inv2dx, inv2dx, -inv2dx]
                arows.append((cols, vals)); qrows.append(empty)
                types.append(ROW_DIV)
                active.append(0 if (i, j) in DROPPED_CELLS_2D else 1)
    for f in range(nt):
        arows.append(empty)
        qrows.append((list(range(f * nf, (f + 1) * nf)), [0.5 * dx * dx] * nf))
        types.append(ROW_KE); active.append(1)
    m = len(types)
    ap, ac, av = _csr(arows, m)
    qp, qc, qv = _csr(qrows, m)
    return Structure("C", nf * nt, m, ap, ac, av, qp, qc, qv,
                     np.asarray(active, np.uint8), np.asarray(types, np.int32),
                     dict(N=N, nt=nt))


def rhs_2d(N, nt, params):
    """params [B, 2] = (K0, r2): divergence rows b = 0, energy rows b = K0 exp(-r2 t_f)."""
    params = np.atleast_2d(np.asarray(params, np.float64))
    t = time_grid(nt)
    K = params[:, 0:1] * np.exp(-params[:, 1:2] * t[None, :])
    return np.concatenate([np.zeros((params.shape[0], nt * N * N)), K], axis=1)


def grad_params_2d(N, nt, params, badj):
    params = np.atleast_2d(np.asarray(params, np.float64))
    t = time_grid(nt)
    e = np.exp(-params[:, 1:2] * t[None, :])
    b_e = np.atleast_2d(badj)[:, nt * N * N:]
    out = np.zeros_like(params)
    out[:, 0] = (b_e * e).sum(axis=1)
    out[:, 1] = (b_e * (-t[None, :]) * params[:, 0:1] * e).sum(axis=1)
    return out


# ----------------------------------------------------------------------------------------
# Appendix C toy family (pins the row / pattern builder)
# ----------------------------------------------------------------------------------------

def structure_toy(nx, nt):
    """IC rows u_i^(1) - f_i, then sum_{i<nx} u_i^(k) - sum_{i<nx} u_i^(1), k = 2..nt."""
    empty = ([], [])
    arows, qrows, types = [], [], []
    for i in range(nx):
        arows.append(([i], [1.0])); qrows.append(empty); types.append(ROW_IC)
    for k in range(1, nt):
        cols = list(range(nx - 1)) + [k * nx + i for i in range(nx - 1)]
        vals = [-1.0] * (nx - 1) + [1.0] * (nx - 1)
        arows.append((cols, vals)); qrows.append(empty); types.append(ROW_TOYMASS)
    m = len(types)
    ap, ac, av = _csr(arows, m)
    qp, qc, qv = _csr(qrows, m)
    return Structure("toy", nx * nt, m, ap, ac, av, qp, qc, qv,
                     np.ones(m, np.uint8), np.asarray(types, np.int32), dict(nx=nx, nt=nt))


# ----------------------------------------------------------------------------------------
# Evaluation helpers (residuals, per-type constraint error)
# ----------------------------------------------------------------------------------------

def eval_h(S, u, b):
    """h(u) for every nominal row; u [B, n], b [B, m] -> [B, m]."""
    import scipy.sparse as sp
    u = np.atleast_2d(np.asarray(u, np.float64))
    A = sp.csr_matrix((S.a_val, S.a_col, S.a_ptr), shape=(S.m, S.n))
    Q = sp.csr_matrix((S.q_val, S.q_col, S.q_ptr), shape=(S.m, S.n))
    return (A @ u.T + Q @ (u * u).T).T - np.atleast_2d(b)


def constraint_error(S, h):
    """Per-type mean Euclidean norm of the residual over the batch (Additional Results,
    eq. constraint_error): E_k = (1/N_s) sum_n ||R_k(u^(n))||_2."""
    h = np.atleast_2d(h)
    out = {}
    for t in np.unique(S.row_type):
        sel = S.row_type == t
        out[ROW_TYPE_NAMES[int(t)]] = float(np.mean(np.linalg.norm(h[:, sel], axis=1)))
    return out
