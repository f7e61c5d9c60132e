"""Closed forms and brute force used to pin the oracle (test code, independent of it).

Family A, slice k >= 1 (mass plane intersected with the energy sphere):
    dx sum_i u_i = M,  dx sum_i u_i^2 = E_k.
Write u = mu 1 + v with v orthogonal to 1.  With nx dx = 1 the first row gives mu = M and
the second ||v||^2 = (E_k - M^2)/dx =: rho^2.  The nearest point to u_hat is
    u* = M 1 + rho w / ||w||,   w = u_hat - mean(u_hat) 1,
and stationarity (1 + 2 dx lam_e) u* = u_hat - lam_m dx 1 gives
    alpha = 1 + 2 dx lam_e = ||w|| / rho,   lam_m = (mean(u_hat) - alpha M) / dx.
Slice 0 (IC rows only): u* = g, lam_IC = u_hat_0 - g.
"""
import numpy as np


def family_a_closed_form(nx, nt, params, u_hat, energy_floor=0.05):
    params = np.atleast_2d(params)
    u_hat = np.asarray(u_hat).reshape(params.shape[0], nt, nx)
    B = params.shape[0]
    dx = 1.0 / nx
    t = np.arange(nt) / (nt - 1)
    u = np.empty_like(u_hat)
    lam = np.zeros((B, nx + 2 * nt))
    for b in range(B):
        g = params[b, :nx]
        r = params[b, nx]
        M = dx * g.sum()
        E0 = dx * (g * g).sum()
        u[b, 0] = g
        lam[b, :nx] = u_hat[b, 0] - g
        for k in range(1, nt):
            Ek = max(E0 * np.exp(-r * t[k]), M * M + energy_floor)
            rho = np.sqrt((Ek - M * M) / dx)
            mean = u_hat[b, k].mean()
            w = u_hat[b, k] - mean
            nw = np.linalg.norm(w)
            u[b, k] = M + rho * w / nw
            alpha = nw / rho
            lam[b, nx + k] = (mean - alpha * M) / dx
            lam[b, nx + nt + k] = (alpha - 1.0) / (2.0 * dx)
    return u.reshape(B, -1), lam


def linear_projection(A, b, u_hat):
    """u = u_hat - A^T (A A^T)^{-1} (A u_hat - b) and lam = (A A^T)^{-1}(A u_hat - b)."""
    y = np.linalg.solve(A @ A.T, A @ u_hat - b)
    return u_hat - A.T @ y, y


def brute_force_b_nx4(u_hat4, M, E, c, n_theta=200000):
    """Global minimum of 1/2||u - u_hat||^2 on {dx sum u = M, dx sum u^2 = E,
    u_0^2 + u_2^2 = c} for nx = 4 (dx = 1/4): the feasible set is a curve, parametrised by
    u_0 = sqrt(c) cos th, u_2 = sqrt(c) sin th, u_1 + u_3 = s, u_1^2 + u_3^2 = q,
    u_1 - u_3 = +-sqrt(2q - s^2).  Grid search then golden-section refinement.
    Returns the list of local minima (objective, u) sorted by objective."""
    dx = 0.25
    sc = np.sqrt(c)

    def points(th, sign):
        u0 = sc * np.cos(th)
        u2 = sc * np.sin(th)
        s = M / dx - u0 - u2
        q = E / dx - c
        disc = 2 * q - s * s
        ok = disc >= 0
        d = sign * np.sqrt(np.where(ok, disc, 0.0))
        u1 = (s + d) / 2
        u3 = (s - d) / 2
        U = np.stack([u0, u1, u2, u3], axis=-1)
        f = 0.5 * np.sum((U - u_hat4) ** 2, axis=-1)
        return np.where(ok, f, np.inf), U

    th = np.linspace(0, 2 * np.pi, n_theta, endpoint=False)
    mins = []
    for sign in (1.0, -1.0):
        f, _ = points(th, sign)
        for i in range(n_theta):
            fl, fc, fr = f[i - 1], f[i], f[(i + 1) % n_theta]
            if np.isfinite(fc) and fc <= fl and fc <= fr and (fc < fl or fc < fr):
                a, bb = th[i] - 2 * np.pi / n_theta, th[i] + 2 * np.pi / n_theta
                gr = (np.sqrt(5) - 1) / 2
                for _ in range(200):
                    x1 = bb - gr * (bb - a)
                    x2 = a + gr * (bb - a)
                    if points(np.array(x1), sign)[0] < points(np.array(x2), sign)[0]:
                        bb = x2
                    else:
                        a = x1
                thm = 0.5 * (a + bb)
                fm, Um = points(np.array(thm), sign)
                mins.append((float(fm), np.asarray(Um)))
    mins.sort(key=lambda z: z[0])
    return mins
