"""Seeded synthetic inputs for the projection workloads.

This module only draws problem data (targets u_hat, constraint parameters, upstream
gradients); it holds none of the projection's arithmetic.  Both the CUDA path and the
oracle consume the same bytes it produces.

The paper's own data (trained functional flow-matching models and their PDE datasets,
Appendix A) are not available, so these generators stand in for the flow model's
one-step extrapolation u_hat_1 of eq. (1): a smooth field plus i.i.d. Gaussian noise.

Workloads (name -> sizes):
  small_1d    family A, B=8,   nx=32,  nt=32   (IC + mass + energy), seed 1000
  burgers_1d  family B, B=512, nx=128, nt=100  (+ boundary invariant), seed 1001
  adjoint_1d  burgers_1d with an upstream gradient dL/du ~ N(0,1), seed 1002
  div_2d      family C, B=64,  N=64,   nt=16   (divergence + kinetic energy), seed 1003
  uneven      1024 instances: 75 % family B with nx in {64,96,128,192,256},
              nt in {50,100,200}; 25 % family C at 32x32x8; seed 1004
  pcfm_1d     burgers_1d shapes: data sample x1 = gen_1d's u_hat (seed 1005), prior sample
              u0 and perturbation xi ~ N(0, 1) (seed 1006), 10 steps, sigma0 = 0.3
  vorticity_2d  2-D vorticity (IC, total vorticity, enstrophy), B=512, 16x16, nt=50, seed 1007
  burgers_bc_1d  family D (Dirichlet, mass, Neumann per slice), B=512, nx=nt=101, seed 1008
  burgers_flux_1d  family E (IC, mass, Godunov flux rows), B=512, nx=nt=101, Flux(5), seed 1009
  heat2_1d    family F (IC, mass, Crank-Nicolson PDE residual, energy evolution), B=512,
              nx=nt=100 (the heat problem's grid), seed 1010
"""
import numpy as np

TWO_PI = 2.0 * np.pi


def grid_1d(nx, nt):
    """x_i = i/nx on the periodic unit interval, t_k = k/(nt-1) on [0, 1]."""
    return np.arange(nx, dtype=np.float64) / nx, np.arange(nt, dtype=np.float64) / (nt - 1)


def gen_1d(seed, B, nx, nt, family="B", noise=0.1, rate=0.5):
    """Per sample b: g(x) = sin(2 pi x) + 0.5 sin(4 pi x + phi_b), phi_b ~ U[0, 2 pi);
    u_hat = g(x) exp(-0.5 t) + N(0, noise^2) i.i.d.

    params[b] = [g(x_0..x_{nx-1}), rate, (c(t_0..t_{nt-1}) for family B)] where
    c(t) = u(0,t)^2 + u(1/2,t)^2 of the noiseless field g(x) exp(-0.5 t).
    Returns (u_hat [B, nt, nx], params [B, n_params]).
    """
    rng = np.random.default_rng(seed)
    x, t = grid_1d(nx, nt)
    phi = rng.uniform(0.0, TWO_PI, size=B)
    g = np.sin(TWO_PI * x)[None, :] + 0.5 * np.sin(2.0 * TWO_PI * x[None, :] + phi[:, None])
    u_hat = g[:, None, :] * np.exp(-0.5 * t)[None, :, None] + rng.normal(0.0, noise, size=(B, nt, nx))
    parts = [g, np.full((B, 1), rate)]
    if family == "B":
        ih = nx // 2
        c = (g[:, 0] ** 2 + g[:, ih] ** 2)[:, None] * np.exp(-t)[None, :]
        parts.append(c)
    params = np.ascontiguousarray(np.concatenate(parts, axis=1))
    return np.ascontiguousarray(u_hat), params


def gen_2d(seed, B, N, nt, noise=0.05, rate=0.2, kmax=8):
    """Per sample: one random streamfunction psi with Fourier modes 0 < |k| <= kmax and
    amplitude ~ |k|^-2 (complex normal), the velocity (u, v) = (D_y psi, -D_x psi) with
    2nd-order central differences, scaled to unit rms over all 2 N^2 components; every
    frame gets fresh N(0, noise^2) noise.  params[b] = [K0, rate] with
    K0 = 1/2 dx^2 ||w_psi||^2 of the noiseless field.
    Returns (w_hat [B, nt, 2, N, N] with [.., j, i] = (y, x), params [B, 2]).
    """
    rng = np.random.default_rng(seed)
    dx = 1.0 / N
    w_hat = np.empty((B, nt, 2, N, N))
    params = np.empty((B, 2))
    for b in range(B):
        spec = np.zeros((N, N), dtype=np.complex128)
        for p in range(-kmax, kmax + 1):
            for q in range(-kmax, kmax + 1):
                k2 = p * p + q * q
                if 0 < k2 <= kmax * kmax:
                    amp = 1.0 / k2                                 # |k|^-2
                    spec[q % N, p % N] = amp * (rng.normal() + 1j * rng.normal())
        psi = np.real(np.fft.ifft2(spec))
        u = (np.roll(psi, -1, axis=0) - np.roll(psi, 1, axis=0)) / (2 * dx)     # D_y psi
        v = -(np.roll(psi, -1, axis=1) - np.roll(psi, 1, axis=1)) / (2 * dx)    # -D_x psi
        s = np.sqrt(np.mean(np.concatenate([u.ravel(), v.ravel()]) ** 2))
        u, v = u / s, v / s
        params[b, 0] = 0.5 * dx * dx * (np.sum(u * u) + np.sum(v * v))
        params[b, 1] = rate
        w_hat[b, :, 0] = u[None] + rng.normal(0.0, noise, size=(nt, N, N))
        w_hat[b, :, 1] = v[None] + rng.normal(0.0, noise, size=(nt, N, N))
    return np.ascontiguousarray(w_hat), params


def gen_gbar(seed, shape):
    """Upstream gradient dL/du ~ N(0, 1), FP64."""
    return np.random.default_rng(seed).normal(0.0, 1.0, size=shape)


UNEVEN_NX = (64, 96, 128, 192, 256)
UNEVEN_NT = (50, 100, 200)


def gen_uneven(seed=1004, n_inst=1024, frac_1d=0.75, n2d=32, nt2d=8):
    """Uneven mix: a list of dicts {family, nx/N, nt, u_hat, params} drawn from one seed."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        s = int(rng.integers(0, 2 ** 31 - 1))
        if rng.uniform() < frac_1d:
            nx = int(rng.choice(UNEVEN_NX))
            nt = int(rng.choice(UNEVEN_NT))
            uh, pr = gen_1d(s, 1, nx, nt, "B")
            out.append(dict(family="B", nx=nx, nt=nt, u_hat=uh[0], params=pr[0]))
        else:
            wh, pr = gen_2d(s, 1, n2d, nt2d)
            out.append(dict(family="C", nx=n2d, nt=nt2d, u_hat=wh[0], params=pr[0]))
    return out


def gen_vorticity(seed, B, N, nt, noise=0.1, decay=0.02, alpha=2.5, tau=7.0):
    """2-D vorticity frames on a periodic N x N grid of [0, 1]^2, nt frames, flattened to
    N^2 values per frame (row j, column i at j N + i).  Per sample: an initial vorticity w_IC
    from a Gaussian random field with spectral amplitude (4 pi^2 |k|^2 + tau^2)^(-alpha/2)
    (zero mean, scaled to unit rms); candidate frames u_hat(t_k) = w_IC (1 - decay t_k) +
    N(0, noise^2) i.i.d. with t_k = k / (nt - 1).  params[b] = [w_IC (N^2 values), 0.0] (the
    family-A layout: IC values, then rate 0: total vorticity and enstrophy conserved).
    Returns (u_hat [B, nt, N^2], params [B, N^2 + 1])."""
    rng = np.random.default_rng(seed)
    k = np.fft.fftfreq(N, d=1.0 / N)
    k2 = k[None, :] ** 2 + k[:, None] ** 2
    amp = (4.0 * np.pi ** 2 * k2 + tau ** 2) ** (-alpha / 2.0)
    amp[0, 0] = 0.0
    t = np.arange(nt) / (nt - 1)
    u_hat = np.empty((B, nt, N * N))
    params = np.zeros((B, N * N + 1))
    for b in range(B):
        spec = amp * (rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N)))
        w = np.real(np.fft.ifft2(spec))
        w = w / np.sqrt(np.mean(w * w))
        params[b, :N * N] = w.ravel()
        u_hat[b] = w.ravel()[None, :] * (1.0 - decay * t)[:, None] + rng.normal(0.0, noise, size=(nt, N * N))
    return np.ascontiguousarray(u_hat), params


def gen_burgers_bc(seed, B, nx, nt, noise=0.1, eps=0.02):
    """Boundary-condition regime of the Burgers problem on [0, 1] (x_i = i / (nx - 1)),
    t_k = k / (nt - 1): per sample a front u_IC(x) = 1 / (1 + exp((x - p_loc) / eps)) with
    p_loc ~ U(0.2, 0.8), travelling at speed 1/2 (the inviscid Burgers shock speed between 1
    and 0), u_hat = u_IC(x - t / 2) + N(0, noise^2); params = [u_L, m0] with u_L ~ U(0, 1)
    and m0 = dx sum_i u_IC(x_i) (the mass of the initial profile, Riemann sum).
    Returns (u_hat [B, nt, nx], params [B, 2])."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx) / (nx - 1)
    t = np.arange(nt) / (nt - 1)
    dx = 1.0 / (nx - 1)
    p_loc = rng.uniform(0.2, 0.8, size=B)
    u_l = rng.uniform(0.0, 1.0, size=B)
    xx = x[None, None, :] - 0.5 * t[None, :, None] - p_loc[:, None, None]
    u_hat = 1.0 / (1.0 + np.exp(np.clip(xx / eps, -700, 700))) + rng.normal(0.0, noise, size=(B, nt, nx))
    u_ic = 1.0 / (1.0 + np.exp(np.clip((x[None, :] - p_loc[:, None]) / eps, -700, 700)))
    params = np.stack([u_l, dx * u_ic.sum(axis=1)], axis=1)
    return np.ascontiguousarray(u_hat), np.ascontiguousarray(params)


def gen_burgers_flux(seed, B, nx, nt, noise=0.1, eps=0.02):
    """IC regime of the Burgers problem on [0, 1] (x_i = i / (nx - 1), t_k = k / (nt - 1)):
    per sample the front u_IC(x) = 1 / (1 + exp((x - p_loc) / eps)), p_loc ~ U(0.2, 0.8),
    as the IC parameters g = u_IC(x_i), and u_hat = u_IC(x - t / 2) + N(0, noise^2) (the
    front at the Burgers shock speed 1/2).  Returns (u_hat [B, nt, nx], params [B, nx])."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx) / (nx - 1)
    t = np.arange(nt) / (nt - 1)
    p_loc = rng.uniform(0.2, 0.8, size=B)
    xx = x[None, None, :] - 0.5 * t[None, :, None] - p_loc[:, None, None]
    u_hat = 1.0 / (1.0 + np.exp(np.clip(xx / eps, -700, 700))) + rng.normal(0.0, noise, size=(B, nt, nx))
    g = 1.0 / (1.0 + np.exp(np.clip((x[None, :] - p_loc[:, None]) / eps, -700, 700)))
    return np.ascontiguousarray(u_hat), np.ascontiguousarray(g)


def gen_heat(seed, B, nx, nt, noise=0.1):
    """Heat problem on the periodic [0, 2 pi) (x_i = 2 pi i / nx, t_k = k / (nt - 1)): per
    sample the phase phi ~ U(0, pi) and the diffusion coefficient alpha ~ U(1, 5) (the
    distributions of the training set of the heat problem), IC g = sin(x_i + phi), and
    u_hat = exp(-alpha t) sin(x + phi) + N(0, noise^2): the analytic solution the flow model
    was trained on, perturbed.  Returns (u_hat [B, nt, nx], params [B, nx + 1] = [g, alpha])."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx) * (TWO_PI / nx)
    t = np.arange(nt) / (nt - 1)
    phi = rng.uniform(0.0, np.pi, size=B)
    alpha = rng.uniform(1.0, 5.0, size=B)
    g = np.sin(x[None, :] + phi[:, None])
    u_hat = (np.exp(-alpha[:, None, None] * t[None, :, None]) * g[:, None, :]
             + rng.normal(0.0, noise, size=(B, nt, nx)))
    params = np.concatenate([g, alpha[:, None]], axis=1)
    return np.ascontiguousarray(u_hat), np.ascontiguousarray(params)


def gen_pcfm(seed, B, nx, nt, family="B"):
    """Inputs of one PCFM sampling pass on a 1-D family: the data sample x1 and the
    parameters from gen_1d (seed), the prior sample u0 ~ N(0, 1) and the perturbation
    direction xi ~ N(0, 1) (seed + 1)."""
    x1, pr = gen_1d(seed, B, nx, nt, family)
    rng = np.random.default_rng(seed + 1)
    u0 = rng.normal(size=(B, nt * nx))
    xi = rng.normal(size=(B, nt * nx))
    return u0, x1.reshape(B, -1), xi, pr


WORKLOADS = {
    "small_1d": dict(family="A", B=8, nx=32, nt=32, seed=1000),
    "burgers_1d": dict(family="B", B=512, nx=128, nt=100, seed=1001),
    "adjoint_1d": dict(family="B", B=512, nx=128, nt=100, seed=1001, gbar_seed=1002),
    "div_2d": dict(family="C", B=64, N=64, nt=16, seed=1003),
    "uneven": dict(n_inst=1024, seed=1004),
    "pcfm_1d": dict(family="B", B=512, nx=128, nt=100, seed=1005, n_steps=10, sigma0=0.3),
    "vorticity_2d": dict(B=512, N=16, nt=50, seed=1007),
    "burgers_bc_1d": dict(B=512, nx=101, nt=101, seed=1008),
    "burgers_flux_1d": dict(B=512, nx=101, nt=101, n_flux=5, seed=1009),
    "heat2_1d": dict(B=512, nx=100, nt=100, seed=1010),
}
