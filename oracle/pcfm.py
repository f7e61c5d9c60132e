"""The PCFM sampling loop around the projection -- TEST INFRASTRUCTURE ONLY.

Three-step variant of the Sampling section (Eqs. 1-3): for tau = k / N, k = 0 .. N-1,
  forward shoot   u_hat_1 = u_tau + (1 - tau) v(u_tau, tau)
  projection      u_1 = argmin 1/2 ||u - u_hat_1||^2  s.t.  h(u) = 0
  OT pull-back    u_tau' = u_0 + tau' (u_1 - u_0)
with the analytic velocity v(u, tau) = (x1 - u0) + sigma0 (1 - tau) xi standing in for the
trained flow model (the straight-path OT velocity from the prior sample to a data sample,
plus a decaying perturbation).  The projection is passed in (the oracle's dense Newton-KKT,
a closed form, ...).
"""
import numpy as np


def velocity(u, tau, u0, x1, xi, sigma0):
    """The analytic stand-in for v_theta(u, tau)."""
    return (x1 - u0) + sigma0 * (1.0 - tau) * xi


def sample(project, u0, x1, xi, n_steps, sigma0):
    """One sampling pass; project(u_hat) -> (u, lam, stats).  Returns the last projection."""
    u0 = np.asarray(u0, np.float64)
    u1 = lam = st = None
    u_tau = u0
    for k in range(n_steps):
        tau = k / n_steps
        u_hat1 = u_tau + (1.0 - tau) * velocity(u_tau, tau, u0, x1, xi, sigma0)   # Eq. 1
        u1, lam, st = project(u_hat1)                                            # Eq. 2
        tau_next = (k + 1) / n_steps
        u_tau = u0 + tau_next * (u1 - u0)                                        # Eq. 3
    return u1, lam, st
