"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and compare with the
oracle on the same seeded inputs.

Tolerances (the workload definition): u relative 1e-8 per sample,
||u_gpu - u_ora||_inf / ||u_ora||_inf; lambda relative 1e-6 per constraint type and sample,
||dlam_T||_inf / max(||lam_T||_inf, 1e-12); ||h||_inf <= 1e-8 over all nominal rows.
"""
import numpy as np
import torch

from oracle import problems
from paper_2607_00095_b300 import Problem, decode_stats, options

U_RTOL = 1e-8
LAM_RTOL = 1e-6
H_TOL = 1e-8
# Adjoint parity: GPU gradient against the oracle's dense adjoint, each at its own solution.
# The two solutions agree to the forward tolerances (both stop at ||F||_inf <= 1e-10, i.e.
# u to ~1e-10 relative and lambda to ~1e-8 relative at these problem scales); the adjoint is a
# smooth function of (u, lambda), so the gradients agree to a few times that (the oracle's
# own gradients at tol_kkt 1e-10 and 1e-14 differ by <= 2.1e-9 on the Burgers workload): per
# sample, ||g_gpu - g_ora||_inf <= 1e-7 max(||g_ora||_inf, 1).  Central differences (relative
# 1e-5) are checked separately.
ADJ_RTOL = 1e-7


def dev():
    return torch.device("cuda:0")


def to_dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev())


def run_gpu(prob, u_hat, params, u0=None, **opt):
    B = u_hat.shape[0]
    uh = to_dev(u_hat.reshape(B, -1))
    pr = to_dev(params)
    u0d = to_dev(u0.reshape(B, -1)) if u0 is not None else None
    u, lam, st = prob.project(uh, pr, u0=u0d, opts=options(**opt))
    torch.cuda.synchronize()
    return (u.cpu().numpy(), lam.cpu().numpy(), decode_stats(st),
            dict(uh=uh, pr=pr, u=u, lam=lam, st=st))


def assert_adjoint_close(g, ge, rtol=ADJ_RTOL):
    g = np.atleast_2d(g)
    ge = np.atleast_2d(ge)
    assert g.shape == ge.shape
    for s in range(g.shape[0]):
        den = max(np.abs(ge[s]).max(), 1.0)
        err = np.abs(g[s] - ge[s]).max() / den
        assert err <= rtol, f"sample {s}: adjoint rel err {err:.3e} > {rtol}"


def oracle_adjoint_1d(family, nx, nt, pr, uh, gbar, **kw):
    """The oracle's forward solution of (u_hat, params), then its dense adjoint there."""
    from oracle import solve
    ue, le, so, _, _ = solve.project_1d(family, nx, nt, pr, uh, nthreads=8, **kw)
    assert (so["status"] == 0).all(), so["status"]
    a, gp, _ = solve.adjoint_1d(family, nx, nt, pr, ue, le, gbar, nthreads=8)
    return a, gp


def assert_u_close(u, ue, rtol=U_RTOL):
    u = np.atleast_2d(u)
    ue = np.atleast_2d(ue)
    for s in range(u.shape[0]):
        den = max(np.abs(ue[s]).max(), 1e-300)
        err = np.abs(u[s] - ue[s]).max() / den
        assert err <= rtol, f"sample {s}: u rel err {err:.3e} > {rtol}"


def assert_lam_close(S, lam, le, rtol=LAM_RTOL):
    lam = np.atleast_2d(lam)
    le = np.atleast_2d(le)
    for t in np.unique(S.row_type):
        sel = S.row_type == t
        for s in range(lam.shape[0]):
            den = max(np.abs(le[s, sel]).max(), 1e-12)
            err = np.abs(lam[s, sel] - le[s, sel]).max() / den
            assert err <= rtol, f"sample {s} type {problems.ROW_TYPE_NAMES[int(t)]}: lam rel err {err:.3e}"
