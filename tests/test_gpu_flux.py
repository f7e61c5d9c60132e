"""GPU parity of family E (Burgers IC + mass + Godunov flux rows) against the oracle's KKT point
(forward Godunov steps, dense stationarity solve) and its adjoint."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

from oracle import flux
from paper_2607_00095_b300 import Problem, _abi, synthetic
from tests import gpu_helpers as H


pytestmark = pytest.mark.gpu


def _types(nx, nt, K):
    return SimpleNamespace(row_type=flux.row_types(nx, nt, K))


def _check(nx, nt, K, B, seed, g_shift=0.0):
    uh, g = synthetic.gen_burgers_flux(seed, B, nx, nt)
    g = g + g_shift
    p = Problem("E", nx, nt, n_flux=K)
    u, lam, st, d = H.run_gpu(p, uh, g)
    assert (st["status"] == 0).all() and st["h_inf"].max() <= 1e-12
    assert (st["iters"] == 1).all()
    ue, le, so = flux.project(nx, nt, K, g, uh.reshape(B, -1))
    H.assert_u_close(u, ue)
    # the time chain rounds each step as the oracle does: the same bits
    np.testing.assert_array_equal(u[:, :(K + 1) * nx], ue[:, :(K + 1) * nx])
    H.assert_lam_close(_types(nx, nt, K), lam, le)
    np.testing.assert_allclose(st["obj"], so["obj"], rtol=1e-10)
    h, hinf = p.residual(d["u"], d["pr"])
    torch.cuda.synchronize()
    he = flux.eval_h(nx, nt, K, g, u)
    np.testing.assert_allclose(h.cpu().numpy(), he, rtol=0, atol=1e-13)
    assert hinf.cpu().numpy().max() <= 1e-12
    return p, u, lam, st, d, uh, g


# dt/dx <= 1 (the paper's 101 x 101 grid has dt/dx = 1) except for single steps: beyond the
# CFL limit the Godunov chain grows by up to 2 dt/dx per step and ||h|| grows with it
@pytest.mark.parametrize("nx,nt,K,B,seed", [
    (12, 7, 1, 3, 90),        # one flux step, dt/dx = 11/6
    (41, 41, 5, 4, 91),       # Flux(5), dt/dx = 1
    (101, 101, 10, 3, 92),    # Flux(10) on the paper's grid
    (20, 37, 36, 2, 93),      # K = nt - 1: no mass slices
    (9, 64, 3, 9, 94),        # B not a multiple of the chain block's four samples
    (3, 2, 1, 2, 95),         # smallest grid
    (512, 512, 2, 2, 96),     # largest nx
    (128, 160, 40, 2, 97),    # a long chain
    (300, 400, 9, 2, 98)])    # 8 values per lane of the chain kernel
def test_flux_against_oracle(nx, nt, K, B, seed):
    _check(nx, nt, K, B, seed)


def test_flux_signed_data():
    """Data of both signs (transonic rarefactions, left- and right-moving shocks)."""
    nx, nt, K, B = 40, 45, 6, 3
    uh, _ = synthetic.gen_burgers_flux(97, B, nx, nt)
    g = np.random.default_rng(98).uniform(-1, 1, size=(B, nx))
    p = Problem("E", nx, nt, n_flux=K)
    u, lam, st, d = H.run_gpu(p, uh, g)
    assert (st["status"] == 0).all()
    ue, le, _ = flux.project(nx, nt, K, g, uh.reshape(B, -1))
    np.testing.assert_array_equal(u[:, :(K + 1) * nx], ue[:, :(K + 1) * nx])
    H.assert_u_close(u, ue)
    H.assert_lam_close(_types(nx, nt, K), lam, le)


@pytest.mark.parametrize("K", [5, 10])
def test_flux_full_size_sampled(K):
    """The Burgers IC sizes: nx = nt = 101, B = 512, Flux(5) and Flux(10)."""
    w = synthetic.WORKLOADS["burgers_flux_1d"]
    B, nx, nt = w["B"], w["nx"], w["nt"]
    uh, g = synthetic.gen_burgers_flux(w["seed"], B, nx, nt)
    p = Problem("E", nx, nt, n_flux=K)
    u, lam, st, d = H.run_gpu(p, uh, g)
    assert (st["status"] == 0).all() and st["h_inf"].max() <= 1e-12
    pick = [0, 255, 511]
    ue, le, _ = flux.project(nx, nt, K, g[pick], uh[pick].reshape(len(pick), -1))
    H.assert_u_close(u[pick], ue)
    H.assert_lam_close(_types(nx, nt, K), lam[pick], le)


def test_flux_batch_independence_and_nan():
    nx, nt, K, B = 10, 24, 3, 6
    uh, g = synthetic.gen_burgers_flux(99, B, nx, nt)
    p = Problem("E", nx, nt, n_flux=K)
    u, lam, st, _ = H.run_gpu(p, uh, g)
    perm = np.array([3, 0, 5, 1, 4, 2])
    up, lp, sp, _ = H.run_gpu(p, uh[perm], g[perm])
    np.testing.assert_array_equal(up, u[perm])
    np.testing.assert_array_equal(lp, lam[perm])
    uh2 = uh.copy()
    uh2[2, 1, 4] = np.nan          # a chain slice
    uh2[4, 18, 0] = np.nan         # a mass slice
    u2, _, st2, _ = H.run_gpu(p, uh2, g)
    assert st2["status"][2] == 3 and st2["status"][4] == 3
    ok = [0, 1, 3, 5]
    assert (st2["status"][ok] == 0).all()
    np.testing.assert_array_equal(u2[ok], u[ok])


def test_flux_adjoint_against_oracle_and_fd():
    nx, nt, K, B = 9, 16, 3, 3
    uh, g = synthetic.gen_burgers_flux(100, B, nx, nt)
    g = g + 0.05                   # flux arguments away from the switches of F
    gbar = synthetic.gen_gbar(101, (B, nx * nt))
    p = Problem("E", nx, nt, n_flux=K)
    u, lam, st, d = H.run_gpu(p, uh, g)
    gh, gp = p.backward(H.to_dev(gbar), d["u"], d["lam"], d["pr"], stats=d["st"])
    torch.cuda.synchronize()
    gh, gp = gh.cpu().numpy(), gp.cpu().numpy()
    # the oracle's adjoint at the oracle's own solution of the same inputs
    ue, _, _ = flux.project(nx, nt, K, g, uh.reshape(B, -1))
    a, gge, _ = flux.adjoint(nx, nt, K, g, ue, gbar)
    np.testing.assert_allclose(gh, a, rtol=0, atol=1e-13 * max(1.0, np.abs(a).max()))
    np.testing.assert_allclose(gp, gge, rtol=1e-10, atol=1e-12)
    e = 1e-6

    def loss(gg, x):
        uu, _, _, _ = H.run_gpu(p, x, gg)
        return (uu * gbar).sum(axis=1)

    for i in range(0, nx, 3):
        dg = np.zeros_like(g)
        dg[:, i] = e
        np.testing.assert_allclose((loss(g + dg, uh) - loss(g - dg, uh)) / (2 * e), gp[:, i],
                                   rtol=1e-6, atol=1e-8)
    rng = np.random.default_rng(10)
    for _ in range(3):
        dr = rng.normal(size=uh.shape)
        fd = (loss(g, uh + e * dr) - loss(g, uh - e * dr)) / (2 * e)
        np.testing.assert_allclose(fd, (gh * dr.reshape(B, -1)).sum(axis=1), rtol=1e-6, atol=1e-8)


def test_flux_adjoint_nan_for_failed_samples():
    nx, nt, K, B = 6, 10, 2, 3
    uh, g = synthetic.gen_burgers_flux(102, B, nx, nt)
    uh[1, 4, 3] = np.nan
    gbar = synthetic.gen_gbar(103, (B, nx * nt))
    p = Problem("E", nx, nt, n_flux=K)
    u, lam, st, d = H.run_gpu(p, uh, g)
    assert st["status"][1] == 3
    gh, gp = p.backward(H.to_dev(gbar), d["u"], d["lam"], d["pr"], stats=d["st"])
    torch.cuda.synchronize()
    gh, gp = gh.cpu().numpy(), gp.cpu().numpy()
    assert np.isnan(gh[1]).all() and np.isnan(gp[1]).all()
    assert np.isfinite(gh[[0, 2]]).all() and np.isfinite(gp[[0, 2]]).all()


def test_flux_rejects_u0():
    nx, nt, K, B = 8, 4, 1, 2
    uh, g = synthetic.gen_burgers_flux(104, B, nx, nt)
    p = Problem("E", nx, nt, n_flux=K)
    with pytest.raises(_abi.SnapError):
        H.run_gpu(p, uh, g, u0=uh + 0.1)


def test_flux_two_shards_equal_one_batch():
    """The samples shard across ranks with no exchange: two halves projected apart give the
    bits of the whole batch (outputs and statistics)."""
    nx, nt, K, B = 33, 40, 5, 10
    uh, g = synthetic.gen_burgers_flux(105, B, nx, nt)
    p = Problem("E", nx, nt, n_flux=K)
    u, lam, st, _ = H.run_gpu(p, uh, g)
    parts = [H.run_gpu(p, uh[s], g[s]) for s in (slice(0, 3), slice(3, B))]
    np.testing.assert_array_equal(np.concatenate([q[0] for q in parts]), u)
    np.testing.assert_array_equal(np.concatenate([q[1] for q in parts]), lam)
    for key in ("status", "iters", "h_inf", "obj"):
        np.testing.assert_array_equal(np.concatenate([q[2][key] for q in parts]), st[key])
