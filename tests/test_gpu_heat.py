"""GPU parity of family F (heat equation: IC, mass, Crank-Nicolson PDE residual and
energy-evolution rows) against the oracle (oracle/heat.py), through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import heat
from paper_2607_00095_b300 import Problem, _abi, synthetic
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _types(nx, nt):
    ic, mass, pde, energy = heat.offsets(nx, nt)
    m = heat.sizes(nx, nt)[1]
    return {"ic": slice(ic, mass), "mass": slice(mass, pde), "pde": slice(pde, energy),
            "energy": slice(energy, m)}


def _assert_lam(nx, nt, lam, le):
    for name, sl in _types(nx, nt).items():
        for s in range(lam.shape[0]):
            den = max(np.abs(le[s, sl]).max(), 1e-12)
            err = np.abs(lam[s, sl] - le[s, sl]).max() / den
            assert err <= H.LAM_RTOL, f"sample {s} {name}: lambda rel err {err:.3e}"


def _run(nx, nt, uh, pr):
    p = Problem("F", nx, nt)
    u, lam, st, d = H.run_gpu(p, uh, pr)
    return p, u, lam, st, d


@pytest.mark.parametrize("B,nx,nt,seed", [(3, 100, 100, 31), (5, 33, 7, 32), (2, 3, 2, 33),
                                          (4, 64, 9, 34), (1, 128, 20, 35), (6, 17, 40, 36),
                                          (2, 256, 5, 37), (1, 512, 3, 38)])
def test_heat_parity(B, nx, nt, seed):
    uh, pr = synthetic.gen_heat(seed, B, nx, nt)
    p, u, lam, st, d = _run(nx, nt, uh, pr)
    ue, le, so = heat.project(nx, nt, pr, uh)
    np.testing.assert_array_equal(st["status"], 0)
    H.assert_u_close(u, ue)
    _assert_lam(nx, nt, lam, le)
    assert st["h_inf"].max() <= H.H_TOL
    # the time chain runs in double-float (relative rounding ~2^-47 per operation); a PDE row
    # scales a rounding of u^k by up to (1 + 4 kappa) / dt
    dt, dx = 1.0 / (nt - 1), 2.0 * np.pi / nx
    kap = pr[:, nx] * dt / (2.0 * dx * dx)
    tol_h = 1e-10 + 16 * 2.0 ** -47 * (1.0 + 4.0 * kap) / dt * np.abs(ue).max(axis=1)
    assert (np.abs(st["h_inf"] - so["h_inf"]) <= tol_h).all()
    np.testing.assert_allclose(st["obj"], 0.5 * ((ue - uh.reshape(B, -1)) ** 2).sum(axis=1),
                               rtol=1e-10)
    # residual entry point against the oracle's rows
    h, hinf = p.residual(d["u"], d["pr"])
    np.testing.assert_allclose(h.cpu().numpy(), heat.eval_h(nx, nt, pr, u), rtol=0, atol=1e-10)
    np.testing.assert_allclose(hinf.cpu().numpy(), np.abs(heat.eval_h(nx, nt, pr, u)).max(axis=1),
                               rtol=0, atol=1e-10)


def test_heat_full_size_sampled():
    """The heat problem's grid (100 x 100) at B = 512, as the bench runs it; 16 sampled
    samples against the oracle."""
    w = synthetic.WORKLOADS["heat2_1d"]
    B, nx, nt = w["B"], w["nx"], w["nt"]
    uh, pr = synthetic.gen_heat(w["seed"], B, nx, nt)
    p, u, lam, st, d = _run(nx, nt, uh, pr)
    np.testing.assert_array_equal(st["status"], 0)
    assert st["h_inf"].max() <= H.H_TOL
    pick = np.sort(np.random.default_rng(7).choice(B, size=16, replace=False))
    ue, le, so = heat.project(nx, nt, pr[pick], uh[pick])
    H.assert_u_close(u[pick], ue)
    _assert_lam(nx, nt, lam[pick], le)


def test_heat_edge_cases():
    nx, nt, B = 20, 6, 5
    uh, pr = synthetic.gen_heat(41, B, nx, nt)
    pr[0, nx] = 0.0                        # alpha = 0: u^k = g for every k
    pr[1, :nx] = 0.7                       # constant IC: u = 0.7 everywhere
    pr[2, nx] = -1.0                       # negative diffusion: infeasible parameters
    uh[3, 2, 5] = np.nan                   # non-finite target: u is unaffected, lambda is not
    p, u, lam, st, d = _run(nx, nt, uh, pr)
    U = u.reshape(B, nt, nx)
    assert st["status"][0] == 0 and np.all(U[0] == pr[0, :nx][None, :])
    assert st["status"][1] == 0
    # double-float chain: a few units of 2^-47 relative per step, over nt - 1 steps
    np.testing.assert_allclose(U[1], 0.7, rtol=0, atol=8 * (nt - 1) * 2.0 ** -47 * 0.7)
    assert st["status"][2] == 4
    assert st["status"][3] == 3
    ue, _, _ = heat.project(nx, nt, pr[3:4], np.nan_to_num(uh[3:4]))
    H.assert_u_close(u[3:4], ue)
    assert st["status"][4] == 0
    with pytest.raises(_abi.SnapError):
        Problem("F", 2, 4)                # nx < 3
    with pytest.raises(_abi.SnapError):
        Problem("F", 8, 4, rows=1)        # rows must be 0
    with pytest.raises(_abi.SnapError) as ei:
        p.project(d["uh"], d["pr"], u0=d["uh"] + 0.0)
    assert ei.value.code == 2


def test_heat_batch_permutation_and_shards():
    nx, nt, B = 24, 8, 7
    uh, pr = synthetic.gen_heat(51, B, nx, nt)
    _, u, lam, st, _ = _run(nx, nt, uh, pr)
    perm = np.random.default_rng(2).permutation(B)
    _, up, lp, sp, _ = _run(nx, nt, uh[perm], pr[perm])
    np.testing.assert_array_equal(up, u[perm])
    np.testing.assert_array_equal(lp, lam[perm])
    _, u1, l1, _, _ = _run(nx, nt, uh[:3], pr[:3])
    _, u2, l2, _, _ = _run(nx, nt, uh[3:], pr[3:])
    np.testing.assert_array_equal(np.concatenate([u1, u2]), u)
    np.testing.assert_array_equal(np.concatenate([l1, l2]), lam)


def test_heat_adjoint_against_oracle_and_fd():
    nx, nt, B = 12, 7, 3
    uh, pr = synthetic.gen_heat(61, B, nx, nt)
    gbar = synthetic.gen_gbar(62, (B, nx * nt))
    p, u, lam, st, d = _run(nx, nt, uh, pr)
    gh, gp = p.backward(H.to_dev(gbar), d["u"], d["lam"], d["pr"], stats=d["st"])
    torch.cuda.synchronize()
    gh, gp = gh.cpu().numpy(), gp.cpu().numpy()
    # the oracle's adjoint at the oracle's own solution of the same inputs
    ue, _, _ = heat.project(nx, nt, pr, uh)
    a, gpo = heat.adjoint(nx, nt, pr, ue, gbar)
    np.testing.assert_array_equal(gh, 0.0)
    H.assert_adjoint_close(gp, gpo)
    h = 1e-6

    def loss(prm, x):
        _, uu, _, _, _ = _run(nx, nt, x, prm)
        return (uu * gbar).sum(axis=1)

    for j in (0, 5, nx - 1, nx):
        pp, pm = pr.copy(), pr.copy()
        pp[:, j] += h
        pm[:, j] -= h
        fd = (loss(pp, uh) - loss(pm, uh)) / (2 * h)
        np.testing.assert_allclose(gp[:, j], fd, rtol=1e-5, atol=1e-8)
    # a failed forward sample gets NaN gradients
    st_bad = d["st"].clone()
    st_bad[1, 8:12] = torch.tensor(list((2).to_bytes(4, "little")), dtype=torch.uint8)
    gh2, gp2 = p.backward(H.to_dev(gbar), d["u"], d["lam"], d["pr"], stats=st_bad)
    torch.cuda.synchronize()
    assert np.isnan(gp2.cpu().numpy()[1]).all() and np.isfinite(gp2.cpu().numpy()[[0, 2]]).all()
