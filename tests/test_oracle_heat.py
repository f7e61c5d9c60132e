"""Pins of the heat-equation oracle (oracle/heat.py: IC, mass, Crank-Nicolson PDE residual and
energy-evolution rows, Crank-Nicolson discretisation) against what the mathematics fixes: the closed-form
Crank-Nicolson decay of a single Fourier mode, the implied mass and energy rows (summation by
parts), the generic dense Newton-KKT on the same active rows, stationarity with a
finite-difference Jacobian, and central differences of the adjoint."""
import numpy as np
import pytest

from oracle import heat, problems, solve


def _params(seed, B, nx, alpha=None):
    rng = np.random.default_rng(seed)
    x = np.arange(nx) * (2.0 * np.pi / nx)
    phi = rng.uniform(0.0, np.pi, size=B)
    g = np.sin(x[None, :] + phi[:, None]) + 0.1 * rng.normal(size=(B, nx))
    a = rng.uniform(1.0, 5.0, size=B) if alpha is None else np.full(B, alpha)
    return np.concatenate([g, a[:, None]], axis=1)


@pytest.mark.parametrize("nx,nt,p,alpha", [(100, 100, 1, 3.7), (16, 9, 3, 1.2), (12, 5, 6, 5.0)])
def test_single_mode_closed_form(nx, nt, p, alpha):
    """g = sin(p x + phase): each Crank-Nicolson step multiplies the mode by
    (1 - s) / (1 + s); the projection is that sequence for any u_hat."""
    uc = heat.cn_mode_solution(nx, nt, alpha, p, 0.3)
    pr = np.concatenate([uc[0], [alpha]])[None]
    uh = np.random.default_rng(1).normal(size=(1, nx * nt))
    u, lam, st = heat.project(nx, nt, pr, uh)
    np.testing.assert_allclose(u[0].reshape(nt, nx), uc, rtol=0, atol=1e-12)
    assert st["h_inf"][0] <= 1e-10


@pytest.mark.parametrize("nx,nt", [(100, 100), (20, 7)])
def test_mass_and_energy_rows_implied(nx, nt):
    """Mass and energy rows vanish at the IC + PDE solution (summation by parts), although
    they take no part in the solve; with the PDE rows perturbed they do not."""
    pr = _params(3, 2, nx)
    uh = np.random.default_rng(4).normal(size=(2, nx * nt))
    u, lam, st = heat.project(nx, nt, pr, uh)
    h = heat.eval_h(nx, nt, pr, u)
    ic, mass, pde, energy = heat.offsets(nx, nt)
    assert np.abs(h[:, mass:pde]).max() <= 1e-12
    assert np.abs(h[:, energy:]).max() <= 1e-9 * max(1.0, np.abs(u).max() ** 2 / heat.grid(nx, nt)[1])
    assert np.abs(h[:, pde:energy]).max() <= 1e-9
    np.testing.assert_array_equal(lam[:, mass:pde], 0.0)
    np.testing.assert_array_equal(lam[:, energy:], 0.0)
    # a field off the Crank-Nicolson solution violates the energy rows
    h2 = heat.eval_h(nx, nt, pr, u + 1e-3 * np.random.default_rng(5).normal(size=u.shape))
    assert np.abs(h2[:, energy:]).max() > 1e-6


def _structure_active(nx, nt, alpha):
    """The active rows (IC + PDE) in the generic oracle's row form (linear only)."""
    J = heat.jacobian_active(nx, nt, alpha).tocsr()
    n = nx * nt
    empty = np.zeros(n + 1, np.int32)
    return problems.Structure("heat", n, n, J.indptr.astype(np.int32), J.indices.astype(np.int32),
                              J.data.astype(np.float64), empty, np.zeros(0, np.int32),
                              np.zeros(0), np.ones(n, np.uint8), np.zeros(n, np.int32))


@pytest.mark.parametrize("nx,nt,seed", [(8, 5, 11), (6, 4, 12)])
def test_dense_newton_kkt_matches_definition(nx, nt, seed):
    pr = _params(seed, 2, nx)
    uh = np.random.default_rng(seed + 1).normal(size=(2, nx * nt))
    u, lam, st = heat.project(nx, nt, pr, uh)
    act = heat.active_rows(nx, nt).astype(bool)
    for b in range(2):
        S = _structure_active(nx, nt, pr[b, nx])
        rhs = np.zeros((1, nx * nt))
        rhs[0, :nx] = pr[b, :nx]
        ud, ld, sd = solve.project(S, rhs, uh[b:b + 1], tol_kkt=1e-12)
        assert sd["status"][0] == 0 and sd["iters"][0] <= 2
        np.testing.assert_allclose(ud[0], u[b], rtol=0, atol=1e-11)
        np.testing.assert_allclose(ld[0], lam[b, act], rtol=1e-9, atol=1e-9)


def test_stationarity_with_fd_jacobian():
    nx, nt = 6, 4
    pr = _params(21, 1, nx)
    uh = np.random.default_rng(22).normal(size=(1, nx * nt))
    u, lam, st = heat.project(nx, nt, pr, uh)
    n = nx * nt
    act = heat.active_rows(nx, nt).astype(bool)
    h = 1e-6
    Jfd = np.zeros((int(act.sum()), n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        Jfd[:, j] = ((heat.eval_h(nx, nt, pr, u + e) - heat.eval_h(nx, nt, pr, u - e)) / (2 * h))[0, act]
    grad = u[0] - uh[0] + Jfd.T @ lam[0, act]
    assert np.abs(grad).max() <= 1e-6 * max(1.0, np.abs(lam).max())


def test_adjoint_central_differences():
    nx, nt = 10, 6
    pr = _params(31, 2, nx)
    uh = np.random.default_rng(32).normal(size=(2, nx * nt))
    gbar = np.random.default_rng(33).normal(size=(2, nx * nt))
    u, lam, st = heat.project(nx, nt, pr, uh)
    a, gp = heat.adjoint(nx, nt, pr, u, gbar)
    assert np.all(a == 0.0)

    def loss(p, x):
        uu, _, _ = heat.project(nx, nt, p, x)
        return (uu * gbar).sum(axis=1)

    h = 1e-6
    for j in (0, 3, nx - 1, nx):
        pp, pm = pr.copy(), pr.copy()
        pp[:, j] += h
        pm[:, j] -= h
        fd = (loss(pp, uh) - loss(pm, uh)) / (2 * h)
        np.testing.assert_allclose(gp[:, j], fd, rtol=1e-6, atol=1e-8)
        assert np.all(np.abs(gp[:, j]) > 1e-4)
    d = np.random.default_rng(34).normal(size=uh.shape)
    np.testing.assert_allclose(loss(pr, uh + h * d) - loss(pr, uh - h * d), 0.0, atol=1e-12)


HEAT_MUTANTS = {
    "stencil_sign": ("cols.append(base + (i + 1) % nx); vals.append(-c)",
                     "cols.append(base + (i + 1) % nx); vals.append(c)"),
    "pde_row_half": ("h_pde = (cur - prev) / dt - 0.5 * alpha", "h_pde = (cur - prev) / dt - alpha"),
    "adjoint_ic_sign": ("gp[b, :nx] = bl[:nx]", "gp[b, :nx] = -bl[:nx]"),
    "energy_dissipation_factor": ("alpha[:, None] * dx * (_dplus", "alpha[:, None] * 2 * dx * (_dplus"),
}


@pytest.mark.parametrize("name", sorted(HEAT_MUTANTS))
def test_planted_mistake_in_heat_oracle_fails_a_pin(name, monkeypatch, tmp_path):
    """A plausible slip planted in a copy of oracle/heat.py makes at least one pin fail."""
    import importlib.util
    import sys
    old, new = HEAT_MUTANTS[name]
    src = open(heat.__file__).read()
    assert src.count(old) == 1, name
    path = tmp_path / "heat_mutant.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("heat_mutant", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    monkeypatch.setattr(sys.modules[__name__], "heat", mod)
    pins = [lambda: test_single_mode_closed_form(16, 9, 3, 1.2),
            lambda: test_mass_and_energy_rows_implied(20, 7),
            lambda: test_dense_newton_kkt_matches_definition(8, 5, 11),
            test_stationarity_with_fd_jacobian, test_adjoint_central_differences]
    failed = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed >= 1, f"mutant {name} passed every pin"
