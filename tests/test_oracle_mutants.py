"""The pins are sensitive: a plausible slip planted in a copy of the oracle's C core
(compiled on the CPU, in a temporary directory) makes at least one pin fail."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import solve
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "kkt_dense.c")

MUTANTS = {
    "quadratic_jacobian_factor": ("F[j] += lam[k] * 2.0 * c->qv[p] * u[j];",
                                  "F[j] += lam[k] * c->qv[p] * u[j];"),
    "linear_jacobian_sign": ("F[j] += lam[k] * c->av[p];", "F[j] -= lam[k] * c->av[p];"),
    "hessian_term_dropped": ("K[j * N + j] += lam[k] * 2.0 * c->qv[p];", "(void)0;"),
    "kkt_block_transposed_value": ("K[rk * N + j] += Jrj;", "K[rk * N + j] += 2.0 * Jrj;"),
    "ldl_2x2_sign": ("f->L[i * N + k + 1] = (m2 * e11 - m1 * e21) / det;",
                     "f->L[i * N + k + 1] = (m2 * e11 + m1 * e21) / det;"),
    "adjoint_rhs_sign": ("for (int j = 0; j < nv; ++j) rhs[j] = gbar[j];",
                         "for (int j = 0; j < nv; ++j) rhs[j] = -gbar[j];"),
    "armijo_direction": ("for (int i = 0; i < N; ++i) Ft[i] = -F[i];",
                         "for (int i = 0; i < N; ++i) Ft[i] = -0.5 * F[i];"),
}

PINS = [
    lambda: pins.test_ldl_solve_and_inertia_match_numpy(60, 4),
    pins.test_linear_projection_random_dense_rows,
    pins.test_family_a_matches_closed_form_small_1d_workload,
    pins.test_family_b_reduces_to_family_a,
    pins.test_adjoint_family_a_against_closed_form_fd,
]


def _build_mutant(name, tmp):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = os.path.join(tmp, "m.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(tmp, "m.so")
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", path, "-o", lib, "-lm"])
    return lib


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, monkeypatch):
    tmp = tempfile.mkdtemp()
    try:
        libpath = _build_mutant(name, tmp)
        saved = solve._lib
        solve._lib = None
        monkeypatch.setattr(solve._build, "build", lambda force=False: libpath)
        failed = 0
        try:
            for pin in PINS:
                try:
                    pin()
                except (AssertionError, RuntimeError, np.linalg.LinAlgError):
                    failed += 1
        finally:
            solve._lib = saved
        assert failed >= 1, f"mutant {name} passed every pin"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
