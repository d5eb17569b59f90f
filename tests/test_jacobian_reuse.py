"""The Jacobian-reuse rule of the Newton loop (Section 5.3): the Jacobian of
problem (1) is assembled again only when the nonlinear convergence rate
rho_l = ||B - A(U^(l))||_inf / ||B - A(U^(l-1))||_inf exceeds gamma_nt.  Host
bookkeeping of the library (nmg_jacobian_reuse_*), exercised without a GPU on
residual sequences and on a small nonlinear problem whose Newton iteration
freezes its Jacobian when the rule says so."""

import ctypes as C

import numpy as np
import pytest


@pytest.fixture(scope="module")
def nmg():
    from paper_1904_02401_gb300 import nmg as lib
    return lib


def _decide(nmg, m, res):
    a = C.c_int(-1)
    assert nmg.nmg_jacobian_reuse_decide(m, res, a) == nmg.NMG_OK
    return a.value


def test_decisions_on_a_residual_sequence(nmg):
    m = nmg.nmg_jacobian_reuse()
    assert nmg.nmg_jacobian_reuse_init(m, 0.5) == nmg.NMG_OK
    # time step 1: no Jacobian yet -> assemble; rates 0.3 (reuse), 0.2/0.3 (assemble), 0.05 (reuse)
    got = [_decide(nmg, m, r) for r in (1.0, 0.3, 0.2, 0.01)]
    assert got == [1, 0, 1, 0]
    assert abs(m.rate - 0.05) < 1e-15
    # time step 2: its first step has no rate and reuses; 0.4 / 0.5 = 0.8 > 0.5 assembles
    assert nmg.nmg_jacobian_reuse_time_step(m) == nmg.NMG_OK
    assert _decide(nmg, m, 0.5) == 0 and m.rate == -1.0
    assert _decide(nmg, m, 0.4) == 1
    assert _decide(nmg, m, 0.2) == 0          # rate exactly 0.5: not above the threshold
    assert (m.steps, m.assemblies) == (7, 3)


def test_gamma_zero_assembles_every_step(nmg):
    m = nmg.nmg_jacobian_reuse()
    nmg.check(nmg.nmg_jacobian_reuse_init(m, 0.0))
    seq = []
    for step in range(3):
        nmg.check(nmg.nmg_jacobian_reuse_time_step(m))
        seq += [_decide(nmg, m, r) for r in (1.0, 1e-2, 1e-5)]
    assert seq == [1] * 9 and m.assemblies == 9


def test_invalid_arguments(nmg):
    m = nmg.nmg_jacobian_reuse()
    assert nmg.nmg_jacobian_reuse_init(m, -0.1) == nmg.NMG_ERR_INVALID
    assert nmg.nmg_jacobian_reuse_init(m, float("nan")) == nmg.NMG_ERR_INVALID
    assert nmg.nmg_jacobian_reuse_init(None, 0.2) == nmg.NMG_ERR_INVALID
    nmg.check(nmg.nmg_jacobian_reuse_init(m, 0.2))
    a = C.c_int()
    assert nmg.nmg_jacobian_reuse_decide(m, float("inf"), a) == nmg.NMG_ERR_NONFINITE
    assert nmg.nmg_jacobian_reuse_decide(m, -1.0, a) == nmg.NMG_ERR_NONFINITE
    assert nmg.nmg_jacobian_reuse_decide(m, 1.0, None) == nmg.NMG_ERR_INVALID


def _newton_run(nmg, gamma, steps=6):
    """Implicit Euler steps of u' = -(A u + u^3) + f (a stiff nonlinear system),
    each solved by Newton's method with the Jacobian I + k (A + 3 diag(u^2))
    assembled only when the rule asks; returns (Newton steps, assemblies, u)."""
    n = 40
    h = 1.0 / (n + 1)
    A = (np.diag(2 * np.ones(n)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)) / h ** 2
    k = 1e-2
    f = 500.0 * np.sin(np.pi * np.arange(1, n + 1) * h)
    u = np.zeros(n)
    m = nmg.nmg_jacobian_reuse()
    nmg.check(nmg.nmg_jacobian_reuse_init(m, gamma))
    J = None
    total = 0
    for _ in range(steps):
        u_old = u.copy()
        nmg.check(nmg.nmg_jacobian_reuse_time_step(m))
        for _ in range(200):
            res = u_old + k * (f - A @ u - u ** 3) - u
            rn = np.abs(res).max()
            if rn <= 1e-10:
                break
            if _decide(nmg, m, rn):
                J = np.eye(n) + k * (A + 3 * np.diag(u ** 2))
            u = u + np.linalg.solve(J, res)
            total += 1
        else:
            raise AssertionError("Newton did not converge")
    return total, int(m.assemblies), u


def test_reuse_trades_assemblies_for_newton_steps(nmg):
    """As in the paper's gamma study: gamma = 0 assembles at every Newton step;
    larger thresholds assemble less often and take at least as many Newton
    steps, and every run reaches the same solution."""
    runs = {g: _newton_run(nmg, g) for g in (0.0, 0.2, 0.5)}
    steps0, asm0, u0 = runs[0.0]
    assert asm0 == steps0
    assert runs[0.5][1] < runs[0.2][1] < asm0
    assert steps0 < runs[0.2][0] < runs[0.5][0]
    for g, (_, _, u) in runs.items():
        assert np.abs(u - u0).max() <= 1e-8 * np.abs(u0).max()
