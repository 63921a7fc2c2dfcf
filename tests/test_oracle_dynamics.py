"""Pins of the oracle's dynamics and RK4 (Eq. 1) against closed forms,
conservation laws and textbook equilibria -- none of them a retyped formula."""
import math
import os

import numpy as np
import pytest

from paper_2202_06111_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def _lin(A, B, dt, substeps):
    dyn = W.linmap(A, B)
    n = dyn["n"]
    return W.problem(dyn, [-1] * n, [1] * n, 1, 2, [[0.0] * dyn["m"]], dt, substeps)


@pytest.mark.parametrize("lam,dt,s", [(-1.0, 0.1, 1), (0.7, 0.3, 4), (-3.0, 0.05, 10), (2.5, 1.0, 3)])
def test_rk4_scalar_stability_polynomial(orc, lam, dt, s):
    """Classic RK4 on x' = lam x is x -> R(z)^s x, R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24,
    z = lam h. A wrong stage weight or stage step breaks the z^3 / z^4 terms."""
    p = _lin([[lam]], [[0.0]], dt, s)
    z = lam * dt / s
    R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    for x0 in (1.0, -0.375, 3.0):
        y = orc.step(p, [x0], [0.0])[0]
        assert y == pytest.approx(x0 * R ** s, rel=1e-14, abs=1e-300)


def test_rk4_matrix_polynomial_and_input(orc):
    """x' = A x + B u with a non-symmetric A (a transposed A or a dropped B u
    would fail): one RK4 step is x -> R(hA) x + h (I + hA/2 + (hA)^2/6 + (hA)^3/24) B u."""
    A = np.array([[0.0, 1.0], [-2.0, -0.5]])
    B = np.array([[0.0], [1.0]])
    h = 0.2
    p = _lin(A.tolist(), B.tolist(), h, 1)
    M = h * A
    I = np.eye(2)
    R = I + M + M @ M / 2 + M @ M @ M / 6 + M @ M @ M @ M / 24
    Q = h * (I + M / 2 + M @ M / 6 + M @ M @ M / 24)
    x0, u = np.array([0.3, -1.1]), np.array([0.7])
    y = orc.step(p, x0, u)
    np.testing.assert_allclose(y, R @ x0 + Q @ B @ u, rtol=1e-13, atol=1e-15)


def test_linear_discrete_map_exact(orc):
    """substeps = 0: the discrete map x+ = A x + B u itself, exact on small dyadics."""
    A = [[2.0, 0.5], [-1.0, 0.25]]
    B = [[1.0], [-2.0]]
    p = _lin(A, B, 1.0, 0)
    y = orc.step(p, [0.5, -0.25], [0.75])
    assert list(y) == [2.0 * 0.5 + 0.5 * -0.25 + 0.75, -1.0 * 0.5 + 0.25 * -0.25 - 1.5]


def test_vdp_rhs_hand_points(orc):
    """x1' = x2, x2' = -x1 + mu (1 - x1^2) x2 + u at hand-computed points."""
    p = W.vdp_64()
    assert list(orc.rhs(p, [2.0, 1.0], [0.0])) == [1.0, -5.0]          # -2 + (1-4)*1
    p2 = dict(p, params=[2.0])
    assert list(orc.rhs(p2, [0.5, -2.0], [0.5])) == [-2.0, -3.0]       # -0.5 + 2*.75*(-2) + .5
    assert list(orc.rhs(p, [0.0, 0.0], [0.0])) == [0.0, 0.0]           # origin is an equilibrium


def test_cstr_dl_rhs_structure(orc):
    """Dimensionless CSTR at points where exp is exact (x2 = 0) and its input
    and Arrhenius structure: d x2'/du = beta, x2/(1+x2/gamma) = 10 at x2 = 20."""
    p = W.cstr_256()
    Da = 0.072
    dx = orc.rhs(p, [0.0, 0.0], [0.0])
    assert dx[0] == pytest.approx(Da, rel=1e-15)            # r = Da * 1 * e^0
    assert dx[1] == pytest.approx(8 * Da, rel=1e-15)        # B r
    d0 = orc.rhs(p, [0.3, 1.5], [0.0])
    d1 = orc.rhs(p, [0.3, 1.5], [1.0])
    assert d1[0] == d0[0]                                   # u enters x2' only
    assert d1[1] - d0[1] == pytest.approx(0.3, rel=1e-12)   # + beta u
    # at x1 = 1 the reaction term vanishes: x1' = -1, x2' = -x2 - beta (x2 - u)
    assert list(orc.rhs(p, [1.0, 4.0], [2.0])) == pytest.approx([-1.0, -4.0 - 0.3 * 2.0], rel=1e-15)
    # x2 = 20: exponent 20/(1+1) = 10
    dx = orc.rhs(p, [0.5, 20.0], [20.0])
    assert dx[0] + 0.5 == pytest.approx(Da * 0.5 * math.e ** 10, rel=1e-14)


def test_cstr_paper_table2_and_equilibrium(orc):
    """Eq. 4 with Table 2: the parameters match the table, and (c_A, T) =
    (0.5 mol/L, 350 K) with T_c = 300 K is the classic steady state of this
    reactor (k0 e^{-E/RT} = 7.2e10 e^{-25} ~ 1/min)."""
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "table2_cstr.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert [float(r[2]) for r in rows] == W.CSTR_PAPER_PARAMS
    p = W.cstr_paper_problem()
    dx = orc.rhs(p, [0.5, 350.0], [300.0])
    k = 7.2e10 * math.exp(-25.0)
    assert abs(dx[0]) < 1e-4 and abs(k - 1.0) < 1e-4
    assert abs(dx[1]) < 1e-2
    # energy balance: at c_A = 0 only flow and jacket terms remain
    dx = orc.rhs(p, [0.0, 340.0], [320.0])
    assert dx[0] == pytest.approx(1.0, rel=1e-15)                      # (q/V)(c_Af - 0)
    assert dx[1] == pytest.approx(10.0 + 5e4 / (100 * 1000 * 0.239) * -20.0, rel=1e-13)


def _cartpole_energy_momentum(x, mc=1.0, mp=0.1, l=0.5, g=9.81):
    p, v, th, om = x
    ke = 0.5 * (mc + mp) * v * v + mp * l * v * om * math.cos(th) + (2.0 / 3.0) * mp * l * l * om * om
    pe = mp * g * l * math.cos(th)
    mom = (mc + mp) * v + mp * l * om * math.cos(th)
    return ke + pe, mom


def test_cartpole_conservation(orc):
    """Frictionless cart-pole with u = 0 conserves energy and horizontal momentum
    (Lagrangian of a cart plus a uniform rod of half-length l). Any wrong sign or
    factor in the coupled accelerations breaks one of them."""
    p = dict(W.cartpole_48(), dt=0.002, substeps=1)
    x = np.array([0.1, 0.4, 0.35, -1.2])
    e0, m0 = _cartpole_energy_momentum(x)
    for _ in range(2000):
        x = orc.step(p, x, [0.0])
    e1, m1 = _cartpole_energy_momentum(x)
    assert abs(e1 - e0) < 1e-9 * max(1.0, abs(e0))
    assert abs(m1 - m0) < 1e-9
    assert list(orc.rhs(p, [0.3, 0.0, 0.0, 0.0], [0.0])) == [0.0, 0.0, 0.0, 0.0]


def test_cartpole_force_balance(orc):
    """Horizontal force balance of cart plus pole: the time derivative of the
    momentum (m_c + m_p) v + m_p l omega cos(theta) equals the applied force,
    (m_c + m_p) p'' + m_p l (theta'' cos(theta) - omega^2 sin(theta)) = u, at any state.
    Upright and at rest a push accelerates the cart forward and tips the pole back."""
    p = W.cartpole_48()
    mc, mp, l = 1.0, 0.1, 0.5
    for x, u in (([0.0, 0.0, 0.0, 0.0], 10.0), ([0.5, -1.0, 0.3, 2.0], -7.5), ([0.0, 2.0, -0.35, -1.5], 3.0)):
        dx = orc.rhs(p, x, [u])
        th, om = x[2], x[3]
        bal = (mc + mp) * dx[1] + mp * l * (dx[3] * math.cos(th) - om * om * math.sin(th))
        assert bal == pytest.approx(u, rel=1e-12, abs=1e-12)
    dx = orc.rhs(p, [0.0, 0.0, 0.0, 0.0], [10.0])
    assert dx[1] > 0 and dx[3] < 0
