"""Surface-tension adjustment kappa (Section 2.3, Eq. mrt_surface, Eq.
li_surface_adjust; D2Q9 MRT) in the oracle, pinned without the oracle itself:

- Q has closed forms on polynomial psi fields. With the D2Q9 force weights
  G_i = w_i / c_s^2, sum_i G_i e_a e_b = delta_ab and
  sum_i G_i e_a e_b e_c e_d = (1/3)(d_ab d_cd + d_ac d_bd + d_ad d_bc), so at x = 0:
    psi = p0 + b.x + x.H.x / 2:  sum_i G_i (psi(e_i) - p0) e_i e_i = (tr(H) I + 2 H) / 6
    psi = p0 + b.x:              sum_i G_i (psi(e_i)^2 - p0^2) e_i e_i = (|b|^2 I + 2 b b) / 3
  (odd moments of the stencil vanish).
- kappa = 0 switches the source off exactly.
- Coexistence densities do not change with kappa (Table coex_dens).
- The surface tension falls with kappa, and Laplace's law (Delta p linear in 1/R)
  still holds (Table eos_surface_tension, Fig. eos_laplace).
"""
import numpy as np
import pytest

import oracle
from synth import cases


def _case(shape=(9, 9, 1), kappa=0.7, A=-0.2, g=-1.0):
    return cases.base_case("D2Q9", shape, collision="MRT", psi=["rho", "rho"], g=[[g, 0], [0, g]],
                           A=[A, A], kappa=[kappa, kappa])


def _grid(n=9):
    xs = np.arange(n) - (n // 2)
    return np.meshgrid(xs, xs)                   # X, Y as [y, x]


def test_surface_Q_psi_term_on_a_quadratic_field():
    kappa, g = 0.7, -1.0
    s = oracle.OracleSim(_case(kappa=kappa, A=0.0, g=g))
    X, Y = _grid()
    p0, b = 1.3, np.array([0.02, -0.015])
    H = np.array([[0.004, 0.0015], [0.0015, -0.003]])
    psi = p0 + b[0] * X + b[1] * Y + 0.5 * (H[0, 0] * X * X + 2 * H[0, 1] * X * Y + H[1, 1] * Y * Y)
    Q = s.surface_Q(psi[None, None], (4, 4))
    T = kappa * 0.5 * g * p0 * (np.trace(H) * np.eye(2) + 2 * H) / 6.0
    assert np.allclose(Q, [T[0, 0], T[1, 1], T[0, 1]], rtol=1e-12, atol=1e-16)


def test_surface_Q_mixing_term_on_a_linear_field():
    kappa, A, g = 0.7, -0.3, -1.0
    s = oracle.OracleSim(_case(kappa=kappa, A=A, g=g))
    X, Y = _grid()
    p0, b = 1.3, np.array([0.02, -0.015])
    psi = p0 + b[0] * X + b[1] * Y
    Q = s.surface_Q(psi[None, None], (4, 4))
    # the (1 - A) psi (psi' - psi) term vanishes on a linear field (odd moment)
    T = kappa * 0.5 * g * 0.5 * A * (np.dot(b, b) * np.eye(2) + 2 * np.outer(b, b)) / 3.0
    assert np.allclose(Q, [T[0, 0], T[1, 1], T[0, 1]], rtol=1e-12, atol=1e-16)


def test_kappa_zero_is_off():
    case, init = cases.droplet_2d_cs(n=48, radius=12)
    case["collision"] = "MRT"
    outs = []
    for kap in (None, 0.0):
        c = dict(case)
        if kap is not None:
            c["kappa"] = [kap, kap]
        s = oracle.OracleSim(c)
        s.init_fields(0, init["rho"][0])
        s.step(50)
        outs.append(s.populations(0))
    assert np.array_equal(outs[0], outs[1])


def _slab(kappa, n=120, steps=12000):
    rg, rl = cases.COEX[("CS", 0.7)]
    case = cases.with_eos(cases.base_case("D2Q9", (n, 4, 1), collision="MRT", A=[cases.A_STAR[("CS", 0.7)]] * 2,
                                          kappa=[kappa, kappa]), "CS", 0.7)
    case["eos_a"] = [0.5, 0.5]
    x = np.arange(n)[None, None, :] * np.ones((1, 4, 1))
    rho = rg + (rl - rg) * ((x > n / 4) & (x < 3 * n / 4))
    s = oracle.OracleSim(case)
    s.init_fields(0, rho)
    s.step(steps)
    r, _ = s.macroscopic(0)
    return r[0, :, n // 2].mean(), r[0, :, 2].mean()


def test_coexistence_densities_do_not_change_with_kappa():
    # Table coex_dens: the densities stay at the Maxwell pair for every kappa
    l0, g0 = _slab(0.0)
    l5, g5 = _slab(0.5)
    assert abs(l5 - l0) / l0 < 5e-3
    assert abs(g5 - g0) / g0 < 2e-2


def _laplace(kappa, radii=(12, 16, 20), steps=6000, n=96):
    pts = []
    for R in radii:
        case, init = cases.droplet_2d_cs(n=n, radius=R)
        case["collision"] = "MRT"
        case["kappa"] = [kappa, kappa]
        s = oracle.OracleSim(case)
        s.init_fields(0, init["rho"][0])
        s.step(steps)
        r, _ = s.macroscopic(0)
        c = n // 2
        rin = r[0, c - 3:c + 3, c - 3:c + 3].mean()
        rout = r[0, :4, :4].mean()
        dp = oracle.bulk_pressure(case, 0, rin) - oracle.bulk_pressure(case, 0, rout)
        Rm = np.sqrt((r > 0.5 * (rin + rout)).sum() / np.pi)
        pts.append((1.0 / Rm, dp))
    x = np.array(pts)
    Am = np.vstack([x[:, 0], np.ones(len(x))]).T
    (sigma, b), *_ = np.linalg.lstsq(Am, x[:, 1], rcond=None)
    pred = Am @ np.array([sigma, b])
    r2 = 1 - ((x[:, 1] - pred) ** 2).sum() / ((x[:, 1] - x[:, 1].mean()) ** 2).sum()
    return sigma, b, r2, x[:, 1].max()


def test_surface_tension_falls_with_kappa_and_laplace_still_holds():
    s0, _, _, _ = _laplace(0.0)
    s5, b5, r25, dpmax = _laplace(0.5)
    assert r25 > 0.99 and abs(b5) < 0.05 * dpmax
    ratio = s5 / s0
    print("sigma(kappa=0.5) / sigma(0) = %.3f" % ratio)
    # falls with kappa; with EDM forcing the measured slope is 1 - 0.61 kappa (the paper's
    # moment-space forcing gives ~1 - kappa)
    assert 0.4 < ratio < 0.8
