"""Brute force on tiny lattices: the whole time step of the FP64 oracle against a direct
numpy restatement of the paper's equations on periodic lattices of a few nodes.

The restatement follows Section 2 step by step, with the readings the oracle states:
density and bare momentum of each component (Eq. macroeq, Eq. macroeq_mcp); the
pseudopotential psi = exp(-1/rho) of Section 5 or psi = rho, with U = g psi^2 / 2; the
interaction force of Eq. software_ff_force_mcmp on all Q-1 links with G_i = w_i / c_s^2,
F = A (-sum_i G_i U(x + e_i) e_i) + (1 - A) (-psi(x) sum_k' g_kk' sum_i G_i psi_k'(x + e_i) e_i)
plus the body force rho a; the BGK collision toward f^eq(rho, u) with the velocity shift
of Eq. edm, f* = f - (f - f^eq(u)) / tau + f^eq(u + F / rho) - f^eq(u); u the bare
velocity, or the common velocity sum_k (j_k / tau_k) / sum_k (rho_k / tau_k); and push
streaming with periodic wrap. With solids: the virtual density of Eq.
improved_virtual_density at boundary solids, rho_s = phi rho_ave - drho clamped, rho_ave
the w_i-weighted mean of the fluid neighbours' densities, psi at solids from rho_s, forces
at fluid nodes only, and halfway bounce-back (a population streaming into a solid returns
to its origin reversed). It shares no code with the oracle: the velocity set is taken
from the oracle only to order the populations the same way, and is checked against the
textbook set.
"""
import numpy as np
import pytest

import oracle
from synth import cases, random_field

CS2 = 1.0 / 3.0


def _weights(e):
    # D2Q9: 4/9, 1/9, 1/36; D3Q19: 1/3, 1/18, 1/36, by |e|^2
    d = e.shape[1]
    table = {2: {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}, 3: {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}}[d]
    return np.array([table[int((v * v).sum())] for v in e])


def _feq(e, w, rho, u):
    # w_i rho (1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u.u)
    eu = np.einsum("id,d...->i...", e, u)
    uu = (u * u).sum(axis=0)
    return w.reshape((-1,) + (1,) * rho.ndim) * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * uu)


def _shift(a, v):
    # a(x + v) on the periodic grid (arrays indexed [..., z, y, x] or [..., y, x])
    d = len(v)
    out = a
    for axis_from_end, comp in zip(range(1, d + 1), v):
        out = np.roll(out, -int(comp), axis=-axis_from_end)
    return out


def _pr_psi(rho, p):
    # Peng-Robinson (Eq. eos_potential with the standard form the paper cites):
    # p = rho R T / (1 - b rho) - a alpha(T) rho^2 / (1 + 2 b rho - b^2 rho^2),
    # alpha(T) = (1 + m (1 - sqrt(T / Tc)))^2, m = 0.37464 + 1.54226 w - 0.26992 w^2;
    # U = alpha p - c_s^2 rho, psi = sqrt(2 U / g) where that is real, else psi = U = 0
    a, b, R, w, Tr, g = p["eos_a"], p["eos_b"], 1.0, p["omega"], p["T_red"], p["g"][0][0]
    T = Tr * p["Tc"]
    m = 0.37464 + 1.54226 * w - 0.26992 * w * w
    al = (1 + m * (1 - np.sqrt(Tr))) ** 2
    pe = rho * R * T / (1 - b * rho) - a * al * rho * rho / (1 + 2 * b * rho - b * b * rho * rho)
    U = p["alpha"] * pe - CS2 * rho
    arg = 2 * U / g
    return np.sqrt(np.where(arg > 0, arg, 0.0)), np.where(arg > 0, U, 0.0)


def _mrt_d3q19(e):
    # d'Humieres' D3Q19 moment polynomials, in the order the rates are given:
    # rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pxz, mx, my, mz
    x, y, z = (e[:, d].astype(float) for d in range(3))
    c2 = x * x + y * y + z * z
    rows = [np.ones_like(x), 19 * c2 - 30, (21 * c2 * c2 - 53 * c2 + 24) / 2,
            x, (5 * c2 - 9) * x, y, (5 * c2 - 9) * y, z, (5 * c2 - 9) * z,
            3 * x * x - c2, (3 * c2 - 5) * (3 * x * x - c2), y * y - z * z, (3 * c2 - 5) * (y * y - z * z),
            x * y, y * z, x * z, (y * y - z * z) * x, (z * z - x * x) * y, (x * x - y * y) * z]
    return np.array(rows)


def _opposite(e):
    return np.array([next(o for o in range(len(e)) if (e[o] == -e[i]).all()) for i in range(len(e))])


def _virtual_density(rho, solid, e, w, phi, drho, lo, hi):
    # boundary solids: rho_s = phi rho_ave - drho, clamped, rho_ave over fluid neighbours
    fluid = ~solid
    num = np.zeros_like(rho)
    den = np.zeros_like(rho)
    for i in range(len(e)):
        if not e[i].any():
            continue
        fl = _shift(fluid, e[i])
        num += np.where(fl, w[i] * _shift(rho, e[i]), 0.0)
        den += np.where(fl, w[i], 0.0)
    boundary = solid & (den > 0)
    rs = np.clip(phi * np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0) - drho, lo, hi)
    return np.where(boundary, rs, rho)


def _step(f, e, w, p, solid=None):
    K, D = len(f), e.shape[1]
    G = w / CS2
    rho = [fk.sum(axis=0) for fk in f]
    j = [np.einsum("id,i...->d...", e, fk) for fk in f]
    if solid is not None:
        rho = [_virtual_density(np.where(solid, 0.0, rho[k]), solid, e, w, p["phi"][k], p["drho"][k],
                                p["lo"][k], p["hi"][k]) for k in range(K)]
    if p["psi"] == "pr":
        psi, U = zip(*[_pr_psi(r, p) for r in rho])
    else:
        psi = [np.exp(-1.0 / r) if p["psi"] == "exp" else r for r in rho]
        U = [0.5 * p["g"][k][k] * psi[k] ** 2 for k in range(K)]
    F = []
    for k in range(K):
        zc = np.zeros((D,) + rho[k].shape)
        sc = np.zeros((D,) + rho[k].shape)
        for i in range(len(e)):
            if not e[i].any():
                continue            # the rest direction is no link
            ev = e[i].reshape((D,) + (1,) * rho[k].ndim)
            zc -= G[i] * _shift(U[k], e[i]) * ev
            tot = sum(p["g"][k][kp] * _shift(psi[kp], e[i]) for kp in range(K))
            sc -= psi[k] * G[i] * tot * ev
        a = np.asarray(p["accel"][k][:D]).reshape((D,) + (1,) * rho[k].ndim)
        F.append(p["A"][k] * zc + (1 - p["A"][k]) * sc + rho[k] * a)
    if p.get("common"):
        num = sum(j[k] / p["tau"][k] for k in range(K))
        den = sum(rho[k] / p["tau"][k] for k in range(K))
        ueq = [num / den] * K
    else:
        ueq = [j[k] / rho[k] for k in range(K)]
    out = []
    opp = _opposite(e)
    for k in range(K):
        u = ueq[k]
        du = F[k] / rho[k]
        fe = _feq(e, w, rho[k], u)
        if p.get("mrt") is not None:
            # f* = f - M^-1 S M (f - f^eq(u)) + f^eq(u + du) - f^eq(u): the stress rows relax at
            # 1/tau, the conserved ones not at all, the rest at the given rates
            M = _mrt_d3q19(e)
            rates = np.array(p["mrt"][k], dtype=float)
            rates[[9, 11, 13, 14, 15]] = 1.0 / p["tau"][k]
            rates[[0, 3, 5, 7]] = 0.0
            C = np.linalg.inv(M) @ np.diag(rates) @ M
            fs = f[k] - np.einsum("ij,j...->i...", C, f[k] - fe) + _feq(e, w, rho[k], u + du) - fe
        else:
            fs = f[k] - (f[k] - fe) / p["tau"][k] + _feq(e, w, rho[k], u + du) - fe
        if solid is None:
            out.append(np.stack([_shift(fs[i], -e[i]) for i in range(len(e))]))
        else:
            # pull: from x - e_i where that node is fluid, else the reversed population of x
            fn = [np.where(_shift(solid, -e[i]), fs[opp[i]], _shift(fs[i], -e[i])) for i in range(len(e))]
            out.append(np.where(solid, 0.0, np.stack(fn)))
    return out


def _check_set(e):
    D = e.shape[1]
    want = {tuple(c - 1 for c in v) for v in np.ndindex(*(3,) * D)}
    want = {v for v in want if D == 2 or sum(abs(c) for c in v) <= 2}
    assert {tuple(v) for v in e} == want and len(e) == len(want)


def _compare(case, rhos, p, steps=4, solid=None):
    s = oracle.OracleSim(case)
    if solid is not None:
        s.set_geometry(solid)
    for k, r in enumerate(rhos):
        s.init_fields(k, r)
    D = 3 if case["lattice"] == "D3Q19" else 2
    e = np.asarray(s.e, dtype=np.int64)[:, :D]
    _check_set(e)
    w = _weights(e)
    sq = (lambda a: a[:, 0]) if D == 2 else (lambda a: a)       # drop the z axis of 2-D lattices
    sm = None if solid is None else sq(solid[None].astype(bool))[0]
    f = [sq(s.populations(k)) for k in range(len(rhos))]
    if sm is not None:
        f = [np.where(sm, 0.0, fk) for fk in f]
    for _ in range(steps):
        f = _step(f, e, w, p, sm)
    s.step(steps)
    keep = (lambda a: a) if sm is None else (lambda a: np.where(sm, 0.0, a))
    err = max(np.abs(keep(sq(s.populations(k))) - f[k]).max() for k in range(len(rhos)))
    scale = max(np.abs(fk).max() for fk in f)
    return err / scale


@pytest.mark.parametrize("lattice,shape", [("D2Q9", (6, 5, 1)), ("D3Q19", (4, 3, 5))])
def test_one_component_step_against_brute_force(lattice, shape):
    # psi = exp(-1/rho) (Section 5), g = -1.5, mixing weight A = 0.3, tau = 0.8, a body force
    g, A, tau = -1.5, 0.3, 0.8
    accel = [[1e-4, -2e-4, 5e-5 if lattice == "D3Q19" else 0.0], [0.0, 0.0, 0.0]]
    case = cases.base_case(lattice, shape, psi=["exp", "exp"], g=[[g, 0.0], [0.0, g]], A=[A, A],
                           collision="BGK", tau=[tau, tau], accel=accel, real="f64")
    p = dict(psi="exp", g=[[g, 0.0], [0.0, g]], A=[A, A], tau=[tau, tau], accel=accel)
    rel = _compare(case, [random_field(shape, 0.6, 1.4, 71)], p)
    print("%s one component, 4 steps: max |f_oracle - f_brute| / max f = %.2e" % (lattice, rel))
    assert rel < 1e-13


def test_two_components_common_velocity_against_brute_force():
    # psi = rho, cross coupling g12 = 0.3 only, common velocity with tau = (1.0, 0.7)
    shape = (6, 5, 1)
    g12 = 0.3
    case = cases.base_case("D2Q9", shape, ncomp=2, psi=["rho", "rho"], g=[[0.0, g12], [g12, 0.0]],
                           velocity="common", collision="BGK", tau=[1.0, 0.7], real="f64")
    p = dict(psi="rho", g=[[0.0, g12], [g12, 0.0]], A=[0.0, 0.0], tau=[1.0, 0.7], common=True,
             accel=[[0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    rel = _compare(case, [random_field(shape, 0.3, 0.9, 72), random_field(shape, 0.2, 0.7, 73)], p)
    print("D2Q9 two components, common velocity, 4 steps: max rel %.2e" % rel)
    assert rel < 1e-13


@pytest.mark.parametrize("lattice,shape", [("D2Q9", (7, 6, 1)), ("D3Q19", (5, 4, 4))])
def test_step_with_wetting_solids_against_brute_force(lattice, shape):
    # a few solid nodes (a block and a lone node), wetting phi = 1.2 and drho = 0.05 with the
    # limiter [0.9, 1.05] clipping some boundary solids at each end (their unclipped rho_s
    # spans 0.84-1.18 and 0.98-1.34 at the start), psi = exp(-1/rho), g = -1.5, A = 0.3, tau = 0.9
    g, A, tau = -1.5, 0.3, 0.9
    nx, ny, nz = shape
    solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    solid[:, 2:4, 2:4] = 1
    solid[0, 0, nx - 1] = 1
    case = cases.base_case(lattice, shape, psi=["exp", "exp"], g=[[g, 0.0], [0.0, g]], A=[A, A],
                           collision="BGK", tau=[tau, tau], wet_phi=[1.2, 1.2], wet_drho=[0.05, 0.05],
                           rho_lo=[0.9, 0.9], rho_hi=[1.05, 1.05], real="f64")
    p = dict(psi="exp", g=[[g, 0.0], [0.0, g]], A=[A, A], tau=[tau, tau], accel=[[0.0] * 3, [0.0] * 3],
             phi=[1.2, 1.2], drho=[0.05, 0.05], lo=[0.9, 0.9], hi=[1.05, 1.05])
    rel = _compare(case, [random_field(shape, 0.6, 1.4, 74)], p, solid=solid)
    print("%s with wetting solids, 4 steps: max rel %.2e" % (lattice, rel))
    assert rel < 1e-13


def test_peng_robinson_step_against_brute_force():
    # the headline workload's fluid: Peng-Robinson at T = 0.6 Tc (a = 2/49, b = 2/21,
    # omega = 0.344), g = -1, mixing weight A = 0.2, BGK tau = 1, densities from vapour to
    # liquid. Tc is the oracle's root of the critical-point conditions (pinned against the
    # closed forms elsewhere); the EOS and psi are restated here
    shape = (4, 3, 5)
    case = cases.with_eos(cases.base_case("D3Q19", shape, collision="BGK", A=[0.2, 0.2], real="f64"), "PR", 0.6)
    pe = cases.EOS_PARAMS["PR"]
    p = dict(psi="pr", g=case["g"], A=[0.2, 0.2], tau=[1.0, 1.0], accel=[[0.0] * 3, [0.0] * 3],
             eos_a=pe["eos_a"], eos_b=pe["eos_b"], omega=pe["eos_omega"], T_red=0.6, alpha=case["alpha"][0],
             Tc=oracle.eos_Tc("PR", pe["eos_a"], pe["eos_b"], 1.0))
    rel = _compare(case, [random_field(shape, 0.05, 6.5, 75)], p)
    print("D3Q19 Peng-Robinson, 4 steps: max rel %.2e" % rel)
    assert rel < 1e-13


def test_headline_workload_step_against_brute_force():
    # the 256^3 benchmark's configuration on a 4x3x5 lattice: D3Q19 MRT (d'Humieres basis,
    # the workload's rates, stress at 1/tau), Peng-Robinson at T = 0.6 Tc with its mixing
    # weight and EOS scaling alpha, EDM forcing
    shape = (4, 3, 5)
    tau = cases.PR06_TAU
    case = cases.with_eos(cases.base_case("D3Q19", shape, collision="MRT", A=[cases.PR06_A] * 2,
                                          alpha=[cases.PR06_ALPHA] * 2, tau=[tau, tau],
                                          mrt_rates=cases.pr06_mrt_rates(tau), real="f64"), "PR", 0.6)
    pe = cases.EOS_PARAMS["PR"]
    p = dict(psi="pr", g=case["g"], A=[cases.PR06_A] * 2, tau=[tau, tau], accel=[[0.0] * 3, [0.0] * 3],
             eos_a=pe["eos_a"], eos_b=pe["eos_b"], omega=pe["eos_omega"], T_red=0.6, alpha=cases.PR06_ALPHA,
             Tc=oracle.eos_Tc("PR", pe["eos_a"], pe["eos_b"], 1.0), mrt=cases.pr06_mrt_rates(tau))
    rg, rl = cases.COEX[("PR", 0.6)]
    rel = _compare(case, [random_field(shape, rg, rl, 76)], p)
    print("D3Q19 MRT Peng-Robinson (headline configuration), 4 steps: max rel %.2e" % rel)
    assert rel < 1e-13


def test_two_components_with_self_coupling_and_mixing_against_brute_force():
    # the general two-component force: self couplings g_kk != 0 with mixing weights A_k (the
    # Zhang-Chen term on U_k = g_kk psi_k^2 / 2) and the cross coupling, psi = exp(-1/rho),
    # each component at its own velocity and tau, a body force on one component
    shape = (4, 3, 5)
    g = [[-1.2, 0.4], [0.4, -1.0]]
    A = [0.3, 0.1]
    tau = [0.9, 1.2]
    accel = [[5e-5, 0.0, -1e-4], [0.0, 0.0, 0.0]]
    case = cases.base_case("D3Q19", shape, ncomp=2, psi=["exp", "exp"], g=g, A=A, velocity="component",
                           collision="BGK", tau=tau, accel=accel, real="f64")
    p = dict(psi="exp", g=g, A=A, tau=tau, accel=accel)
    rel = _compare(case, [random_field(shape, 0.5, 1.3, 77), random_field(shape, 0.4, 1.1, 78)], p)
    print("D3Q19 two components, self coupling and mixing, 4 steps: max rel %.2e" % rel)
    assert rel < 1e-13


def _mrt_d2q9(e):
    # Lallemand and Luo's D2Q9 moments: rho, e, eps, jx, qx, jy, qy, pxx, pxy
    x, y = (e[:, d].astype(float) for d in range(2))
    c2 = x * x + y * y
    return np.array([np.ones_like(x), -4 + 3 * c2, 4 - 10.5 * c2 + 4.5 * c2 * c2, x, (-5 + 3 * c2) * x,
                     y, (-5 + 3 * c2) * y, x * x - y * y, x * y])


def _step_kappa(f, e, w, p):
    # Section 2.3 with the reading the oracle states: f* = f - M^-1 [S (m - m^eq(v)) - C - F_m],
    # v = (sum f e + F / 2) / rho, F_m = (I - S / 2) M S_G with Guo's source
    # S_G,i = w_i [3 (e_i - v) + 9 (e_i . v) e_i] . F, and C of Eq. li_surface_adjust in the
    # e, eps, pxx, pxy moments from Q = kappa g / 2 [(1 - A) psi sum_i G_i (psi_i - psi) e_i e_i
    # + A / 2 sum_i G_i (psi_i^2 - psi^2) e_i e_i]; one component, psi = exp(-1/rho)
    g, A, kap, tau = p["g"], p["A"], p["kappa"], p["tau"]
    G = w / CS2
    fk = f[0]
    rho = fk.sum(axis=0)
    j = np.einsum("id,i...->d...", e, fk)
    psi = np.exp(-1.0 / rho)
    U = 0.5 * g * psi * psi
    F = np.zeros((2,) + rho.shape)
    Qxx, Qyy, Qxy = (np.zeros_like(rho) for _ in range(3))
    for i in range(len(e)):
        if not e[i].any():
            continue
        pn = _shift(psi, e[i])
        ev = e[i].reshape(2, 1, 1)
        F += A * (-G[i] * _shift(U, e[i]) * ev) + (1 - A) * (-psi * g * G[i] * pn * ev)
        t = G[i] * ((1 - A) * psi * (pn - psi) + 0.5 * A * (pn * pn - psi * psi))
        Qxx += t * e[i][0] ** 2
        Qyy += t * e[i][1] ** 2
        Qxy += t * e[i][0] * e[i][1]
    F += rho * np.asarray(p["accel"][:2]).reshape(2, 1, 1)
    kg = 0.5 * kap * g
    Qxx, Qyy, Qxy = kg * Qxx, kg * Qyy, kg * Qxy
    rates = np.array(p["rates"], dtype=float)[:9]
    rates[[7, 8]] = 1.0 / tau
    rates[[0, 3, 5]] = 0.0
    M = _mrt_d2q9(e)
    Mi = np.linalg.inv(M)
    v = (j + 0.5 * F) / rho
    m = np.einsum("ai,i...->a...", M, fk)
    meq = np.einsum("ai,i...->a...", M, _feq(e, w, rho, v))
    ev = np.einsum("id,d...->i...", e, v)
    eF = np.einsum("id,d...->i...", e, F)
    vF = (v * F).sum(axis=0)
    SG = w.reshape(-1, 1, 1) * (3 * (eF - vF) + 9 * ev * eF)
    Fm = np.einsum("ai,i...->a...", M, SG) * (1 - 0.5 * rates).reshape(-1, 1, 1)
    C = np.zeros_like(m)
    C[1] = 1.5 * rates[1] * (Qxx + Qyy)
    C[2] = -1.5 * rates[2] * (Qxx + Qyy)
    C[7] = -rates[7] * (Qxx - Qyy)
    C[8] = -rates[8] * Qxy
    ms = m - rates.reshape(-1, 1, 1) * (m - meq) + C + Fm
    fs = np.einsum("ia,a...->i...", Mi, ms)
    return [np.stack([_shift(fs[i], -e[i]) for i in range(len(e))])]


@pytest.mark.parametrize("kappa", [0.0, 0.5])
def test_surface_tension_adjustment_step_against_brute_force(kappa):
    # D2Q9 MRT with the moment-space forcing of Eq. mrt_surface and the source C of Eq.
    # li_surface_adjust (kappa = 0.5; kappa = 0 checks the forcing alone), psi = exp(-1/rho),
    # g = -1.5, A = -0.4, tau = 1, a body force
    shape = (7, 6, 1)
    g, A, tau = -1.5, -0.4, 1.0
    accel = [[2e-5, -1e-5, 0.0], [0.0, 0.0, 0.0]]
    case = cases.base_case("D2Q9", shape, collision="MRT", psi=["exp", "exp"], g=[[g, 0.0], [0.0, g]], A=[A, A],
                           tau=[tau, tau], kappa=[kappa, kappa], forcing="moment", accel=accel, real="f64")
    p = dict(g=g, A=A, kappa=kappa, tau=tau, accel=accel[0], rates=case["mrt_rates"][0])
    s = oracle.OracleSim(case)
    s.init_fields(0, random_field(shape, 0.6, 1.4, 79))
    e = np.asarray(s.e, dtype=np.int64)[:, :2]
    _check_set(e)
    w = _weights(e)
    f = [s.populations(0)[:, 0]]
    for _ in range(4):
        f = _step_kappa(f, e, w, p)
    s.step(4)
    rel = np.abs(s.populations(0)[:, 0] - f[0]).max() / np.abs(f[0]).max()
    print("D2Q9 MRT, moment-space forcing, kappa = %.1f, 4 steps: max rel %.2e" % (kappa, rel))
    assert rel < 1e-13
