"""Sessile-drop contact angle: the set-up and the measurement used by the oracle pins,
the calibration script of tests/golden and the GPU parity test.

The angle is that of a drop resting on a flat solid wall at steady state (Section 2.4
sets it through the virtual density of Eq. improved_virtual_density; the paper measures
it on drops and menisci, Sections 3.3.1-3.4.3). Reading of the measurement: the interface
is the iso-line where the drop's phase indicator (rho for one component, rho_0 - rho_1 for
two) is half way between its bulk values; iso-line points more than `skip` nodes above the
wall are fitted by a circle (algebraic least squares, Kasa 1976), and the angle through the
drop is arccos((y_w - y_c) / R), y_w being the halfway bounce-back wall between the solid
row y = 0 and the first fluid row. Drops are cylinders (2-D, or D3Q19 boxes two nodes deep
along the periodic z axis), whose angle obeys the same Young balance as a spherical cap.
"""
import numpy as np

from synth import cases, droplet_field

WALL_Y = 0.5


def calibration():
    """The calibrated wetting parameters of tests/golden/wetting_calibration.json."""
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "wetting_calibration.json")) as fh:
        return json.load(fh)


def circle_angle(ind, mid, skip=3.0, wall_y=WALL_Y):
    """Contact angle (degrees) of the drop where ind > mid, ind [ny, nx], wall at y = wall_y."""
    return circle_fit(ind, mid, skip, wall_y)[0]


def circle_fit(ind, mid, skip=3.0, wall_y=WALL_Y):
    """(contact angle in degrees, radius, centre x, centre y) of the circle fitted to the
    half-way iso-line of the drop where ind > mid, ind [ny, nx], wall at y = wall_y."""
    ny, nx = ind.shape
    pts = []
    a = ind - mid
    for x in range(nx):                       # crossings along y
        col = a[:, x]
        for y in range(1, ny - 1):
            if col[y] > 0 >= col[y + 1] or col[y] <= 0 < col[y + 1]:
                pts.append((x, y + col[y] / (col[y] - col[y + 1])))
    for y in range(1, ny):                    # crossings along x (steep flanks)
        row = a[y]
        for x in range(nx - 1):
            if row[x] > 0 >= row[x + 1] or row[x] <= 0 < row[x + 1]:
                pts.append((x + row[x] / (row[x] - row[x + 1]), y))
    p = np.array([q for q in pts if q[1] > wall_y + skip])
    A = np.column_stack([p[:, 0], p[:, 1], np.ones(len(p))])
    rhs = -(p[:, 0] ** 2 + p[:, 1] ** 2)
    (D, E, F), *_ = np.linalg.lstsq(A, rhs, rcond=None)
    xc, yc = -D / 2, -E / 2
    R = np.sqrt(xc * xc + yc * yc - F)
    return float(np.degrees(np.arccos(np.clip((wall_y - yc) / R, -1.0, 1.0)))), float(R), float(xc), float(yc)


def _cap_centre(radius, theta0):
    """Centre height and radius of a circular cap on the wall with contact angle theta0
    (degrees) and the area of a half disk of the given radius."""
    t = np.radians(theta0)
    R0 = radius * np.sqrt((np.pi / 2) / (t - np.sin(t) * np.cos(t)))
    return WALL_Y - R0 * np.cos(t), R0


def sessile_case(model, phi, shape=None, radius=None, real="f64", theta0=90.0):
    """(case, rhos, solid, indicator) of a drop on the wall row y = 0, started as a
    circular cap with contact angle theta0 and the area of a half disk of `radius`.

    model "cs_d2q9": D2Q9 single-component CS, T = 0.7 Tc (a = 0.5), BGK tau = 1.
    model "pr08": the sphere-pack workload's fluid, D3Q19 single-component Peng-Robinson
      at T = 0.8 Tc, MRT tau = 1.5; phi on the liquid (the drop).
    model "two_component": the porous drainage workload's fluids, D3Q19 two-component
      psi = rho, g12 = G12_IMMISCIBLE, common velocity, BGK tau = 1, each phase started at
      its equilibrium composition RHO_IMMISCIBLE; the drop is the wetting component (phi on
      it; the other takes drho = WET_DRHO_NW, which clamps its virtual density to 0).
    indicator(lat_or_sim_fields) -> (ind, mid) maps per-component densities [K][ny][nx]."""
    if model == "cs_d2q9":
        nx, ny, nz = shape or (120, 60, 1)
        R = radius or 20.0
        A = cases.A_STAR[("CS", 0.7)]
        case = cases.base_case("D2Q9", (nx, ny, nz), A=[A, A], wet_phi=[phi, phi], real=real,
                               bc=["periodic", "periodic", "wall", "wall", "periodic", "periodic"])
        case = cases.with_eos(case, "CS", 0.7)
        case["eos_a"] = [0.5, 0.5]
        rg, rl = cases.COEX[("CS", 0.7)]
        case["rho_lo"], case["rho_hi"] = [rg, rg], [rl, rl]
        yc, R0 = _cap_centre(R, theta0)
        rhos = [droplet_field((nx, ny, nz), [(nx / 2, yc)], [R0], rl, rg, 5.0, periodic=False)]
        mid = 0.5 * (rl + rg)
        ind = lambda r: (r[0], mid)
    elif model == "vdw07_kappa":
        # the capillary-rise fluid: D2Q9 van der Waals at T = 0.7 Tc (alpha = 0.5), MRT with the
        # surface-tension adjustment kappa = 0.5 and the moment-space forcing, tau = 1
        nx, ny, nz = shape or (320, 60, 1)
        R = radius or 30.0
        A = cases.A_STAR_MOMENT[("VdW", 0.7)]
        case = cases.with_eos(cases.base_case("D2Q9", (nx, ny, nz), collision="MRT", A=[A, A], real=real,
                                              alpha=[cases.VDW07_ALPHA] * 2, kappa=[0.5, 0.5], forcing="moment",
                                              wet_phi=[phi, phi],
                                              bc=["periodic", "periodic", "wall", "wall", "periodic", "periodic"]),
                              "VdW", 0.7)
        rg, rl = cases.COEX[("VdW", 0.7)]
        case["rho_lo"], case["rho_hi"] = [rg, rg], [rl, rl]
        yc, R0 = _cap_centre(R, theta0)
        rhos = [droplet_field((nx, ny, nz), [(nx / 2, yc)], [R0], rl, rg, 5.0, periodic=False)]
        mid = 0.5 * (rl + rg)
        ind = lambda r: (r[0], mid)
    elif model == "pr08":
        nx, ny, nz = shape or (120, 60, 2)
        R = radius or 22.0
        rg, rl = cases.COEX[("PR", 0.8)]
        tau = 1.5
        case = cases.with_eos(cases.base_case("D3Q19", (nx, ny, nz), real=real, collision="MRT", tau=[tau, tau],
                                              mrt_rates=cases.pr06_mrt_rates(tau), A=[cases.A_STAR[("PR", 0.8)]] * 2,
                                              wet_phi=[phi, phi], rho_lo=[rg, rg], rho_hi=[rl, rl],
                                              bc=["periodic", "periodic", "wall", "wall", "periodic", "periodic"]),
                              "PR", 0.8, comps=(0,))
        yc, R0 = _cap_centre(R, theta0)
        prof = droplet_field((nx, ny, 1), [(nx / 2, yc)], [R0], rl, rg, 5.0, periodic=False)
        rhos = [np.repeat(prof, nz, axis=0)]
        mid = 0.5 * (rl + rg)
        ind = lambda r: (r[0], mid)
    elif model == "two_component":
        nx, ny, nz = shape or (120, 60, 2)
        R = radius or 22.0
        hi, lo = cases.RHO_IMMISCIBLE                # the two bulk compositions at equilibrium
        case = cases.base_case("D3Q19", (nx, ny, nz), real=real, ncomp=2, psi=["rho", "rho"], velocity="common",
                               g=[[0.0, cases.G12_IMMISCIBLE], [cases.G12_IMMISCIBLE, 0.0]], tau=[1.0, 1.0],
                               wet_phi=[phi, 1.0], wet_drho=[0.0, cases.WET_DRHO_NW],
                               rho_lo=[0.0, 0.0], rho_hi=[5.0, 5.0],
                               bc=["periodic", "periodic", "wall", "wall", "periodic", "periodic"])
        yc, R0 = _cap_centre(R, theta0)
        s = droplet_field((nx, ny, 1), [(nx / 2, yc)], [R0], 1.0, 0.0, 4.0, periodic=False)
        s = np.repeat(s, nz, axis=0)
        rhos = [lo + (hi - lo) * s, lo + (hi - lo) * (1.0 - s)]
        ind = lambda r: (r[0] - r[1], 0.0)
    else:
        raise ValueError(model)
    solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    solid[:, 0, :] = 1
    return case, rhos, solid, ind


def oracle_angle(model, phi, steps, **kw):
    """Contact angle of the oracle's drop after `steps` steps (z-averaged fields)."""
    import oracle
    case, rhos, solid, ind = sessile_case(model, phi, **kw)
    s = oracle.OracleSim(case)
    s.set_geometry(solid)
    for k, r in enumerate(rhos):
        s.init_fields(k, r)
    s.step(steps)
    dens = [s.macroscopic(k)[0].mean(axis=0) for k in range(s.K)]
    a, mid = ind(dens)
    return circle_angle(a, mid)
