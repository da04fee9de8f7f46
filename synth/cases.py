"""Problem descriptions of the paper's workloads, as plain parameter dicts.

A problem description is a dict of parameter VALUES in the paper's notation
(lattice, EOS parameters a, b, R, omega, T_r, interaction strengths g_kk',
mixing weight A_kk, relaxation times, wetting phi / drho, boundary kinds). Both
the CUDA binding and the oracle binding translate it with their own code.

Keys:
  lattice      "D2Q9" | "D3Q19"
  shape        (nx, ny, nz), nz = 1 for D2Q9
  ncomp        1 | 2
  real         "f32" | "f64" (storage and compute type of the CUDA path)
  collision    "BGK" | "MRT"
  velocity     "component" (u^k = j^k / rho^k) | "common" (Shan-Chen common velocity)
  tau          [tau_1, tau_2]
  mrt_rates    per component, 19 rates in the moment order of the MRT basis
               (stress rates are replaced by 1/tau, conserved rates by 0)
  psi          per component "eos" | "rho" | "exp"
  eos          per component "CS" | "PR" | "VdW" | "RK" | "RKS"
  eos_a, eos_b, eos_R, eos_omega, T_red, alpha, A   per component
  g            2x2 interaction strengths
  wet_phi, wet_drho, rho_lo, rho_hi                per component
  accel        per component body acceleration (3)
  bc           6 faces (-x, +x, -y, +y, -z, +z): "periodic" | "wall" | "pressure"
  bc_rho       6 x ncomp face densities (pressure faces)
  kappa        per component surface-tension adjustment (D2Q9 MRT; 0 = off)
  forcing      "edm" (Eq. edm, the default) | "moment" (the moment-space forcing that
               Eq. mrt_surface places inside M^-1[...]; D2Q9)
"""
import numpy as np

from . import droplet_field, grf_porous_medium, random_droplets

# Non-hydrodynamic MRT relaxation rates. D2Q9 after Lallemand & Luo (2000):
# s_e = 1.64, s_eps = 1.54, s_q = 1.9. D3Q19 after d'Humieres et al. (2002):
# s_e = 1.19, s_eps = 1.4, s_q = 1.2, s_pi = 1.4, s_m = 1.98.
MRT_D2Q9 = [0.0, 1.64, 1.54, 0.0, 1.9, 0.0, 1.9, 1.0, 1.0] + [0.0] * 10
MRT_D3Q19 = [0.0, 1.19, 1.4, 0.0, 1.2, 0.0, 1.2, 0.0, 1.2, 1.0, 1.4, 1.0, 1.4, 1.0, 1.0,
             1.0, 1.98, 1.98, 1.98]

# EOS parameter sets of the paper's thermodynamic-consistency runs (Yuan & Schaefer 2006):
EOS_PARAMS = {
    "CS": dict(eos_a=1.0, eos_b=4.0, eos_R=1.0, eos_omega=0.0),
    "PR": dict(eos_a=2.0 / 49.0, eos_b=2.0 / 21.0, eos_R=1.0, eos_omega=0.344),
    "RK": dict(eos_a=2.0 / 49.0, eos_b=2.0 / 21.0, eos_R=1.0, eos_omega=0.0),
    "RKS": dict(eos_a=2.0 / 49.0, eos_b=2.0 / 21.0, eos_R=1.0, eos_omega=0.344),
    "VdW": dict(eos_a=9.0 / 49.0, eos_b=2.0 / 21.0, eos_R=1.0, eos_omega=0.0),
}

# Liquid / vapour densities used to shape initial droplets (Maxwell construction of
# the EOS at the stated reduced temperature; only the initial condition uses them).
COEX = {
    ("CS", 0.7): (0.00929415, 0.358131),     # a = 0.5, b = 4 (coexistence is independent of a)
    ("PR", 0.6): (0.0102274, 8.72493),       # a = 2/49, b = 2/21, omega = 0.344
    ("PR", 0.8): (0.197079, 7.20405),
    ("CS", 0.8): (0.0217232, 0.307196),
    ("VdW", 0.8): (0.838834, 6.76447),
    ("VdW", 0.7): (0.448078, 7.49155),        # a = 9/49, b = 2/21
}

# Zhang-Chen / Shan-Chen mixing weight A_kk that satisfies mechanical stability
# (flat-interface coexistence equal to the Maxwell pair within 0.1 %), found by
# bisection on the vapour density of a flat liquid slab (D2Q9, BGK, tau = 1).
A_STAR = {("CS", 0.7): -0.276, ("CS", 0.8): -0.275, ("PR", 0.6): -0.233, ("PR", 0.8): -0.249}
# Two-component psi = rho fluids (Section 3.3.2 form, A = 0, g_kk = 0): with G_i = w_i / c_s^2
# the mixture's free energy c_s^2 (rho_1 ln rho_1 + rho_2 ln rho_2) + g12 rho_1 rho_2 separates
# only for g12 > c_s^2 / sqrt(rho_1 rho_2) (0.63 at rho_1 = rho_2 = 0.53). g12 = 0.8 gives sharp
# interfaces (one node between 10 % and 90 %) with 1.6 % of each component dissolved in the
# other's phase (flat D3Q19 slab, BGK tau = 1, common velocity).
G12_IMMISCIBLE = 0.8
# (major, dissolved minor) density of each bulk phase of these fluids at equilibrium, read
# off a resting drop (a phase started elsewhere relaxes to it by slow diffusion)
RHO_IMMISCIBLE = (1.07, 0.008)

# Wetting parameters of Eq. improved_virtual_density for the contact angles the workloads
# name, from tests/golden/wetting_calibration.json (FP64 oracle, drop on a flat wall).
# Two components, 45 degrees through the wetting one: each component takes the branch of
# its own wettability -- phi = WET_PHI_45 on the wetting component, drho = WET_DRHO_NW on the
# non-wetting one, which clamps its virtual density to 0 at every wall (a phi of 2.5 on the
# wetting component alone reaches 45 degrees too, but depletes the dissolved non-wetting
# component at the walls to 3e-5 and the pressure-driven porous runs blow up).
# One component, 30 degrees: phi = WET_PHI_30_PR08 for the Peng-Robinson liquid at
# T = 0.8 Tc of the sphere packs (limiter: the Maxwell pair).
WET_DRHO_NW = 1.5
WET_PHI_45 = 1.110625
WET_PHI_30_PR08 = 1.669687

# The same bisection with the moment-space forcing of the surface-tension collision
# (forcing = "moment", D2Q9 MRT with the Lallemand-Luo rates, tau = 1): that forcing lacks
# EDM's F F / rho stress, so mechanical stability needs a stronger Zhang-Chen share.
A_STAR_MOMENT = {("CS", 0.7): -0.886, ("VdW", 0.7): -0.494}
# van der Waals at T = 0.7 Tc (a = 9/49, b = 2/21: the capillary-rise fluid of Section 3.4.1):
# c_s^2 rho - p < 0 inside the loop for alpha = 1, so the pressure scaling alpha = 0.5
# keeps psi real (the Maxwell pair is that of p itself); its A* above is for that alpha
VDW07_ALPHA = 0.5

# Peng-Robinson at T = 0.6 Tc (density ratio 853): the liquid sits close to the
# repulsive pole 1/b, so the EOS is stiff and droplets blow up with alpha = 1.
# The pressure scaling alpha^k of Eq. eos_potential keeps the Maxwell pair but
# widens the interface; alpha = 0.1 with the matching mixing weight (flat-slab
# bisection as above, interface width 10) is stable in 3-D.
PR06_ALPHA = 0.1
PR06_A = -0.3227
PR06_WIDTH = 10.0
# Large droplets (R >~ 25 at tau = 1, R >~ 34 at tau = 1.5) blow up in the
# initial transient with the d'Humieres energy rates (s_e = 1.19, s_eps = 1.4):
# the compression modes are too weakly damped. tau = 1.5 with s_e = s_eps = 1/tau
# runs the 256^3 eight-droplet field 5000 steps (two seeds tried).
PR06_TAU = 1.5


def pr06_mrt_rates(tau=PR06_TAU):
    r = list(MRT_D3Q19)
    r[1] = r[2] = 1.0 / tau
    return [r, r]

# psi = exp(-1/rho) with g = -10/3: coexistence 0.367528 / 2.78279, ratio 7.57,
# the ratio of about 7.6 of the paper's performance droplet (Section 5)
EXP_G = -10.0 / 3.0
EXP_COEX = (0.367528, 2.78279)


def base_case(lattice, shape, **kw):
    case = dict(lattice=lattice, shape=tuple(shape), ncomp=1, real="f32", collision="BGK",
                velocity="component", tau=[1.0, 1.0],
                mrt_rates=[MRT_D2Q9 if lattice == "D2Q9" else MRT_D3Q19] * 2,
                psi=["eos", "eos"], eos=["CS", "CS"], T_red=[0.7, 0.7], alpha=[1.0, 1.0],
                A=[0.0, 0.0], g=[[-1.0, 0.0], [0.0, -1.0]], wet_phi=[1.0, 1.0],
                wet_drho=[0.0, 0.0], rho_lo=[0.0, 0.0], rho_hi=[1e30, 1e30],
                accel=[[0.0, 0.0, 0.0], [0.0, 0.0, 0.0]], bc=["periodic"] * 6,
                bc_rho=[[0.0, 0.0]] * 6)
    case.update(kw)
    return case


def with_eos(case, name, T_red, comps=(0, 1)):
    """Set the EOS (and its paper parameter set) of the given components."""
    c = dict(case)
    for key in ("eos_a", "eos_b", "eos_R", "eos_omega"):
        v = list(c.get(key, [0.0, 0.0]))
        v = v + [v[-1]] * (2 - len(v))
        for k in comps:
            v[k] = EOS_PARAMS[name][key]
        c[key] = v
    eos = list(c.get("eos", ["CS", "CS"]))
    tr = list(c.get("T_red", [0.7, 0.7]))
    psi = list(c.get("psi", ["eos", "eos"]))
    for k in comps:
        eos[k] = name
        tr[k] = T_red
        psi[k] = "eos"
    c.update(eos=eos, T_red=tr, psi=psi)
    return c


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def droplet_2d_cs(n=128, radius=25.0, width=5.0, real="f64"):
    """D2Q9 single-component Shan-Chen, Carnahan-Starling (a = 0.5, b = 4, R = 1,
    T = 0.7 Tc), BGK tau = 1, n x n periodic, one droplet of radius 25 with a
    tanh interface of width 5 at the centre."""
    A = A_STAR[("CS", 0.7)]
    case = base_case("D2Q9", (n, n, 1), real=real, A=[A, A])
    case = with_eos(case, "CS", 0.7)
    case["eos_a"] = [0.5, 0.5]
    rg, rl = COEX[("CS", 0.7)]
    rho = droplet_field((n, n, 1), [(n / 2.0, n / 2.0)], [radius], rl, rg, width)
    return case, dict(rho=[rho])


def droplets_3d_pr(n=256, count=8, rmin=12.0, rmax=40.0, width=PR06_WIDTH, seed=1234, real="f32",
                   shape=None, A=PR06_A, alpha=PR06_ALPHA, tau=PR06_TAU):
    """D3Q19 single-component Shan-Chen, Peng-Robinson (a = 2/49, b = 2/21, R = 1,
    omega = 0.344, T = 0.6 Tc), MRT, periodic cube, `count` droplets with seeded
    radii U[rmin, rmax] at random non-overlapping centres."""
    shape = tuple(shape) if shape is not None else (n, n, n)
    case = base_case("D3Q19", shape, real=real, collision="MRT", A=[A, A], alpha=[alpha, alpha],
                     tau=[tau, tau], mrt_rates=pr06_mrt_rates(tau))
    case = with_eos(case, "PR", 0.6)
    rg, rl = COEX[("PR", 0.6)]
    centers, radii = random_droplets(shape, count, rmin, rmax, width, seed)
    rho = droplet_field(shape, centers, radii, rl, rg, width)
    return case, dict(rho=[rho], centers=centers, radii=radii)


def droplet_3d_exp(n=256, radius=30.0, width=5.0, real="f32", shape=None):
    """The paper's performance case: D3Q19 BGK, psi = exp(-1/rho), one droplet of
    radius 30 in its vapour, periodic."""
    shape = tuple(shape) if shape is not None else (n, n, n)
    case = base_case("D3Q19", shape, real=real, psi=["exp", "exp"],
                     g=[[EXP_G, 0.0], [0.0, EXP_G]])
    rg, rl = EXP_COEX
    c = [s / 2.0 for s in shape]
    rho = droplet_field(shape, [c], [radius], rl, rg, width)
    return case, dict(rho=[rho])


POROUS_BUFFER = 8


def porous_two_component(shape=(400, 400, 400), porosity=0.15, corr_length=6.0, seed=7,
                         buffer=POROUS_BUFFER, real="f32", theta_phi=None, rho_major=RHO_IMMISCIBLE[0],
                         rho_minor=RHO_IMMISCIBLE[1], g12=G12_IMMISCIBLE, gkk=0.0, tau_w=1.0, tau_nw=1.0,
                         drho_in=0.3):
    """D3Q19 two-component Shan-Chen (psi = rho, A = 0) in a Gaussian-random-field
    porous medium (porosity 0.15, correlation length 6) with 8-lu fluid buffers.
    Component 0 = wetting phase initially saturating the domain, component 1 =
    non-wetting phase injected at x = 0 through a constant-density face against
    a constant-density outlet.

    Fluids: immiscible (g12 = G12_IMMISCIBLE, interfaces one to two nodes wide, surface
    tension 0.163 from Laplace's law), each phase at its equilibrium composition. The
    wetting component wets the solid at 45 degrees (theta_phi None: the calibrated
    virtual-density factor WET_PHI_45, with WET_DRHO_NW on the non-wetting component). drho_in raises the inlet's non-wetting density
    above the outlet's wetting one: a pressure step of about drho_in / 3 = 0.1, near the
    capillary entry pressure 2 sigma cos(45) / r of throats of radius 2.
    Viscosity ratio 1 (tau 1 for both): in this common-velocity model unequal relaxation
    times move the phases' equilibrium compositions (1:10 measured to leave 4 % dissolved
    and widen interfaces to 10 nodes), so the configured 1:10 ratio is not used."""
    nx, ny, nz = shape
    if theta_phi is None:
        theta_phi = WET_PHI_45
    solid, used_seed = grf_porous_medium(shape, porosity, corr_length, seed, buffer=buffer)
    case = base_case("D3Q19", shape, real=real, ncomp=2, psi=["rho", "rho"], velocity="common",
                     g=[[gkk, g12], [g12, gkk]], tau=[tau_w, tau_nw],
                     wet_phi=[theta_phi, 1.0], wet_drho=[0.0, WET_DRHO_NW],
                     rho_lo=[0.0, 0.0], rho_hi=[5.0, 5.0],
                     bc=["pressure", "pressure", "periodic", "periodic", "periodic", "periodic"])
    bc_rho = [[0.0, 0.0] for _ in range(6)]
    bc_rho[0] = [rho_minor, rho_major + drho_in]   # inlet: non-wetting phase
    bc_rho[1] = [rho_major, rho_minor]             # outlet: wetting phase
    case["bc_rho"] = bc_rho
    # the non-wetting phase fills the inlet buffer; the composition changes over a
    # tanh profile of width 4 at the buffer edge (a sharp step drives the dilute
    # component negative in the first steps)
    x = np.arange(nx, dtype=np.float64)
    s = 0.5 * (1.0 - np.tanh(2.0 * (x - buffer + 0.5) / 4.0))
    rho_nw = np.broadcast_to(rho_minor + (rho_major - rho_minor) * s, (nz, ny, nx)).copy()
    rho_w = np.broadcast_to(rho_minor + (rho_major - rho_minor) * (1.0 - s), (nz, ny, nx)).copy()
    return case, dict(rho=[rho_w, rho_nw], solid=solid, seed=used_seed)


def sphere_pack_batch(count=64, edge_lo=64, edge_hi=192, porosity=0.38, rmin=8.0, rmax=12.0, seed=2024,
                      real="f32", T_red=0.8, wet_phi=WET_PHI_30_PR08, buffer=6, width=5.0, tau=1.5):
    """Batch of drainage samples: each a D3Q19 box with edges U[edge_lo, edge_hi]
    (seeded per sample), an overlapping-sphere pack (radius U[rmin, rmax]) to the given
    porosity, single-component Peng-Robinson at T_red with MRT collision (tau, energy
    rates 1/tau as in the 256^3 droplet workload) and wetting
    solids (virtual density, phi > 1: wetting liquid), liquid reservoir of `buffer`
    planes at the x-min face and vapour elsewhere (tanh profile of the given width). The x faces are constant-density
    faces: inlet liquid density raised by a per-sample capillary-pressure step
    (0 to 2 %), outlet vapour density. The buffer planes are kept free of solids.
    Returns a list of (case, init) pairs."""
    from synth import sphere_pack, uniform
    rg, rl = COEX[("PR", T_red)]
    u = uniform(seed, 4 * count)
    out = []
    for s in range(count):
        nx, ny, nz = (int(edge_lo + (edge_hi - edge_lo + 1) * u[4 * s + d]) for d in range(3))
        nx, ny, nz = (min(v, edge_hi) for v in (nx, ny, nz))
        solid = sphere_pack((nx, ny, nz), rmin, rmax, porosity, seed + 1 + s)
        solid[:, :, :buffer] = 0
        solid[:, :, nx - buffer:] = 0
        step = 0.02 * u[4 * s + 3]
        case = with_eos(base_case("D3Q19", (nx, ny, nz), real=real, collision="MRT",
                                  tau=[tau, tau], mrt_rates=pr06_mrt_rates(tau),
                                  A=[A_STAR[("PR", T_red)]] * 2, wet_phi=[wet_phi, wet_phi],
                                  rho_lo=[rg, rg], rho_hi=[rl, rl],
                                  bc=["pressure", "pressure", "periodic", "periodic", "periodic", "periodic"]),
                        "PR", T_red, comps=(0,))
        bc_rho = [[0.0, 0.0] for _ in range(6)]
        bc_rho[0] = [rl * (1.0 + step), rl * (1.0 + step)]
        bc_rho[1] = [rg, rg]
        case["bc_rho"] = bc_rho
        x = np.arange(nx, dtype=float)[None, None, :] * np.ones((nz, ny, 1))
        rho = 0.5 * (rl + rg) - 0.5 * (rl - rg) * np.tanh(2.0 * (x - buffer) / width)
        out.append((case, {"rho": [rho], "solid": solid}))
    return out
