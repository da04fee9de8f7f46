"""Capillary rise (horizontal imbibition) in a slit, Section 3.4.1, on the CUDA
path: D2Q9 MRT, surface-tension adjustment kappa = 0.5, liquid reservoir at the
channel entrance, periodic box.

The paper uses van der Waals at T = 0.7 T_c. Van der Waals needs alpha < 1 to keep
c_s^2 rho - p positive inside the loop, and its mixing weight is not calibrated
here, so the test uses the calibrated Carnahan-Starling case at T = 0.7 T_c; the
slit is 20 wide (paper: 28) and 200 long (paper: 300).

Checked:
- wetting walls (phi > 1) draw the liquid in monotonically, non-wetting walls
  (phi = 1, drho > 0) do not;
- once viscous resistance dominates, l^2 grows linearly in t (Lucas-Washburn);
- the meniscus position against the RK4 solution of the imbibition equation
  (oracle/washburn.py), with sigma from a Laplace fit and the dynamic contact
  angle from the meniscus depth h_m (theta_d = acos(4 h_m H / (H^2 + 4 h_m^2)),
  both measured on the same model). The ratio is stated and bounded; the
  simulation runs 20-25 % ahead of the equation here.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import washburn
from synth import cases

pytestmark = pytest.mark.gpu

RG, RL = cases.COEX[("CS", 0.7)]
KAPPA = 0.5
NX, NY, X0, X1, H, TW = 400, 60, 100, 300, 20, 4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_17713_gb300.build import build
    build()


def _case(shape, phi=1.0, drho=0.0):
    A = cases.A_STAR[("CS", 0.7)]
    c = cases.with_eos(cases.base_case("D2Q9", shape, collision="MRT", A=[A, A], kappa=[KAPPA, KAPPA],
                                       wet_phi=[phi, phi], wet_drho=[drho, drho]), "CS", 0.7)
    c["eos_a"] = [0.5, 0.5]
    c["rho_lo"] = [RG, RG]
    c["rho_hi"] = [RL, RL]
    return c


def _sigma():
    from paper_2506_17713_gb300 import Lattice
    pts = []
    for R in (12, 16, 20):
        case, init = cases.droplet_2d_cs(n=96, radius=R)
        case = dict(case, collision="MRT", kappa=[KAPPA, KAPPA])
        lat = Lattice(case)
        lat.init_fields(0, init["rho"][0])
        lat.step(8000)
        r, _ = lat.macroscopic_host(0)
        r = r.astype(float)
        rin, rout = r[0, 45:51, 45:51].mean(), r[0, :4, :4].mean()
        dp = oracle.bulk_pressure(case, 0, rin) - oracle.bulk_pressure(case, 0, rout)
        pts.append((1.0 / math.sqrt((r > 0.5 * (rin + rout)).sum() / math.pi), dp))
    x = np.array(pts)
    (sig, _), *_ = np.linalg.lstsq(np.vstack([x[:, 0], np.ones(3)]).T, x[:, 1], rcond=None)
    return sig


def _imbibition(phi, drho=0.0, steps=28000, every=500):
    """meniscus position l(t) on the channel axis and next to the wall"""
    from paper_2506_17713_gb300 import Lattice
    y0 = (NY - H) // 2
    solid = np.zeros((1, NY, NX), np.uint8)
    solid[0, y0 - TW:y0, X0:X1] = 1
    solid[0, y0 + H:y0 + H + TW, X0:X1] = 1
    X = np.arange(NX)[None, None, :] * np.ones((1, NY, 1))
    rho = 0.5 * (RL + RG) - 0.5 * (RL - RG) * np.tanh(2 * (X - X0) / 4.0)
    lat = Lattice(_case((NX, NY, 1), phi, drho))
    lat.set_geometry(solid)
    lat.init_fields(0, rho)
    mid = 0.5 * (RL + RG)

    def front(r, row):
        seg = r[row, X0:X1]
        idx = np.where(seg < mid)[0]
        if len(idx) == 0:
            return float(X1 - X0)
        i = idx[0]
        return 0.0 if i == 0 else i - 1 + (seg[i - 1] - mid) / (seg[i - 1] - seg[i])

    t, lc, lw = [], [], []
    for b in range(steps // every):
        lat.step(every)
        r, _ = lat.macroscopic_host(0)
        r = r[0].astype(float)
        t.append((b + 1) * every)
        lc.append(front(r, y0 + H // 2))
        lw.append(front(r, y0))
    return np.array(t, float), np.array(lc), np.array(lw)


def test_wetting_slit_imbibes_and_follows_the_imbibition_equation():
    t, lc, lw = _imbibition(1.15)
    inside = lc < 0.9 * (X1 - X0)
    t, lc, lw = t[inside], lc[inside], lw[inside]
    assert len(t) > 20 and lc[-1] > 0.3 * (X1 - X0)
    assert np.all(np.diff(lc) > 0)                                  # advances monotonically
    # viscous regime: l^2 linear in t over the second half
    h = len(t) // 2
    p = np.polyfit(t[h:], lc[h:] ** 2, 1)
    pred = np.polyval(p, t[h:])
    r2 = 1 - ((lc[h:] ** 2 - pred) ** 2).sum() / ((lc[h:] ** 2 - (lc[h:] ** 2).mean()) ** 2).sum()
    assert r2 > 0.99
    # against the imbibition equation with the model's own sigma and dynamic angle
    hm = np.abs(lw - lc)
    theta = float(np.mean(np.arccos(4 * hm[h:] * H / (H * H + 4 * hm[h:] ** 2))))
    sig = _sigma()
    nu = (1.0 - 0.5) / 3.0
    ode = washburn.meniscus(list(t), sig, theta, H, X1 - X0, RL, RG, RL * nu, RG * nu, dt=0.5)
    ratio = lc[-1] / ode[-1]
    print("sigma %.5f, theta_d %.1f deg, l_LBM %.1f, l_ODE %.1f, ratio %.3f"
          % (sig, math.degrees(theta), lc[-1], ode[-1], ratio))
    assert 0.8 < ratio < 1.4


def test_non_wetting_slit_stays_empty():
    # phi = 1, drho > 0: contact angle above 90 degrees (Eq. improved_virtual_density)
    t, lc, _ = _imbibition(1.0, drho=0.05, steps=8000)
    assert lc.max() < 6.0
