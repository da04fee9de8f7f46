"""Write tests/golden/wetting_calibration.json: the virtual-density parameter phi
(Eq. improved_virtual_density, Section 2.4) that gives the contact angle a workload
names, found with the FP64 oracle alone.

  sphere-pack drainage fluid (Peng-Robinson, T = 0.8 Tc):  30 degrees
  porous drainage fluids (two components, psi = rho):     45 degrees (through the wetting one;
                                                          phi on it, drho = WET_DRHO_NW on the other)
  capillary-rise fluid (van der Waals, T = 0.7 Tc,
    kappa = 0.5, Section 3.4.1):                          19 degrees

The angle is measured on a drop resting on a flat wall (tests/wetting.py). theta(phi)
decreases monotonically; the script brackets the target and bisects to 0.25 degrees.
Run from the repository root: python tests/golden/make_wetting_calibration.py [model ...]
(no model: all; the others keep their stored entries).
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import wetting  # noqa: E402

TARGETS = {
    "pr08": dict(theta=30.0, shape=(200, 60, 2), radius=22.0, steps=6000, lo=1.0, hi=2.5),
    "two_component": dict(theta=45.0, shape=(120, 60, 2), radius=22.0, steps=6000, lo=0.95, hi=1.4),
    "vdw07_kappa": dict(theta=19.0, shape=(320, 60, 1), radius=30.0, steps=8000, lo=1.4, hi=2.5),
}


def calibrate(model, t):
    # each drop starts as a cap at the target angle: near the calibrated phi it barely moves,
    # and away from it, it moves towards its own angle, which keeps the bisection's sign
    f = lambda phi: wetting.oracle_angle(model, phi, t["steps"], shape=t["shape"], radius=t["radius"],
                                         theta0=t["theta"])
    lo, hi = t["lo"], t["hi"]
    th_lo, th_hi = f(lo), f(hi)
    print(model, "bracket", lo, th_lo, hi, th_hi, flush=True)
    assert th_lo > t["theta"] > th_hi, "target not bracketed"
    best = (abs(th_lo - t["theta"]), lo, th_lo)
    for _ in range(12):
        mid = 0.5 * (lo + hi)
        th = f(mid)
        print(model, "phi %.5f theta %.3f" % (mid, th), flush=True)
        best = min(best, (abs(th - t["theta"]), mid, th))
        if abs(th - t["theta"]) < 0.25:
            break
        if th > t["theta"]:
            lo = mid
        else:
            hi = mid
    # the contact line of a sharp interface can hop between lattice positions, which makes
    # theta(phi) steep in places; keep, among phi within 0.03 of the bisection's result, one
    # whose angle is within 1 degree of the target and changes least over +-0.01
    phis = [round(best[1] + 0.01 * k, 6) for k in range(-4, 5)]
    ths = [f(p) for p in phis]
    print(model, "neighbourhood", list(zip(phis, ths)), flush=True)
    ok = [i for i in range(1, len(phis) - 1) if abs(ths[i] - t["theta"]) < 1.0]
    i = min(ok, key=lambda i: abs(ths[i + 1] - ths[i - 1]))
    return phis[i], ths[i]


def main():
    path = os.path.join(HERE, "wetting_calibration.json")
    out = {}
    if len(sys.argv) > 1 and os.path.exists(path):
        with open(path) as fh:
            out = json.load(fh)
    for model, t in TARGETS.items():
        if len(sys.argv) > 1 and model not in sys.argv[1:]:
            continue
        phi, th = calibrate(model, t)
        out[model] = dict(theta_set=t["theta"], phi=round(phi, 6), theta_oracle=round(th, 4),
                          shape=list(t["shape"]), radius=t["radius"], steps=t["steps"], theta0=t["theta"])
    out["_source"] = ("FP64 oracle, sessile drop on a flat wall, circle fit of the half-way iso-line "
                      "(tests/wetting.py); written by tests/golden/make_wetting_calibration.py")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
