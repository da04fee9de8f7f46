"""Contact angle of the CUDA path against the FP64 oracle (Section 2.4, Eq.
improved_virtual_density): drops on a flat wall with the calibrated wetting parameters of
the two workloads that name an angle (tests/golden/wetting_calibration.json), measured the
same way on both sides (tests/wetting.py). The physics observables of the GPU path must
agree with the oracle's within 1 %.
"""
import numpy as np
import pytest

import oracle
import wetting

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_17713_gb300.build import build
    build()


@pytest.mark.parametrize("model", ["pr08", "two_component", "vdw07_kappa"])
def test_contact_angle_matches_oracle_within_one_percent(model):
    from paper_2506_17713_gb300 import Lattice
    cal = wetting.calibration()[model]
    kw = dict(shape=tuple(cal["shape"]), radius=cal["radius"], theta0=cal["theta0"])
    angles = {}
    for side, real in (("gpu", "f32"), ("oracle", "f64")):
        case, rhos, solid, ind = wetting.sessile_case(model, cal["phi"], real=real, **kw)
        sim = Lattice(case) if side == "gpu" else oracle.OracleSim(case)
        sim.set_geometry(solid)
        for k, r in enumerate(rhos):
            sim.init_fields(k, r)
        sim.step(cal["steps"])
        if side == "gpu":
            dens = [sim.macroscopic_host(k)[0].astype(np.float64).mean(axis=0) for k in range(sim.K)]
            sim.close()
        else:
            dens = [sim.macroscopic(k)[0].mean(axis=0) for k in range(sim.K)]
        a, mid = ind(dens)
        angles[side] = wetting.circle_angle(a, mid)
    print("%s: set %.1f, oracle %.3f, GPU %.3f degrees" % (model, cal["theta_set"], angles["oracle"], angles["gpu"]))
    assert abs(angles["gpu"] - angles["oracle"]) <= 0.01 * angles["oracle"]
    assert abs(angles["oracle"] - cal["theta_set"]) < 1.0
