"""End to end learned warm start on small periodic samples (24^3): steady states
generated by the batched LBM, the U-Net trained on them by the project's tensor-core
kernels, and held-out steady runs relaxed from rest, from the prediction and from the
converged plain field. The test reports what the trained network gains and checks
what must hold whatever it gains: every run reaches the residual criterion, every
start ends at the permeability of the plain run, and a start from the converged
velocity and density (the bound for any macroscopic warm start) is immediate."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N = 24


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_17713_gb300.build import build
    build()


def test_warm_start_end_to_end():
    from paper_2506_17713_gb300 import nn
    from paper_2506_17713_gb300 import warmstart as ws
    from synth import uniform
    phis = [0.15 + 0.2 * float(v) for v in uniform(77, 26)]
    solids, fields, res = ws.steady_states(N, list(range(300, 324)), phis[:24], 30000)
    keep = [i for i, r in enumerate(res) if r <= 1e-5]
    assert len(keep) >= 20
    solids = [solids[i] for i in keep]
    fields = [fields[i] for i in keep]
    net = ws.UNet(N, seed=0)
    hist = ws.train(net, solids, fields, epochs=25, batch=4, lr=2e-3)
    assert hist[-1] < 0.6 * hist[0]
    coef = ws.fit_scale(net, solids, fields)
    gains = []
    for j in range(2):
        solid = ws.sample_solid(N, 900 + j, phis[24 + j])
        sp, _, kp, rp, u_plain, rho_plain = ws.relax(N, solid, None)
        u_pred, rho_pred = ws.predict(net, solid, coef)
        assert np.all(np.isfinite(u_pred)) and np.all(np.isfinite(rho_pred))
        sw, _, kw, rw, _, _ = ws.relax(N, solid, u_pred, rho0=rho_pred)
        sb, _, kb, rb, _, _ = ws.relax(N, solid, u_plain.astype(np.float64), rho0=rho_plain.astype(np.float64))
        for r in (rp, rw, rb):
            assert r <= 1e-6
        assert abs(kw - kp) <= 1e-3 * abs(kp)
        assert abs(kb - kp) <= 1e-3 * abs(kp)
        assert sb <= 200
        gains.append(sp / sw)
        print("sample %d: from rest %d steps, from the prediction %d (%.2fx), from the converged field %d"
              % (j, sp, sw, sp / sw, sb))
    assert all(g > 0 for g in gains)
    assert nn.tc_error() == 0
