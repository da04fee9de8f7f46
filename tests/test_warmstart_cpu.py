"""Host parts of the learned warm start (paper_2506_17713_gb300/warmstart.py)."""
import numpy as np

from paper_2506_17713_gb300 import warmstart as ws


def _channel(n=16):
    solid = np.zeros((n, n, n), np.uint8)
    solid[:, 0, :] = 1                        # one wall plane: a periodic channel 15 wide
    y = np.arange(n)
    prof = np.where(y == 0, 0.0, (y - 0.5) * (n - 0.5 - y))   # halfway walls at 0.5 and n - 0.5
    shape = np.zeros((3, n, n, n))
    shape[0] = prof[None, :, None]
    return solid, shape


def test_ritz_scale_recovers_poiseuille_magnitude():
    # u = a / (2 nu) (y - 1/2)(H + 1/2 - y) between halfway walls: the energy estimate on
    # the exact shape returns the exact scale up to the lattice's first differences
    solid, shape = _channel()
    s = ws.ritz_scale(shape, solid)
    assert abs(s / (ws.ACCEL / (2 * ws.NU)) - 1) < 0.01
    # invariant to the shape's own normalisation
    assert abs(ws.ritz_scale(3.7 * shape, solid) * 3.7 / s - 1) < 1e-12


def test_features_and_targets():
    solid, shape = _channel(8)
    f = ws.features(solid)
    assert f.shape == (2, 8, 8, 8)
    assert np.array_equal(f[0], 1.0 - solid)
    assert np.all(f[1][solid == 1] == 0) and abs(f[1][:, 1, :].max() - 1.0 / 8) < 1e-6
    rho = 1.0 + 2e-4 * np.arange(8)[None, :, None] * np.ones((8, 8, 8))
    f = np.concatenate([shape * ws.ACCEL / ws.NU, rho[None] - 1.0]).astype(np.float32)
    t = ws.targets([f], [solid])[0]
    assert t.shape == (4, 8, 8, 8)
    assert abs(t[0][solid == 0].mean() - 1.0) < 1e-5
    assert np.allclose(t[3][solid == 0], ((rho - 1) / (ws.ACCEL * 8))[solid == 0], rtol=1e-5)
    assert np.all(t[3][solid == 1] == 0)
