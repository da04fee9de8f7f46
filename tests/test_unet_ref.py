"""The numpy reference of the warm-start network's operations (oracle/unet_ref.py)
pinned against brute-force definitions, finite differences and identities."""
import numpy as np

from oracle import unet_ref as U


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_conv3d_against_per_voxel_brute_force():
    x = _rand((2, 4, 3, 5), 1)
    w = _rand((3, 2, 3, 3, 3), 2)
    b = _rand(3, 3)
    y = U.conv3d(x, w, b)
    C, D, H, W = x.shape
    for (o, z, yy, xx) in [(0, 0, 0, 0), (2, 3, 2, 4), (1, 1, 2, 0)]:
        v = b[o]
        for i in range(C):
            for a in range(3):
                for c in range(3):
                    for e in range(3):
                        v += w[o, i, a, c, e] * x[i, (z + a - 1) % D, (yy + c - 1) % H, (xx + e - 1) % W]
        assert abs(y[o, z, yy, xx] - v) < 1e-12


def test_identity_kernel_and_shift_kernel():
    x = _rand((1, 4, 4, 4), 4)
    w = np.zeros((1, 1, 3, 3, 3))
    w[0, 0, 1, 1, 1] = 1.0
    assert np.array_equal(U.conv3d(x, w, [0.0])[0], x[0])
    w[:] = 0
    w[0, 0, 1, 1, 2] = 1.0                      # picks x[z, y, x + 1]
    assert np.array_equal(U.conv3d(x, w, [0.0])[0], np.roll(x[0], -1, axis=2))


def test_conv3d_gradients_by_finite_differences():
    x = _rand((2, 4, 4, 4), 5)
    w = _rand((2, 2, 3, 3, 3), 6)
    b = _rand(2, 7)
    g = _rand((2, 4, 4, 4), 8)
    gx, gw, gb = U.conv3d_grads(x, w, g)
    f = lambda xx, ww, bb: np.sum(g * U.conv3d(xx, ww, bb))
    h = 1e-6
    for idx in [(0, 1, 2, 3), (1, 3, 0, 0)]:
        xp = x.copy(); xp[idx] += h
        xm = x.copy(); xm[idx] -= h
        assert abs((f(xp, w, b) - f(xm, w, b)) / (2 * h) - gx[idx]) < 1e-6
    for idx in [(0, 1, 0, 2, 1), (1, 0, 2, 2, 2)]:
        wp = w.copy(); wp[idx] += h
        wm = w.copy(); wm[idx] -= h
        assert abs((f(x, wp, b) - f(x, wm, b)) / (2 * h) - gw[idx]) < 1e-6
    assert np.allclose(gb, g.reshape(2, -1).sum(axis=1))


def test_pool_and_upsample_are_adjoint_up_to_the_block_size():
    x = _rand((2, 4, 6, 8), 9)
    y = _rand((2, 2, 3, 4), 10)
    # <avg_pool2(x), y> = <x, up2(y)> / 8
    assert abs(np.sum(U.avg_pool2(x) * y) - np.sum(x * U.up2(y)) / 8) < 1e-12


def test_relative_loss_gradient():
    p = _rand((3, 2, 2, 2), 11)
    t = _rand((3, 2, 2, 2), 12)
    L, g = U.rel_loss(p, t)
    h = 1e-7
    pp = p.copy(); pp[1, 0, 1, 1] += h
    assert abs((U.rel_loss(pp, t)[0] - L) / h - g[1, 0, 1, 1]) < 1e-5


def test_leaky_relu_and_its_gradient():
    x = np.array([-2.0, -0.5, 0.0, 0.3, 4.0])
    assert np.allclose(U.relu(x), [-0.02, -0.005, 0.0, 0.3, 4.0])
    g = np.ones(5)
    assert np.allclose(U.relu_grad(U.relu(x), g), [0.01, 0.01, 0.01, 1.0, 1.0])


def test_bf16_rounding_against_exact_cases():
    # bfloat16 keeps 8 significant bits: spacing 2^-7 on [1, 2)
    u = 2.0 ** -7
    cases = [(1.0, 1.0), (1.0 + u, 1.0 + u), (1.0 + u / 2, 1.0),          # tie -> even (1.0)
             (1.0 + 3 * u / 2, 1.0 + 2 * u),                                  # tie -> even (1 + 2u)
             (1.0 + u / 2 + 2.0 ** -20, 1.0 + u),                             # above the tie
             (1.0 + u / 2 - 2.0 ** -20, 1.0),                                 # below the tie
             (-3.0 - 0.75 * 2 * u, -3.0 - 2 * u),                             # spacing 2u on [2, 4)
             (2.0 - u / 4, 2.0),                                              # carries into the exponent
             (0.0, 0.0), (2.0 ** -130, 2.0 ** -130)]                          # zero, subnormal kept exactly
    for v, r in cases:
        assert U.bf16(np.array([v]))[0] == r, (v, U.bf16(np.array([v]))[0], r)


def test_bf16_rounding_error_bound_and_idempotence():
    x = _rand(10000, 30) * 10.0 ** np.random.default_rng(31).integers(-6, 6, 10000)
    r = U.bf16(x)
    xf = x.astype(np.float32).astype(np.float64)
    assert np.all(np.abs(r - xf) <= 2.0 ** -8 * np.abs(xf))      # unit roundoff of 8 significant bits
    assert np.array_equal(U.bf16(r), r)
    # every result has at most 8 significant bits
    m, _ = np.frexp(r[r != 0])
    assert np.array_equal(m * 2 ** 8, np.round(m * 2 ** 8))
