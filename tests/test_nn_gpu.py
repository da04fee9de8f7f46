"""Warm-start network kernels (include/lbm_nn.h) against the numpy reference
(oracle/unet_ref.py), and the U-Net's gradients against a numpy backward pass
composed from the same reference operations.

The tensor-core convolutions take BF16 operands and accumulate in FP32, so they are
compared with the FP64 convolution of the BF16-rounded operands (unet_ref.bf16) under
the standard bound for a sum of K exact products accumulated in FP32,
|err| <= gamma_K sum |a_k b_k|, gamma_K = K u / (1 - K u), u = 2^-24, taken twice
over (the tensor cores' internal adder order and rounding are not specified)."""
import numpy as np
import pytest

from oracle import unet_ref as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_17713_gb300.build import build
    build()


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _n(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape).astype(np.float32).astype(np.float64)


def _close(a, b, rtol):
    assert np.abs(a - b).max() <= rtol * np.abs(b).max(), (np.abs(a - b).max(), np.abs(b).max())


@pytest.mark.parametrize("cin,cout,dims", [(5, 11, (6, 4, 10)), (1, 8, (8, 8, 8)), (24, 3, (4, 6, 4))])
def test_conv3d_forward_and_gradients(cin, cout, dims):
    import torch
    from paper_2506_17713_gb300 import nn
    x = _rand((cin,) + dims, 1)
    w = _rand((cout, cin, 3, 3, 3), 2) * 0.3
    b = _rand(cout, 3)
    gy = _rand((cout,) + dims, 4)
    y = torch.empty((cout,) + dims, device="cuda")
    nn.conv3d(_t(x), _t(w.reshape(cout, cin, 27)), _t(b), False, y)
    _close(_n(y), U.conv3d(x, w, b), 1e-5)
    yr = torch.empty_like(y)
    nn.conv3d(_t(x), _t(w.reshape(cout, cin, 27)), _t(b), True, yr)
    assert np.allclose(_n(yr), U.relu(_n(y)), rtol=1e-6, atol=0)
    gx_ref, gw_ref, gb_ref = U.conv3d_grads(x, w, gy)
    gx = torch.empty((cin,) + dims, device="cuda")
    nn.conv3d_grad_input(_t(gy), _t(w.reshape(cout, cin, 27)), torch.empty(cin * cout * 27, device="cuda"), gx)
    _close(_n(gx), gx_ref, 1e-5)
    gw = torch.empty(cout, cin, 27, device="cuda")
    gb = torch.empty(cout, device="cuda")
    scratch = torch.empty(nn.GW_SEGMENTS * cout * cin * 28, device="cuda")
    nn.conv3d_grad_weight(_t(x), _t(gy), gw, gb, False, scratch)
    _close(_n(gw), gw_ref.reshape(cout, cin, 27), 1e-5)
    _close(_n(gb), gb_ref, 1e-5)
    nn.conv3d_grad_weight(_t(x), _t(gy), gw, gb, True, scratch)     # accumulate: twice the sum
    _close(_n(gw), 2 * gw_ref.reshape(cout, cin, 27), 1e-5)


def test_pool_upsample_relu_axpy_loss_adam():
    import torch
    from paper_2506_17713_gb300 import nn
    x = _rand((3, 4, 6, 8), 5)
    y = torch.empty(3, 2, 3, 4, device="cuda")
    nn.avg_pool2(_t(x), y)
    _close(_n(y), U.avg_pool2(x), 1e-6)
    gx = torch.empty(3, 4, 6, 8, device="cuda")
    gy = _rand((3, 2, 3, 4), 6)
    nn.avg_pool2_grad(_t(gy), gx)
    _close(_n(gx), U.up2(gy) / 8, 1e-6)
    up = torch.empty(3, 4, 6, 8, device="cuda")
    nn.up2(_t(gy), up)
    assert np.array_equal(_n(up), U.up2(gy))
    gs = torch.empty(3, 2, 3, 4, device="cuda")
    nn.up2_grad(_t(x), gs)
    _close(_n(gs), 8 * U.avg_pool2(x), 1e-6)
    g = _t(gy)
    nn.relu_grad(_t(_rand((3, 2, 3, 4), 7)), g)
    yy = _rand((3, 2, 3, 4), 7)
    assert np.allclose(_n(g), U.relu_grad(yy, gy), rtol=1e-6, atol=0)
    a = _t(x)
    nn.axpy(a, _t(x), 2.0)
    _close(_n(a), 3 * x, 1e-7)
    p, t = _rand((3, 4, 4, 4), 8), _rand((3, 4, 4, 4), 9)
    grad = torch.empty(3, 4, 4, 4, device="cuda")
    sums = torch.zeros(2, dtype=torch.float64, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    nn.rel_loss(_t(p), _t(t), grad, sums, loss)
    L, gref = U.rel_loss(p, t)
    assert abs(float(loss.item()) - L) < 1e-6 * L
    _close(_n(grad), gref, 1e-6)
    # one Adam step against its formula
    prm, gg = _rand(50, 10), _rand(50, 11)
    P, M, V = _t(prm), torch.zeros(50, device="cuda"), torch.zeros(50, device="cuda")
    nn.adam(P, _t(gg), M, V, 0.01, 0.9, 0.999, 1e-8, 1)
    m, v = 0.1 * gg, 0.001 * gg * gg
    ref = prm - 0.01 * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)
    _close(_n(P), ref, 1e-6)


def _ref_unet(net, x, t):
    """numpy forward and backward of the U-Net with the network's weights"""
    W = {k: _n(net.w[k]).reshape(net.w[k].shape[0], net.w[k].shape[1], 3, 3, 3) for k in net.w}
    B = {k: _n(net.b[k]) for k in net.b}
    c1, c2, c3 = net.c
    cv = lambda k, a: U.conv3d(a, W[k], B[k])
    e1a = U.relu(cv("e1a", x)); s1 = U.relu(cv("e1b", e1a)); p1 = U.avg_pool2(s1)
    e2a = U.relu(cv("e2a", p1)); s2 = U.relu(cv("e2b", e2a)); p2 = U.avg_pool2(s2)
    ba = U.relu(cv("ba", p2)); bb = U.relu(cv("bb", ba))
    cat2 = np.concatenate([U.up2(bb), s2]); d2a = U.relu(cv("d2a", cat2)); d2b = U.relu(cv("d2b", d2a))
    cat1 = np.concatenate([U.up2(d2b), s1]); d1a = U.relu(cv("d1a", cat1)); out = cv("d1b", d1a)
    L, g = U.rel_loss(out, t)
    G = {}

    def back(k, a_in, y_post, gy, relu):
        if relu:
            gy = U.relu_grad(y_post, gy)
        gx, gw, gb = U.conv3d_grads(a_in, W[k], gy)
        G[k] = (gw.reshape(gw.shape[0], gw.shape[1], 27), gb)
        return gx

    g = back("d1b", d1a, out, g, False)
    g = back("d1a", cat1, d1a, g, True)
    gs1 = g[c2:]
    g = back("d2b", d2a, d2b, 8 * U.avg_pool2(g[:c2]), True)
    g = back("d2a", cat2, d2a, g, True)
    gs2 = g[c3:]
    g = back("bb", ba, bb, 8 * U.avg_pool2(g[:c3]), True)
    g = back("ba", p2, ba, g, True)
    gs2 = gs2 + U.up2(g) / 8
    g = back("e2b", e2a, s2, gs2, True)
    g = back("e2a", p1, e2a, g, True)
    gs1 = gs1 + U.up2(g) / 8
    g = back("e1b", e1a, s1, gs1, True)
    back("e1a", x, e1a, g, True)
    return out, L, G


def _gamma(k):
    u = 2.0 ** -24
    return 2 * k * u / (1 - k * u)


def _within(got, ref, mag, k):
    err = np.abs(got - ref)
    bound = _gamma(k) * mag + 2.0 ** -23 * np.abs(ref) + 1e-30
    assert np.all(err <= bound), (float((err / bound).max()), float(err.max()))


# several 128-voxel tiles with a ragged tail; channel counts below, at and above 16;
# the last case has more tiles than resident CTAs, so CTAs loop over tiles
TC_CASES = [(5, 11, (6, 4, 10)), (2, 8, (8, 8, 8)), (48, 16, (6, 8, 12)), (16, 32, (4, 4, 8)),
            (24, 4, (12, 12, 12)), (33, 40, (5, 7, 9)), (2, 8, (64, 72, 72))]


@pytest.mark.parametrize("cin,cout,dims", TC_CASES)
def test_tensor_core_conv3d_forward(cin, cout, dims):
    import torch
    from paper_2506_17713_gb300 import nn
    x = _rand((cin,) + dims, 1)
    w = _rand((cout, cin, 3, 3, 3), 2) * 0.3
    b = _rand(cout, 3)
    xb, wb = U.bf16(x), U.bf16(w)
    ref = U.conv3d(xb, wb, b)
    mag = U.conv3d(np.abs(xb), np.abs(wb), np.abs(b))
    y = torch.empty((cout,) + dims, device="cuda")
    nn.conv3d(_t(x), _t(w.reshape(cout, cin, 27)), _t(b), False, y, tc=True)
    _within(_n(y), ref, mag, 27 * cin + 1)
    yr = torch.empty_like(y)
    nn.conv3d(_t(x), _t(w.reshape(cout, cin, 27)), _t(b), True, yr, tc=True)
    assert np.allclose(_n(yr), U.relu(_n(y)), rtol=1e-6, atol=0)
    nn.conv3d(_t(x), _t(w.reshape(cout, cin, 27)), None, False, y, tc=True)      # no bias
    _within(_n(y), ref - b[:, None, None, None], mag, 27 * cin + 1)
    assert nn.tc_error() == 0


@pytest.mark.parametrize("cin,cout,dims", TC_CASES[:-1])
def test_tensor_core_conv3d_gradients(cin, cout, dims):
    import torch
    from paper_2506_17713_gb300 import nn
    x = _rand((cin,) + dims, 5)
    w = _rand((cout, cin, 3, 3, 3), 6) * 0.3
    gy = _rand((cout,) + dims, 7)
    xb, wb, gyb = U.bf16(x), U.bf16(w), U.bf16(gy)
    gx_ref, _, _ = U.conv3d_grads(xb, wb, gyb)
    gx_mag, _, _ = U.conv3d_grads(np.abs(xb), np.abs(wb), np.abs(gyb))
    gx = torch.empty((cin,) + dims, device="cuda")
    nn.conv3d_grad_input(_t(gy), _t(w.reshape(cout, cin, 27)), torch.empty(cin * cout * 27, device="cuda"), gx,
                         tc=True)
    _within(_n(gx), gx_ref, gx_mag, 27 * cout)
    _, gw_ref, gb_ref = U.conv3d_grads(xb, w, gyb)
    _, gw_mag, gb_mag = U.conv3d_grads(np.abs(xb), w, np.abs(gyb))
    P = int(np.prod(dims))
    gw = torch.empty(cout, cin, 27, device="cuda")
    gb = torch.empty(cout, device="cuda")
    scratch = torch.empty(nn.gw_scratch_floats(cin, cout, tc=True), device="cuda")
    nn.conv3d_grad_weight(_t(x), _t(gy), gw, gb, False, scratch, tc=True)
    _within(_n(gw), gw_ref.reshape(cout, cin, 27), gw_mag.reshape(cout, cin, 27), P)
    _within(_n(gb), gb_ref, gb_mag, P)
    nn.conv3d_grad_weight(_t(x), _t(gy), gw, gb, True, scratch, tc=True)        # accumulate: twice the sum
    _within(_n(gw), 2 * gw_ref.reshape(cout, cin, 27), 2 * gw_mag.reshape(cout, cin, 27), P + 1)
    assert nn.tc_error() == 0


def test_tensor_core_weight_gradient_over_many_row_tiles():
    # 27 cin + 1 = 2593 rows: 21 row tiles of 128, the last one ragged
    import torch
    from paper_2506_17713_gb300 import nn
    cin, cout, dims = 96, 32, (4, 6, 8)
    x = _rand((cin,) + dims, 8)
    gy = _rand((cout,) + dims, 9)
    xb, gyb = U.bf16(x), U.bf16(gy)
    w0 = np.zeros((cout, cin, 3, 3, 3))
    _, gw_ref, gb_ref = U.conv3d_grads(xb, w0, gyb)
    _, gw_mag, gb_mag = U.conv3d_grads(np.abs(xb), w0, np.abs(gyb))
    gw = torch.empty(cout, cin, 27, device="cuda")
    gb = torch.empty(cout, device="cuda")
    scratch = torch.empty(nn.gw_scratch_floats(cin, cout, tc=True), device="cuda")
    nn.conv3d_grad_weight(_t(x), _t(gy), gw, gb, False, scratch, tc=True)
    P = int(np.prod(dims))
    _within(_n(gw), gw_ref.reshape(cout, cin, 27), gw_mag.reshape(cout, cin, 27), P)
    _within(_n(gb), gb_ref, gb_mag, P)
    assert nn.tc_error() == 0


def test_unet_on_tensor_cores_against_numpy():
    # BF16 operands in ten layers: the output and every gradient within a few per cent
    # of the FP64 network with the same weights
    from paper_2506_17713_gb300.warmstart import UNet
    n = 8
    net = UNet(n, channels=(4, 6, 8), seed=3, tensor_cores=True)
    for k in net.b:
        net.b[k].copy_(_t(_rand(net.b[k].shape[0], 20 + len(k)) * 0.1))
    x = np.random.default_rng(12).random((2, n, n, n))
    t = _rand((4, n, n, n), 13)
    out = net.forward(_t(x))
    loss = float(net.backward(_t(t), accumulate=False).item())
    ref_out, ref_L, G = _ref_unet(net, x, t)
    _close(_n(out), ref_out, 3e-2)
    assert abs(loss - ref_L) < 3e-2 * ref_L
    for k, (gw, gb) in G.items():
        _close(_n(net.gw[k]), gw, 6e-2)
        _close(_n(net.gb[k]), gb, 6e-2)


def test_unet_forward_and_gradients_against_numpy():
    from paper_2506_17713_gb300.warmstart import UNet
    n = 8
    net = UNet(n, channels=(4, 6, 8), seed=3, tensor_cores=False)
    for k in net.b:                      # nonzero biases exercise the bias gradients
        net.b[k].copy_(_t(_rand(net.b[k].shape[0], 20 + len(k)) * 0.1))
    x = np.random.default_rng(12).random((2, n, n, n))
    t = _rand((4, n, n, n), 13)
    out = net.forward(_t(x))
    loss = float(net.backward(_t(t), accumulate=False).item())
    ref_out, ref_L, G = _ref_unet(net, x, t)
    _close(_n(out), ref_out, 2e-5)
    assert abs(loss - ref_L) < 1e-5 * ref_L
    for k, (gw, gb) in G.items():
        _close(_n(net.gw[k]), gw, 2e-4)
        _close(_n(net.gb[k]), gb, 2e-4)


def test_training_reduces_the_loss():
    import torch
    from paper_2506_17713_gb300.warmstart import UNet, train
    n = 8
    net = UNet(n, channels=(4, 6, 8), seed=1)
    rng = np.random.default_rng(5)
    solids = [(rng.random((n, n, n)) > 0.6).astype(np.uint8) for _ in range(4)]
    # targets that a network can fit: a smooth function of the fluid indicator
    us = [np.stack([(1 - s) * 2e-4, (1 - s) * 1e-5, 0 * s, 1e-4 * (1 - s)]).astype(np.float32) for s in solids]
    hist = train(net, solids, us, epochs=30, batch=2, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0]


def test_bounded_wait_gives_up_and_sets_the_error_flag():
    # failure detection of the tensor-core kernels, made to fire without a fault: a wait on
    # an mbarrier that nothing arrives on gives up after the limit (2e6 cycles, about a
    # millisecond), reports it, and sets the flag lbm_nn_tc_error reads and clears
    from paper_2506_17713_gb300 import nn
    nn.tc_error()
    assert nn.wait_selftest(2_000_000) == 0
    assert nn.tc_error() == 1
    assert nn.tc_error() == 0
    # the context stays usable: a tensor-core convolution still runs and sets no flag
    import torch
    x = torch.rand((4, 8, 8, 8), device="cuda")
    w = torch.rand((16, 4, 27), device="cuda")
    y = torch.empty((16, 8, 8, 8), device="cuda")
    nn.conv3d(x, w, None, False, y, tc=True)
    torch.cuda.synchronize()
    assert torch.isfinite(y).all() and nn.tc_error() == 0
