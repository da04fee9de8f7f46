"""ctypes binding of the warm-start network kernels (include/lbm_nn.h): argument
marshalling only. Tensors are torch CUDA float32 tensors, contiguous,
channel-major [C, D, H, W]."""
import ctypes as C

from .lbm import LbmError, library as _lbm_library

EXPORTS = ["lbm_nn_conv3d", "lbm_nn_conv3d_grad_input", "lbm_nn_conv3d_grad_weight", "lbm_nn_axpy", "lbm_nn_relu_grad",
           "lbm_nn_avg_pool2", "lbm_nn_avg_pool2_grad", "lbm_nn_up2", "lbm_nn_up2_grad", "lbm_nn_rel_loss",
           "lbm_nn_adam", "lbm_nn_conv3d_tc", "lbm_nn_conv3d_tc_grad_input", "lbm_nn_conv3d_tc_grad_weight",
           "lbm_nn_tc_error", "lbm_nn_wait_selftest"]
GW_SEGMENTS = 64          # LBM_NN_GW_SEGMENTS: scratch of conv3d_grad_weight, 64 cout cin 28 floats
GW_TC_SEGMENTS = 512      # LBM_NN_GW_TC_SEGMENTS: scratch of the tensor-core form, 512 cout (27 cin + 1) floats


def gw_scratch_floats(cin, cout, tc=False):
    return GW_TC_SEGMENTS * cout * (27 * cin + 1) if tc else GW_SEGMENTS * cout * cin * 28

_ready = False


def library():
    global _ready
    L = _lbm_library()
    if not _ready:
        vp, i, ll, f = C.c_void_p, C.c_int, C.c_longlong, C.c_float
        L.lbm_nn_conv3d.argtypes = [vp, i, i, i, i, vp, vp, i, i, vp, vp]
        L.lbm_nn_conv3d_grad_input.argtypes = [vp, i, i, i, i, vp, i, vp, vp, vp]
        L.lbm_nn_conv3d_grad_weight.argtypes = [vp, i, vp, i, i, i, i, vp, vp, i, vp, vp]
        L.lbm_nn_axpy.argtypes = [vp, vp, ll, f, vp]
        L.lbm_nn_relu_grad.argtypes = [vp, vp, ll, vp]
        L.lbm_nn_avg_pool2.argtypes = [vp, i, i, i, i, vp, vp]
        L.lbm_nn_avg_pool2_grad.argtypes = [vp, i, i, i, i, vp, vp]
        L.lbm_nn_up2.argtypes = [vp, i, i, i, i, vp, vp]
        L.lbm_nn_up2_grad.argtypes = [vp, i, i, i, i, vp, vp]
        L.lbm_nn_rel_loss.argtypes = [vp, vp, ll, vp, vp, vp, vp]
        L.lbm_nn_adam.argtypes = [vp, vp, vp, vp, ll, f, f, f, f, f, f, vp]
        L.lbm_nn_conv3d_tc.argtypes = L.lbm_nn_conv3d.argtypes
        L.lbm_nn_conv3d_tc_grad_input.argtypes = L.lbm_nn_conv3d_grad_input.argtypes
        L.lbm_nn_conv3d_tc_grad_weight.argtypes = L.lbm_nn_conv3d_grad_weight.argtypes
        L.lbm_nn_tc_error.argtypes = [C.POINTER(C.c_int)]
        L.lbm_nn_wait_selftest.argtypes = [C.c_longlong, C.POINTER(C.c_int), vp]
        for n in EXPORTS:
            getattr(L, n).restype = C.c_int
        _ready = True
    return L


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _st(stream):
    import torch
    return C.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)


def _check(s, where):
    if s != 0:
        raise LbmError(s, where)


def _name(base, tc):
    return base.replace("lbm_nn_conv3d", "lbm_nn_conv3d_tc") if tc else base


def conv3d(x, w, b, relu, y, stream=None, tc=False):
    """tc: BF16 operands on the tensor cores (lbm_nn_conv3d_tc), else FP32 CUDA cores"""
    cin, d, h, wd = x.shape
    n = _name("lbm_nn_conv3d", tc)
    _check(getattr(library(), n)(_p(x), cin, d, h, wd, _p(w), _p(b), w.shape[0], int(relu), _p(y), _st(stream)), n)


def conv3d_grad_input(gy, w, wt_scratch, gx, stream=None, tc=False):
    cout, d, h, wd = gy.shape
    n = _name("lbm_nn_conv3d_grad_input", tc)
    _check(getattr(library(), n)(_p(gy), cout, d, h, wd, _p(w), w.shape[1], _p(wt_scratch), _p(gx), _st(stream)), n)


def conv3d_grad_weight(x, gy, gw, gb, accumulate, scratch, stream=None, tc=False):
    cin, d, h, wd = x.shape
    n = _name("lbm_nn_conv3d_grad_weight", tc)
    _check(getattr(library(), n)(_p(x), cin, _p(gy), gy.shape[0], d, h, wd, _p(gw), _p(gb), int(accumulate),
                                 _p(scratch), _st(stream)), n)


def tc_error():
    """1 if a tensor-core kernel gave up waiting since the last call (clears the flag)"""
    flag = C.c_int(0)
    _check(library().lbm_nn_tc_error(C.byref(flag)), "lbm_nn_tc_error")
    return flag.value


def wait_selftest(limit_cycles, stream=None):
    """1 if a bounded wait on a barrier that nothing arrives on completed, 0 if it gave up."""
    done = C.c_int(-1)
    _check(library().lbm_nn_wait_selftest(int(limit_cycles), C.byref(done), _st(stream)), "lbm_nn_wait_selftest")
    return done.value


def axpy(y, x, a=1.0, stream=None):
    _check(library().lbm_nn_axpy(_p(y), _p(x), y.numel(), a, _st(stream)), "lbm_nn_axpy")


def relu_grad(y, g, stream=None):
    _check(library().lbm_nn_relu_grad(_p(y), _p(g), y.numel(), _st(stream)), "lbm_nn_relu_grad")


def avg_pool2(x, y, stream=None):
    c, d, h, w = x.shape
    _check(library().lbm_nn_avg_pool2(_p(x), c, d, h, w, _p(y), _st(stream)), "lbm_nn_avg_pool2")


def avg_pool2_grad(gy, gx, stream=None):
    c, d, h, w = gx.shape
    _check(library().lbm_nn_avg_pool2_grad(_p(gy), c, d, h, w, _p(gx), _st(stream)), "lbm_nn_avg_pool2_grad")


def up2(x, y, stream=None):
    c, d, h, w = x.shape
    _check(library().lbm_nn_up2(_p(x), c, d, h, w, _p(y), _st(stream)), "lbm_nn_up2")


def up2_grad(gy, gx, stream=None):
    c, d, h, w = gx.shape
    _check(library().lbm_nn_up2_grad(_p(gy), c, d, h, w, _p(gx), _st(stream)), "lbm_nn_up2_grad")


def rel_loss(p, t, grad, sums, loss=None, stream=None):
    _check(library().lbm_nn_rel_loss(_p(p), _p(t), p.numel(), _p(grad), _p(sums), _p(loss), _st(stream)),
           "lbm_nn_rel_loss")


def adam(p, g, m, v, lr, b1, b2, eps, step, stream=None):
    c1, c2 = 1.0 - b1 ** step, 1.0 - b2 ** step
    _check(library().lbm_nn_adam(_p(p), _p(g), _p(m), _p(v), p.numel(), lr, b1, b2, eps, c1, c2, _st(stream)),
           "lbm_nn_adam")
