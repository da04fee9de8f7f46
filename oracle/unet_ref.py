"""Plain numpy definitions of the operations of the warm-start network (the
learned initial field of a steady-state run, the project's row f3; the paper
cites the idea in Section 1). Test infrastructure: only tests import this module.

Fields are channel-major arrays [C, D, H, W] on a periodic box (the lattices are
periodic), so a 3x3x3 convolution wraps around instead of padding with zeros:

  conv(x, w, b)[o, z, y, x] = b[o] + sum_{i, dz, dy, dx} w[o, i, dz+1, dy+1, dx+1]
                                     x[i, (z+dz) mod D, (y+dy) mod H, (x+dx) mod W]

avg_pool2 averages 2x2x2 blocks; up2 repeats each voxel into a 2x2x2 block; relu is
the leaky ReLU (slope 0.01 below zero); the loss is the relative squared error
sum (p - t)^2 / sum t^2. bf16 rounds FP32 values to bfloat16 (8 significant bits, the
FP32 exponent range), to nearest with ties to even: the operand rounding of the
tensor-core convolutions.
"""
import numpy as np

OFFS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shift(x, dz, dy, dx):
    """x[(z+dz), (y+dy), (x+dx)] on the periodic box (last three axes)"""
    return np.roll(x, (-dz, -dy, -dx), axis=(-3, -2, -1))


def bf16(a):
    """a (any float array, taken as FP32) rounded to the nearest bfloat16, ties to even,
    returned as float64. Finite values only."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    keep = u >> 16                      # sign, exponent and the 7 stored fraction bits
    rest = u & 0xFFFF                   # the 16 dropped bits
    up = (rest > 0x8000) | ((rest == 0x8000) & (keep & 1 == 1))
    out = ((keep + up) << 16).astype(np.uint32)
    return out.view(np.float32).astype(np.float64).reshape(f.shape)


def conv3d(x, w, b):
    out = np.zeros((w.shape[0],) + x.shape[1:])
    for o in range(w.shape[0]):
        acc = np.full(x.shape[1:], float(b[o]))
        for (dz, dy, dx) in OFFS:
            for i in range(x.shape[0]):
                acc += w[o, i, dz + 1, dy + 1, dx + 1] * shift(x[i], dz, dy, dx)
        out[o] = acc
    return out


def conv3d_grads(x, w, gout):
    """(d/dx, d/dw, d/db) of sum(gout * conv3d(x, w, b))"""
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for o in range(w.shape[0]):
        for (dz, dy, dx) in OFFS:
            for i in range(x.shape[0]):
                gw[o, i, dz + 1, dy + 1, dx + 1] = np.sum(gout[o] * shift(x[i], dz, dy, dx))
                gx[i] += w[o, i, dz + 1, dy + 1, dx + 1] * shift(gout[o], -dz, -dy, -dx)
    gb = gout.reshape(gout.shape[0], -1).sum(axis=1)
    return gx, gw, gb


LEAK = 0.01


def relu(x):
    """leaky ReLU: x for x > 0, 0.01 x otherwise"""
    return np.where(x > 0, x, LEAK * x)


def relu_grad(y, g):
    """gradient through the leaky ReLU, from its output y"""
    return np.where(y > 0, g, LEAK * g)


def avg_pool2(x):
    C, D, H, W = x.shape
    return x.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(2, 4, 6))


def up2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


def rel_loss(p, t):
    d = p - t
    s = np.sum(t * t)
    return np.sum(d * d) / s, 2.0 * d / s
