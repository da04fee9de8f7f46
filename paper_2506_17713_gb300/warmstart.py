"""Learned warm start of steady-state runs (the project's row f3; the paper cites
learned initial fields in Section 1 but defines no network).

Workload: single-phase flow through periodic porous samples (thresholded Gaussian
random fields) under a body force, the permeability estimate of Section 3.4. A 3-D
U-Net maps the fluid indicator of a sample to its steady velocity field, scaled as
nu u / a (a "local permeability", independent of the force), and its density
deviation. A steady-state run then starts from the predicted density and velocity
instead of from rest, and relaxes to the same residual (||u^n - u^{n-100}||_2 / ||u^n||_2 <= 1e-6); the plain
run from rest is the fallback and the arbiter of the prediction.

Every operation of the network runs in the project's CUDA kernels (nn.py /
include/lbm_nn.h); torch only provides device memory.
"""
import time

import numpy as np

from . import nn
from .lbm import Batch, Lattice

ACCEL = 1e-5          # body acceleration along x (creeping flow)
TAU = 1.0             # BGK relaxation time: nu = 1/6
NU = (TAU - 0.5) / 3.0


def flow_case(n):
    """D3Q19 single-phase BGK on a periodic n^3 box, body force along x (no
    interaction: psi = rho with g = 0). FP64: in FP32 the residual stalls at a
    rounding floor (about 2e-4 at this force) above the 1e-6 criterion."""
    from synth import cases
    return cases.base_case("D3Q19", (n, n, n), collision="BGK", psi=["rho", "rho"], g=[[0.0, 0.0], [0.0, 0.0]],
                           tau=[TAU, TAU], accel=[[ACCEL, 0.0, 0.0], [0.0, 0.0, 0.0]], real="f64")


def sample_solid(n, seed, porosity):
    from synth import grf_porous_medium
    solid, _ = grf_porous_medium((n, n, n), porosity, 6.0, seed, buffer=0, periodic_x=True)
    return solid


def steady_states(n, seeds, porosities, steps, stream=None, tol=1e-6, chunk=1000):
    """Steady fields of the samples, advanced together as one batch in chunks of
    `chunk` steps until every residual (change over the last chunk) is <= tol or
    `steps` steps have run; returns (solids, [4, n, n, n] arrays of u_x, u_y, u_z,
    rho - 1, residuals). The density deviation is formed in FP64 before the FP32 cast."""
    lats, solids = [], []
    for s, phi in zip(seeds, porosities):
        solid = sample_solid(n, s, phi)
        lat = Lattice(flow_case(n), stream)
        lat.set_geometry(solid)
        lat.init_fields(0, np.ones((n, n, n)))
        lats.append(lat)
        solids.append(solid)
    batch = Batch(lats)
    for lat in lats:
        lat.diagnostics(residual=True)
    done, res = 0, [1.0] * len(lats)
    while done < steps:
        batch.step(chunk)
        done += chunk
        res = [lat.diagnostics(residual=True)[2] for lat in lats]
        if max(res) <= tol:
            break
    us = []
    for lat in lats:
        rho, u = lat.macroscopic_host(0)
        us.append(np.concatenate([u, rho[None] - 1.0]).astype(np.float32))
    batch.close()
    for lat in lats:
        lat.close()
    return solids, us, res


class UNet:
    """3-D U-Net on [C, n, n, n] fields (n divisible by 4), periodic 3x3x3 convolutions:

      e1: 2 -> c1 -> c1           (n)      skip 1   (inputs: fluid indicator, distance to solid)
      e2: pool, c1 -> c2 -> c2    (n/2)    skip 2
      b : pool, c2 -> c3 -> c3    (n/4)
      d2: up, [c3 | skip 2] -> c2 -> c2   (n/2)
      d1: up, [c2 | skip 1] -> c1 -> 4    (n), the last layer linear
          (outputs: the flow shape, 3 channels, and the density deviation (rho - 1) / (a n))

    Leaky ReLU after every convolution but the last. Parameters and Adam moments are
    FP32; the last layer starts at a tenth of its He initialisation, so the first
    predictions are small and the relative loss starts near 1. With tensor_cores (the
    default) the convolutions and their gradients run as BF16 implicit GEMMs on the
    tensor cores with FP32 accumulation; otherwise in FP32 on the CUDA cores."""
    CIN = 2
    COUT = 4

    LAYERS = [("e1a", "in", "c1"), ("e1b", "c1", "c1"), ("e2a", "c1", "c2"), ("e2b", "c2", "c2"),
              ("ba", "c2", "c3"), ("bb", "c3", "c3"), ("d2a", "c3+c2", "c2"), ("d2b", "c2", "c2"),
              ("d1a", "c2+c1", "c1"), ("d1b", "c1", "out")]

    def __init__(self, n, channels=(8, 16, 32), seed=0, tensor_cores=True):
        import torch
        assert n % 4 == 0
        self.torch = torch
        self.n = n
        self.tc = bool(tensor_cores)
        c1, c2, c3 = channels
        size = {"in": self.CIN, "out": self.COUT, "c1": c1, "c2": c2, "c3": c3, "c3+c2": c3 + c2, "c2+c1": c2 + c1}
        g = torch.Generator().manual_seed(seed)
        dev = "cuda"
        self.shape = {}
        self.w, self.b, self.gw, self.gb, self.m, self.v = {}, {}, {}, {}, {}, {}
        for name, ci, co in self.LAYERS:
            cin, cout = size[ci], size[co]
            self.shape[name] = (cin, cout)
            std = (2.0 / (cin * 27)) ** 0.5
            if name == "d1b":
                std *= 0.1
            self.w[name] = (torch.randn(cout, cin, 27, generator=g) * std).to(dev)
            self.b[name] = torch.zeros(cout, device=dev)
            for d in (self.gw, self.m, self.v):
                d[name] = torch.zeros(cout, cin, 27, device=dev)
            for d in (self.gb,):
                d[name] = torch.zeros(cout, device=dev)
            self.m[name + ".b"] = torch.zeros(cout, device=dev)
            self.v[name + ".b"] = torch.zeros(cout, device=dev)
        self.step_count = 0
        h, q = n // 2, n // 4
        e = lambda c, s: torch.empty(c, s, s, s, device=dev)
        # activations (kept for the backward pass); skips written into the concat buffers
        self.a = {"x": e(self.CIN, n), "e1a": e(c1, n), "cat1": e(c2 + c1, n), "p1": e(c1, h), "e2a": e(c2, h),
                  "cat2": e(c3 + c2, h), "p2": e(c2, q), "ba": e(c3, q), "bb": e(c3, q), "d2a": e(c2, h),
                  "d2b": e(c2, h), "d1a": e(c1, n), "out": e(self.COUT, n)}
        self.g = {k: torch.empty_like(v) for k, v in self.a.items()}
        self.g["skip1"] = e(c1, n)
        self.g["skip2"] = e(c2, h)
        maxw = max(ci * co for ci, co in self.shape.values())
        self.wt = torch.empty(maxw * 27, device=dev)
        self.gw_scratch = torch.empty(max(nn.gw_scratch_floats(ci, co, self.tc) for ci, co in self.shape.values()),
                                      device=dev)
        self.sums = torch.zeros(2, dtype=torch.float64, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.c = (c1, c2, c3)

    def parameters(self):
        return sum(self.w[k].numel() + self.b[k].numel() for k in self.w)

    def _conv(self, name, x, y, relu):
        nn.conv3d(x, self.w[name], self.b[name], relu, y, tc=self.tc)

    def forward(self, x):
        """x: [2, n, n, n] float32 input features (see features()) -> [4, n, n, n]"""
        a, (c1, c2, c3) = self.a, self.c
        a["x"].copy_(x)
        skip1 = a["cat1"][c2:]
        skip2 = a["cat2"][c3:]
        self._conv("e1a", a["x"], a["e1a"], True)
        self._conv("e1b", a["e1a"], skip1, True)
        nn.avg_pool2(skip1, a["p1"])
        self._conv("e2a", a["p1"], a["e2a"], True)
        self._conv("e2b", a["e2a"], skip2, True)
        nn.avg_pool2(skip2, a["p2"])
        self._conv("ba", a["p2"], a["ba"], True)
        self._conv("bb", a["ba"], a["bb"], True)
        nn.up2(a["bb"], a["cat2"][:c3])
        self._conv("d2a", a["cat2"], a["d2a"], True)
        self._conv("d2b", a["d2a"], a["d2b"], True)
        nn.up2(a["d2b"], a["cat1"][:c2])
        self._conv("d1a", a["cat1"], a["d1a"], True)
        self._conv("d1b", a["d1a"], a["out"], False)
        return a["out"]

    def _conv_back(self, name, x, y_post, gy, gx, relu, accumulate):
        """gy: gradient at the layer output (post-activation); gx: gradient at x (or None)"""
        if relu:
            nn.relu_grad(y_post, gy)
        cin, cout = self.shape[name]
        nn.conv3d_grad_weight(x, gy, self.gw[name], self.gb[name], accumulate, self.gw_scratch, tc=self.tc)
        if gx is not None:
            nn.conv3d_grad_input(gy, self.w[name], self.wt[: cin * cout * 27], gx, tc=self.tc)

    def backward(self, target, accumulate):
        """loss = sum (out - target)^2 / sum target^2; accumulate adds to the stored
        parameter gradients. Returns the loss as a device tensor."""
        a, g, (c1, c2, c3) = self.a, self.g, self.c
        nn.rel_loss(a["out"], target, g["out"], self.sums, self.loss)
        skip1 = a["cat1"][c2:]
        skip2 = a["cat2"][c3:]
        self._conv_back("d1b", a["d1a"], a["out"], g["out"], g["d1a"], False, accumulate)
        self._conv_back("d1a", a["cat1"], a["d1a"], g["d1a"], g["cat1"], True, accumulate)
        g["skip1"].copy_(g["cat1"][c2:])
        nn.up2_grad(g["cat1"][:c2], g["d2b"])
        self._conv_back("d2b", a["d2a"], a["d2b"], g["d2b"], g["d2a"], True, accumulate)
        self._conv_back("d2a", a["cat2"], a["d2a"], g["d2a"], g["cat2"], True, accumulate)
        g["skip2"].copy_(g["cat2"][c3:])
        nn.up2_grad(g["cat2"][:c3], g["bb"])
        self._conv_back("bb", a["ba"], a["bb"], g["bb"], g["ba"], True, accumulate)
        self._conv_back("ba", a["p2"], a["ba"], g["ba"], g["p2"], True, accumulate)
        nn.avg_pool2_grad(g["p2"], g["cat2"][c3:])
        nn.axpy(g["skip2"], g["cat2"][c3:])
        self._conv_back("e2b", a["e2a"], skip2, g["skip2"], g["e2a"], True, accumulate)
        self._conv_back("e2a", a["p1"], a["e2a"], g["e2a"], g["p1"], True, accumulate)
        nn.avg_pool2_grad(g["p1"], g["cat1"][c2:])
        nn.axpy(g["skip1"], g["cat1"][c2:])
        self._conv_back("e1b", a["e1a"], skip1, g["skip1"], g["e1a"], True, accumulate)
        self._conv_back("e1a", a["x"], a["e1a"], g["e1a"], None, True, accumulate)
        return self.loss

    def adam_step(self, lr, b1=0.9, b2=0.999, eps=1e-8):
        """one Adam step on the accumulated (summed) gradients; Adam's update does not
        depend on a common scale of the gradients, so the sum needs no averaging"""
        self.step_count += 1
        for name in self.w:
            nn.adam(self.w[name], self.gw[name], self.m[name], self.v[name], lr, b1, b2, eps, self.step_count)
            nn.adam(self.b[name], self.gb[name], self.m[name + ".b"], self.v[name + ".b"], lr, b1, b2, eps,
                    self.step_count)


def features(solid, cap=8):
    """network input [2, n, n, n]: the fluid indicator and the Euclidean distance to the
    nearest solid on the periodic box (capped at `cap`, scaled by 1/cap)"""
    from scipy.ndimage import distance_transform_edt
    fluid = (1 - solid).astype(np.float32)
    padded = np.pad(fluid, cap, mode="wrap")
    d = distance_transform_edt(padded)[cap:-cap, cap:-cap, cap:-cap]
    return np.stack([fluid, (np.minimum(d, cap) / cap).astype(np.float32)])


def scale_of(u, solid):
    """mean of nu u_x / a over the fluid nodes (the sample's velocity scale)"""
    return float((u[0] * (NU / ACCEL))[solid == 0].mean())


def targets(fields, solids):
    """network targets from steady [u_x, u_y, u_z, rho - 1] fields: the velocity nu u / a
    divided by its scale (unit mean x-velocity over the fluid), so samples of very
    different permeability weigh alike, and the density deviation (rho - 1) / (a n),
    whose size the body force sets (zero in solids)"""
    out = []
    for f, s in zip(fields, solids):
        n = s.shape[0]
        shape = f[:3] * (NU / ACCEL) / scale_of(f, s)
        drho = np.where(s == 0, f[3] / (ACCEL * n), 0.0)
        out.append(np.concatenate([shape, drho[None]]).astype(np.float32))
    return out


def ritz_scale(shape, solid):
    """Velocity scale of a predicted flow shape u_hat (zero in solids): creeping flow
    under the body force a minimises nu/2 sum |grad u|^2 - a sum u_x, so along the
    direction u_hat the minimiser is u = s u_hat with
      s = a sum u_hat_x / (nu sum |grad u_hat|^2)
    (first differences on the periodic box; links that cross the halfway wall count
    twice). Exact when the shape is exact; otherwise the best scale for that shape."""
    fluid = solid == 0
    u = shape * fluid
    num = ACCEL * float(u[0].sum())
    den = 0.0
    for ax in (1, 2, 3):
        nb = np.roll(fluid, -1, axis=ax - 1)
        d2 = (np.roll(u, -1, axis=ax) - u) ** 2
        # a link between a fluid node and a solid one ends at the halfway wall, half a
        # link away: gradient u / (1/2) over length 1/2, twice the first-difference term
        both = fluid & nb
        cross = fluid ^ nb
        den += float(d2[:, both].sum()) + 2.0 * float(d2[:, cross].sum())
    return num / (NU * den) if den > 0 else 0.0


def train(net, solids, us, epochs, batch=8, lr=1e-3, seed=0, log=None):
    import torch
    rng = np.random.default_rng(seed)
    xs = [torch.from_numpy(features(s)).cuda() for s in solids]
    ts = [torch.from_numpy(t).cuda() for t in targets(us, solids)]
    history = []
    for ep in range(epochs):
        order = rng.permutation(len(xs))
        tot = 0.0
        for b0 in range(0, len(order), batch):
            idx = order[b0:b0 + batch]
            for j, i in enumerate(idx):
                net.forward(xs[i])
                tot += float(net.backward(ts[i], accumulate=j > 0).item())
            net.adam_step(lr)
        history.append(tot / len(xs))
        if log:
            log("epoch %d loss %.4f" % (ep, history[-1]))
    return history


def _net_out(net, solid):
    import torch
    x = torch.from_numpy(features(solid)).cuda()
    return net.forward(x).detach().cpu().numpy().astype(np.float64)


def scale_inputs(solid, shape):
    """regressors of log(velocity scale): 1, log porosity, log mean squared distance to
    solid over the fluid, and log of the Ritz scale of the predicted shape"""
    fl = solid == 0
    d = features(solid)[1] * 8.0
    r = ritz_scale(shape, solid) * (NU / ACCEL)
    return np.array([1.0, np.log(fl.mean()), np.log(np.mean(d[fl] ** 2)), np.log(max(r, 1e-12))])


def fit_scale(net, solids, fields):
    """least-squares fit of log(scale) on scale_inputs over converged training fields"""
    X = np.array([scale_inputs(s, _net_out(net, s)[:3]) for s in solids])
    y = np.log([scale_of(f, s) for f, s in zip(fields, solids)])
    coef, *_ = np.linalg.lstsq(X, y, rcond=None)
    return coef


def predict(net, solid, coef=None):
    """predicted steady (velocity [3, n, n, n], density [n, n, n]): the network's flow
    shape at the fitted scale (coef from fit_scale) or else at its Ritz scale, and its
    density deviation"""
    out = _net_out(net, solid)
    shape = out[:3]
    rho = 1.0 + out[3] * ACCEL * solid.shape[0]
    if coef is None:
        return shape * ritz_scale(shape, solid), rho
    scale = float(np.exp(scale_inputs(solid, shape) @ coef)) * (ACCEL / NU)
    return shape * scale, rho


def relax(n, solid, u0, check=100, max_steps=60000, tol=1e-6, rho0=None):
    """steps (multiple of `check`) and wall seconds until the residual is <= tol, from
    density rho0 (None: 1) and velocity u0 (None: rest); the permeability
    nu <u_x> / a, the last residual and the final velocity and density"""
    import torch
    lat = Lattice(flow_case(n))
    lat.set_geometry(solid)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rho = np.ones((n, n, n)) if rho0 is None else np.where(solid == 0, rho0, 1.0).astype(np.float64)
    ub = None
    if u0 is not None:
        # u0 is the reported velocity (sum f e + F/2) / rho; the populations are set at
        # equilibrium with the bare velocity, half a body-force step lower (Eq. edm)
        ub = u0.astype(np.float64).copy()
        ub[0] -= 0.5 * ACCEL * (solid == 0)
    lat.init_fields(0, rho, ub)
    lat.diagnostics(residual=True)
    steps = 0
    while steps < max_steps:
        lat.step(check)
        steps += check
        _, _, r = lat.diagnostics(residual=True)
        if r <= tol:
            break
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    rho_f, u = lat.macroscopic_host(0)
    k = NU * float(u[0].astype(np.float64).mean()) / ACCEL
    lat.close()
    return steps, dt, k, r, u, rho_f


def relax_scaled_early_field(n, solid, m, q_inf, check=100, max_steps=60000, tol=1e-6):
    """Steps until the residual is <= tol when the run from rest is stopped after m steps and
    its departure from rest is scaled by s = q_inf / q(m), q being the mean x-velocity over
    the fluid: f <- w + s (f - w) at fluid nodes. In creeping flow the step is linear in that
    departure, so this completes the magnitude of the slowest flow mode. Returns (total steps
    including the m, s)."""
    import torch
    lat = Lattice(flow_case(n))
    lat.set_geometry(solid)
    lat.init_fields(0, np.ones((n, n, n)))
    lat.step(m)
    fl = solid == 0
    _, u = lat.macroscopic_host(0)
    s = q_inf / float(u[0].astype(np.float64)[fl].mean())
    f = lat.populations(0)
    _, w = lat.velocity_set()
    w = torch.tensor(np.asarray(w), dtype=f.dtype, device=f.device).view(-1, 1, 1, 1)
    mask = torch.from_numpy(fl).to(device=f.device, dtype=f.dtype)
    lat.set_populations(0, (w + s * (f - w)) * mask)
    lat.diagnostics(residual=True)
    steps = 0
    while steps < max_steps:
        lat.step(check)
        steps += check
        if lat.diagnostics(residual=True)[2] <= tol:
            break
    lat.close()
    return m + steps, s
