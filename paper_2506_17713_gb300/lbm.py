"""ctypes binding of the C ABI in include/lbm.h.

Argument marshalling only: every step of the lattice update runs in the CUDA
kernels of liblbm.so. PyTorch provides the device workspace (the library never
allocates) and the stream. There is no CPU fallback: if the library or a GPU is
missing the calls raise.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_OK = 0
STATUS = {0: "LBM_OK", 1: "LBM_ERR_INVALID_ARG", 2: "LBM_ERR_WORKSPACE", 3: "LBM_ERR_CUDA",
          4: "LBM_ERR_UNSTABLE", 5: "LBM_ERR_TIMEOUT", 6: "LBM_ERR_STATE"}
LBM_D2Q9, LBM_D3Q19 = 0, 1
LBM_FP32, LBM_FP64, LBM_FP16S, LBM_BF16S = 0, 1, 2, 3
LBM_BGK, LBM_MRT = 0, 1
LBM_UEQ_COMPONENT, LBM_UEQ_COMMON = 0, 1
PSI = {"eos": 0, "rho": 1, "exp": 2}
EOS = {"CS": 0, "PR": 1, "VdW": 2, "RK": 3, "RKS": 4}
BC = {"periodic": 0, "wall": 1, "pressure": 2}
LBM_HOST, LBM_DEVICE = 0, 1

# every entry point declared in include/lbm.h
EXPORTS = ["lbm_workspace_size", "lbm_create", "lbm_set_geometry", "lbm_init_fields", "lbm_step",
           "lbm_macroscopic", "lbm_diagnostics", "lbm_get_populations", "lbm_set_populations",
           "lbm_velocity_set", "lbm_sync", "lbm_kernel_launches", "lbm_temperature", "lbm_destroy",
           "lbm_status_str", "lbm_profile_step", "lbm_stream_probe", "lbm_mass_noalloc", "lbm_batch_workspace_size",
           "lbm_batch_create", "lbm_batch_autotune", "lbm_batch_step", "lbm_batch_launches",
           "lbm_batch_destroy"]


class LbmError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s" % (where, STATUS.get(status, str(status))))


class lbm_params(C.Structure):
    _fields_ = [
        ("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("ncomp", C.c_int), ("real", C.c_int), ("collision", C.c_int), ("velocity", C.c_int),
        ("tau", C.c_double * 2), ("mrt_s", (C.c_double * 19) * 2),
        ("psi_kind", C.c_int * 2), ("eos", C.c_int * 2),
        ("eos_a", C.c_double * 2), ("eos_b", C.c_double * 2), ("eos_R", C.c_double * 2),
        ("eos_omega", C.c_double * 2), ("T_red", C.c_double * 2),
        ("alpha", C.c_double * 2), ("A", C.c_double * 2), ("g", (C.c_double * 2) * 2),
        ("wet_phi", C.c_double * 2), ("wet_drho", C.c_double * 2),
        ("rho_min", C.c_double * 2), ("rho_max", C.c_double * 2),
        ("body_accel", (C.c_double * 3) * 2),
        ("bc", C.c_int * 6), ("bc_rho", (C.c_double * 2) * 6),
        ("schedule", C.c_int),
        ("rho_ref", C.c_double * 2),
        ("kappa", C.c_double * 2),
        ("forcing", C.c_int),
    ]


_lib = None


def library():
    """Load liblbm.so (built by __graft_entry__.build() / paper_2506_17713_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("liblbm.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, dp, ip, sz = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_size_t
    pp = C.POINTER(lbm_params)
    L.lbm_workspace_size.argtypes = [pp, C.POINTER(sz)]
    L.lbm_create.argtypes = [pp, vp, sz, vp, C.POINTER(vp)]
    L.lbm_set_geometry.argtypes = [vp, vp, C.c_int]
    L.lbm_init_fields.argtypes = [vp, C.c_int, vp, vp, C.c_int]
    L.lbm_step.argtypes = [vp, C.c_int]
    L.lbm_macroscopic.argtypes = [vp, C.c_int, vp, vp, C.c_int]
    L.lbm_diagnostics.argtypes = [vp, dp, dp, dp]
    L.lbm_get_populations.argtypes = [vp, C.c_int, vp, C.c_int]
    L.lbm_set_populations.argtypes = [vp, C.c_int, vp, C.c_int]
    L.lbm_velocity_set.argtypes = [vp, ip, ip, dp]
    L.lbm_sync.argtypes = [vp]
    L.lbm_kernel_launches.argtypes = [vp]
    L.lbm_kernel_launches.restype = C.c_longlong
    L.lbm_temperature.argtypes = [vp, C.c_int, dp]
    L.lbm_profile_step.argtypes = [vp, C.c_int, dp, C.POINTER(C.c_longlong)]
    L.lbm_stream_probe.argtypes = [vp, C.c_int, dp]
    L.lbm_mass_noalloc.argtypes = [pp, vp, dp, vp]
    L.lbm_batch_workspace_size.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(sz)]
    L.lbm_batch_create.argtypes = [C.POINTER(vp), C.c_int, vp, sz, vp, C.POINTER(vp)]
    L.lbm_batch_autotune.argtypes = [vp, ip]
    L.lbm_batch_step.argtypes = [vp, C.c_int]
    L.lbm_batch_launches.argtypes = [vp]
    L.lbm_batch_launches.restype = C.c_longlong
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_status_str.argtypes = [C.c_int]
    L.lbm_status_str.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("lbm_kernel_launches", "lbm_destroy", "lbm_status_str", "lbm_batch_launches",
                        "lbm_batch_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(status, where):
    if status != LBM_OK:
        raise LbmError(status, where)


# ---------------------------------------------------------------------------
# Entry points, same names as the C ABI (marshalling only)
# ---------------------------------------------------------------------------

def lbm_workspace_size(params):
    n = C.c_size_t(0)
    _check(library().lbm_workspace_size(C.byref(params), C.byref(n)), "lbm_workspace_size")
    return n.value


def lbm_create(params, d_workspace, nbytes, stream):
    ctx = C.c_void_p()
    _check(library().lbm_create(C.byref(params), C.c_void_p(d_workspace), nbytes, C.c_void_p(stream),
                                C.byref(ctx)), "lbm_create")
    return ctx


def lbm_set_geometry(ctx, solid_ptr, where):
    _check(library().lbm_set_geometry(ctx, C.c_void_p(solid_ptr), where), "lbm_set_geometry")


def lbm_init_fields(ctx, comp, rho_ptr, u_ptr, where):
    _check(library().lbm_init_fields(ctx, comp, C.c_void_p(rho_ptr), C.c_void_p(u_ptr), where),
           "lbm_init_fields")


def lbm_step(ctx, nsteps):
    _check(library().lbm_step(ctx, int(nsteps)), "lbm_step")


def lbm_macroscopic(ctx, comp, rho_ptr, u_ptr, where):
    _check(library().lbm_macroscopic(ctx, comp, C.c_void_p(rho_ptr), C.c_void_p(u_ptr), where),
           "lbm_macroscopic")


def lbm_diagnostics(ctx, ncomp, residual=False):
    mass = (C.c_double * 2)()
    mom = (C.c_double * 6)()
    res = C.c_double(0.0)
    _check(library().lbm_diagnostics(ctx, mass, mom, C.byref(res) if residual else None),
           "lbm_diagnostics")
    m = np.array(mass[:ncomp])
    p = np.array(mom[: 3 * ncomp]).reshape(ncomp, 3)
    return (m, p, res.value) if residual else (m, p)


def lbm_get_populations(ctx, comp, f_ptr, where):
    _check(library().lbm_get_populations(ctx, comp, C.c_void_p(f_ptr), where), "lbm_get_populations")


def lbm_set_populations(ctx, comp, f_ptr, where):
    _check(library().lbm_set_populations(ctx, comp, C.c_void_p(f_ptr), where), "lbm_set_populations")


def lbm_velocity_set(ctx):
    q = C.c_int(0)
    e = (C.c_int * 57)()
    w = (C.c_double * 19)()
    _check(library().lbm_velocity_set(ctx, C.byref(q), e, w), "lbm_velocity_set")
    Q = q.value
    return np.array(e[: 3 * Q]).reshape(Q, 3), np.array(w[:Q])


def lbm_sync(ctx):
    _check(library().lbm_sync(ctx), "lbm_sync")


def lbm_kernel_launches(ctx):
    return int(library().lbm_kernel_launches(ctx))


def lbm_temperature(ctx, comp):
    T = C.c_double(0.0)
    _check(library().lbm_temperature(ctx, comp, C.byref(T)), "lbm_temperature")
    return T.value


def lbm_stream_probe(ctx, nsteps):
    """summed milliseconds of nsteps free-streaming launches (replaces the lattice state)"""
    ms = C.c_double(0.0)
    _check(library().lbm_stream_probe(ctx, int(nsteps), C.byref(ms)), "lbm_stream_probe")
    return ms.value


def lbm_profile_step(ctx, nsteps):
    """(milliseconds, launches) per kernel kind: density, virtual density, collide."""
    ms = (C.c_double * 3)()
    n = (C.c_longlong * 3)()
    _check(library().lbm_profile_step(ctx, int(nsteps), ms, n), "lbm_profile_step")
    return list(ms), list(n)


def lbm_mass_noalloc(params, d_f, stream):
    """Mass per component of device populations [K][Q][N], without any allocation."""
    mass = (C.c_double * 2)()
    _check(library().lbm_mass_noalloc(C.byref(params), C.c_void_p(d_f), mass, C.c_void_p(stream)),
           "lbm_mass_noalloc")
    return np.array(mass[: params.ncomp])


def lbm_destroy(ctx):
    library().lbm_destroy(ctx)


def lbm_status_str(status):
    return library().lbm_status_str(status).decode()


# ---------------------------------------------------------------------------
# Problem description -> lbm_params
# ---------------------------------------------------------------------------

def _two(v, default):
    if v is None:
        v = default
    if np.isscalar(v):
        return [float(v)] * 2
    v = [float(x) for x in v]
    return (v + [v[-1]] * 2)[:2]


def params_from_case(case):
    """Translate a problem description (dict of parameter values) to lbm_params."""
    p = lbm_params()
    p.lattice = LBM_D2Q9 if case["lattice"] == "D2Q9" else LBM_D3Q19
    p.nx, p.ny, p.nz = [int(v) for v in case["shape"]]
    p.ncomp = int(case.get("ncomp", 1))
    p.real = {"f32": LBM_FP32, "f64": LBM_FP64, "f16s": LBM_FP16S, "bf16s": LBM_BF16S}[case.get("real", "f32")]
    rr = case.get("rho_ref", [1.0, 1.0])
    kap = case.get("kappa", [0.0, 0.0])
    for k in range(2):
        p.rho_ref[k] = float(rr[k] if k < len(rr) else rr[0])
        p.kappa[k] = float(kap[k] if k < len(kap) else kap[0])
    p.forcing = {"edm": 0, "moment": 1}[case.get("forcing", "edm")]
    p.collision = LBM_MRT if case.get("collision", "BGK") == "MRT" else LBM_BGK
    p.velocity = LBM_UEQ_COMMON if case.get("velocity", "component") == "common" else LBM_UEQ_COMPONENT
    p.tau[:] = _two(case.get("tau"), 1.0)
    rates = case.get("mrt_rates") or [[1.0] * 19]
    for k in range(2):
        r = list(rates[min(k, len(rates) - 1)]) + [1.0] * 19
        for m in range(19):
            p.mrt_s[k][m] = float(r[m])
    psi = list(case.get("psi", ["eos"]))
    eos = list(case.get("eos", ["CS"]))
    for k in range(2):
        p.psi_kind[k] = PSI[psi[min(k, len(psi) - 1)]]
        p.eos[k] = EOS[eos[min(k, len(eos) - 1)]]
    p.eos_a[:] = _two(case.get("eos_a"), 1.0)
    p.eos_b[:] = _two(case.get("eos_b"), 4.0)
    p.eos_R[:] = _two(case.get("eos_R"), 1.0)
    p.eos_omega[:] = _two(case.get("eos_omega"), 0.0)
    p.T_red[:] = _two(case.get("T_red"), 0.7)
    p.alpha[:] = _two(case.get("alpha"), 1.0)
    p.A[:] = _two(case.get("A"), 0.0)
    g = np.asarray(case.get("g", [[-1.0, 0.0], [0.0, -1.0]]), dtype=float).reshape(2, 2)
    for a in range(2):
        for b in range(2):
            p.g[a][b] = float(g[a, b])
    p.wet_phi[:] = _two(case.get("wet_phi"), 1.0)
    p.wet_drho[:] = _two(case.get("wet_drho"), 0.0)
    p.rho_min[:] = _two(case.get("rho_lo"), 0.0)
    p.rho_max[:] = _two(case.get("rho_hi"), 1e30)
    acc = np.zeros((2, 3))
    if case.get("accel") is not None:
        a = np.asarray(case["accel"], dtype=float).reshape(-1, 3)
        acc[: a.shape[0]] = a[:2]
        if a.shape[0] == 1:
            acc[1] = a[0]
    for k in range(2):
        for d in range(3):
            p.body_accel[k][d] = float(acc[k, d])
    bc = case.get("bc", ["periodic"] * 6)
    for f in range(6):
        p.bc[f] = BC[bc[f]]
    br = np.zeros((6, 2))
    if case.get("bc_rho") is not None:
        b = np.asarray(case["bc_rho"], dtype=float).reshape(6, -1)
        br[:, : b.shape[1]] = b[:, :2]
    for f in range(6):
        for k in range(2):
            p.bc_rho[f][k] = float(br[f, k])
    p.schedule = {"auto": 0, "two_pass": 1, "single_pass": 2, "slab_overlap": 3}[case.get("schedule", "auto")]
    return p


# ---------------------------------------------------------------------------
# Convenience object: a lattice on the current CUDA device
# ---------------------------------------------------------------------------

class Lattice:
    """One lattice on the current CUDA device. Field arrays are torch tensors on
    the device (or host numpy arrays where noted), shaped (nz, ny, nx)."""

    def __init__(self, case, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the CUDA lattice Boltzmann path needs a CUDA device")
        self.torch = torch
        self.case = case
        self.params = params_from_case(case)
        self.K = self.params.ncomp
        nx, ny, nz = case["shape"]
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.D = 2 if self.params.lattice == LBM_D2Q9 else 3
        self.Q = 9 if self.D == 2 else 19
        self.dtype = torch.float64 if self.params.real == LBM_FP64 else torch.float32
        self.nbytes = lbm_workspace_size(self.params)
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = lbm_create(self.params, self.workspace.data_ptr(), self.nbytes,
                              self.stream.cuda_stream)

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()

    # set-up ------------------------------------------------------------------
    def set_geometry(self, solid):
        s = np.ascontiguousarray(np.asarray(solid, dtype=np.uint8).reshape(self.shape))
        lbm_set_geometry(self.ctx, s.ctypes.data, LBM_HOST)

    def init_fields(self, comp, rho, u=None):
        r = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(self.shape))
        up = 0
        if u is not None:
            uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape((self.D,) + self.shape))
            up = uu.ctypes.data
        lbm_init_fields(self.ctx, comp, r.ctypes.data, up or None, LBM_HOST)

    def init_fields_device(self, comp, rho, u=None):
        r = rho.to(dtype=self.torch.float64).contiguous()
        uu = None if u is None else u.to(dtype=self.torch.float64).contiguous()
        lbm_init_fields(self.ctx, comp, r.data_ptr(), None if uu is None else uu.data_ptr(), LBM_DEVICE)
        return r, uu

    # stepping and outputs ----------------------------------------------------
    def step(self, n=1):
        lbm_step(self.ctx, n)

    def macroscopic(self, comp=0):
        """(rho, u) device tensors; comp = -1 for the mixture."""
        t = self.torch
        rho = t.empty(self.shape, dtype=self.dtype, device="cuda")
        u = t.empty((self.D,) + self.shape, dtype=self.dtype, device="cuda")
        lbm_macroscopic(self.ctx, comp, rho.data_ptr(), u.data_ptr(), LBM_DEVICE)
        return rho, u

    def macroscopic_host(self, comp=0):
        npdt = np.float64 if self.params.real == LBM_FP64 else np.float32
        rho = np.empty(self.shape, dtype=npdt)
        u = np.empty((self.D,) + self.shape, dtype=npdt)
        lbm_macroscopic(self.ctx, comp, rho.ctypes.data, u.ctypes.data, LBM_HOST)
        return rho, u

    def diagnostics(self, residual=False):
        return lbm_diagnostics(self.ctx, self.K, residual)

    def populations(self, comp=0):
        f = self.torch.empty((self.Q,) + self.shape, dtype=self.dtype, device="cuda")
        lbm_get_populations(self.ctx, comp, f.data_ptr(), LBM_DEVICE)
        return f

    def set_populations(self, comp, f):
        ff = f.to(dtype=self.dtype, device="cuda").contiguous()
        lbm_set_populations(self.ctx, comp, ff.data_ptr(), LBM_DEVICE)

    def velocity_set(self):
        return lbm_velocity_set(self.ctx)

    def sync(self):
        lbm_sync(self.ctx)

    def launches(self):
        return lbm_kernel_launches(self.ctx)

    def profile_step(self, n):
        return lbm_profile_step(self.ctx, n)

    def stream_probe(self, n):
        return lbm_stream_probe(self.ctx, n)

    def temperature(self, comp=0):
        return lbm_temperature(self.ctx, comp)


# ---------------------------------------------------------------------------
# Batches of lattices (one persistent launch per pass for all of them)
# ---------------------------------------------------------------------------

def lbm_batch_workspace_size(ctxs):
    arr = (C.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    n = C.c_size_t(0)
    _check(library().lbm_batch_workspace_size(arr, len(ctxs), C.byref(n)), "lbm_batch_workspace_size")
    return n.value


def lbm_batch_create(ctxs, d_workspace, nbytes, stream):
    arr = (C.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    b = C.c_void_p()
    _check(library().lbm_batch_create(arr, len(ctxs), C.c_void_p(d_workspace), nbytes, C.c_void_p(stream),
                                      C.byref(b)), "lbm_batch_create")
    return b


def lbm_batch_autotune(batch):
    cfg = (C.c_int * 6)()
    _check(library().lbm_batch_autotune(batch, cfg), "lbm_batch_autotune")
    return [(cfg[2 * i], cfg[2 * i + 1]) for i in range(3)]


def lbm_batch_step(batch, nsteps):
    _check(library().lbm_batch_step(batch, nsteps), "lbm_batch_step")


def lbm_batch_launches(batch):
    return library().lbm_batch_launches(batch)


def lbm_batch_destroy(batch):
    library().lbm_batch_destroy(batch)


class Batch:
    """Lattices advanced together: one persistent launch per pass for all of them,
    two time steps per CUDA graph replay. The lattices must outlive the batch."""

    def __init__(self, lattices, stream=None):
        import torch
        self.lattices = list(lattices)
        ctxs = [lat.ctx for lat in self.lattices]
        self.nbytes = lbm_batch_workspace_size(ctxs)
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else self.lattices[0].stream
        self.batch = lbm_batch_create(ctxs, self.workspace.data_ptr(), self.nbytes, self.stream.cuda_stream)

    def autotune(self):
        """[(CTA size, grid)] chosen for the density, virtual-density and collide passes."""
        return lbm_batch_autotune(self.batch)

    def step(self, n=1):
        lbm_batch_step(self.batch, n)

    def launches(self):
        return lbm_batch_launches(self.batch)

    def close(self):
        if getattr(self, "batch", None):
            lbm_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        self.close()
