"""FP64 CPU oracle of the Shan-Chen multiphase lattice Boltzmann step.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package. The CUDA product path
(``paper_2506_17713_gb300``) never imports it, and the two share no code: the
only thing both sides consume is a plain problem description (a dict of
parameter values, see ``synth.cases``) and the seeded input arrays.

The arithmetic lives in ``lbm_oracle.c`` (double precision, written step by
step after Section 2 of arXiv 2506.17713); this module is ctypes marshalling.
"""
import ctypes as C

import numpy as np

from .build import build_oracle

_LIB = None

BGK, MRT = 0, 1
PSI = {"eos": 0, "rho": 1, "exp": 2}
EOS = {"CS": 0, "PR": 1, "VdW": 2, "RK": 3, "RKS": 4}
BC = {"periodic": 0, "wall": 1, "pressure": 2}


class OrcParams(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("ncomp", C.c_int), ("collision", C.c_int), ("common_velocity", C.c_int),
        ("tau", C.c_double * 2), ("mrt_rates", (C.c_double * 19) * 2),
        ("psi_kind", C.c_int * 2), ("eos", C.c_int * 2),
        ("eos_a", C.c_double * 2), ("eos_b", C.c_double * 2), ("eos_R", C.c_double * 2),
        ("eos_omega", C.c_double * 2), ("T_red", C.c_double * 2),
        ("alpha", C.c_double * 2), ("A", C.c_double * 2), ("g", (C.c_double * 2) * 2),
        ("wet_phi", C.c_double * 2), ("wet_drho", C.c_double * 2),
        ("rho_lo", C.c_double * 2), ("rho_hi", C.c_double * 2),
        ("accel", (C.c_double * 3) * 2),
        ("face_bc", C.c_int * 6), ("face_rho", (C.c_double * 2) * 6),
        ("kappa", C.c_double * 2),
        ("forcing", C.c_int),
    ]


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _LIB
    if _LIB is None:
        L = C.CDLL(build_oracle())
        vp, dp, ip, up = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p
        L.orc_create.restype = vp
        L.orc_create.argtypes = [C.POINTER(OrcParams)]
        L.orc_destroy.argtypes = [vp]
        L.orc_Q.argtypes = [vp]
        L.orc_steps.restype = C.c_long
        L.orc_steps.argtypes = [vp]
        L.orc_velocity_set.argtypes = [vp, ip, dp]
        L.orc_mrt_matrices.argtypes = [vp, dp, dp]
        L.orc_set_geometry.argtypes = [vp, up]
        L.orc_init_fields.argtypes = [vp, C.c_int, dp, dp]
        L.orc_set_populations.argtypes = [vp, C.c_int, dp]
        L.orc_get_populations.argtypes = [vp, C.c_int, dp]
        L.orc_step.argtypes = [vp, C.c_int]
        L.orc_macroscopic.argtypes = [vp, C.c_int, dp, dp]
        L.orc_force.argtypes = [vp, C.c_int, dp]
        L.orc_psi.argtypes = [vp, C.c_int, dp, dp]
        L.orc_diagnostics.argtypes = [vp, dp, dp]
        L.orc_boundary_solids.argtypes = [vp, up]
        L.orc_interaction_force.argtypes = [vp, dp, dp, dp, C.c_int, dp]
        L.orc_surface_Q.argtypes = [vp, dp, C.c_long, C.c_int, dp]
        L.orc_collide_single.argtypes = [vp, C.c_int, dp, dp, dp]
        L.orc_eos_Tc.restype = C.c_double
        L.orc_eos_Tc.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
        L.orc_eos_pressure.restype = C.c_double
        L.orc_eos_pressure.argtypes = [C.c_int] + [C.c_double] * 6
        L.orc_bulk_pressure.restype = C.c_double
        L.orc_bulk_pressure.argtypes = [C.POINTER(OrcParams), C.c_int, C.c_double]
        L.orc_maxwell_eos.argtypes = [C.c_int] + [C.c_double] * 5 + [dp, dp, dp]
        L.orc_maxwell_bulk.argtypes = [C.POINTER(OrcParams), C.c_int, C.c_double, C.c_double,
                                       dp, dp, dp]
        L.orc_threads.restype = C.c_int
        _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _pair(v, K, default):
    if v is None:
        v = default
    if np.isscalar(v):
        return [float(v)] * 2
    v = list(v) + [v[-1]] * (2 - len(v))
    return [float(x) for x in v[:2]]


def params_from_case(case):
    """Map a problem description (plain dict, see synth.cases) to OrcParams."""
    p = OrcParams()
    nx, ny, nz = case["shape"]
    p.dim = 2 if case["lattice"] == "D2Q9" else 3
    p.nx, p.ny, p.nz = nx, ny, nz
    K = int(case.get("ncomp", 1))
    p.ncomp = K
    p.collision = MRT if case.get("collision", "BGK") == "MRT" else BGK
    p.common_velocity = 1 if case.get("velocity", "component") == "common" else 0
    p.tau[:] = _pair(case.get("tau"), K, 1.0)
    rates = case.get("mrt_rates")
    for k in range(2):
        rk = rates[min(k, len(rates) - 1)] if rates is not None else [1.0] * 19
        for a in range(19):
            p.mrt_rates[k][a] = float(rk[a]) if a < len(rk) else 1.0
    psi = case.get("psi", ["eos"])
    eos = case.get("eos", ["CS"])
    for k in range(2):
        p.psi_kind[k] = PSI[psi[min(k, len(psi) - 1)]]
        p.eos[k] = EOS[eos[min(k, len(eos) - 1)]]
    p.eos_a[:] = _pair(case.get("eos_a"), K, 1.0)
    p.eos_b[:] = _pair(case.get("eos_b"), K, 4.0)
    p.eos_R[:] = _pair(case.get("eos_R"), K, 1.0)
    p.eos_omega[:] = _pair(case.get("eos_omega"), K, 0.0)
    p.T_red[:] = _pair(case.get("T_red"), K, 0.7)
    p.alpha[:] = _pair(case.get("alpha"), K, 1.0)
    p.A[:] = _pair(case.get("A"), K, 0.0)
    g = np.array(case.get("g", [[-1.0, 0.0], [0.0, -1.0]]), dtype=float).reshape(-1)
    g = np.resize(g, 4) if g.size < 4 else g
    for a in range(2):
        for b in range(2):
            p.g[a][b] = float(g[2 * a + b])
    p.wet_phi[:] = _pair(case.get("wet_phi"), K, 1.0)
    p.wet_drho[:] = _pair(case.get("wet_drho"), K, 0.0)
    p.rho_lo[:] = _pair(case.get("rho_lo"), K, 0.0)
    p.rho_hi[:] = _pair(case.get("rho_hi"), K, 1e30)
    acc = np.zeros((2, 3))
    if case.get("accel") is not None:
        a = np.array(case["accel"], dtype=float).reshape(-1, 3)
        acc[: a.shape[0]] = a
        if a.shape[0] == 1:
            acc[1] = a[0]
    for k in range(2):
        for d in range(3):
            p.accel[k][d] = acc[k, d]
    bc = case.get("bc", ["periodic"] * 6)
    for f in range(6):
        p.face_bc[f] = BC[bc[f]]
    br = np.zeros((6, 2))
    if case.get("bc_rho") is not None:
        b = np.array(case["bc_rho"], dtype=float).reshape(6, -1)
        br[:, : b.shape[1]] = b
    for f in range(6):
        for k in range(2):
            p.face_rho[f][k] = br[f, k]
    p.forcing = {"edm": 0, "moment": 1}[case.get("forcing", "edm")]
    kap = case.get("kappa", [0.0, 0.0])
    for k in range(2):
        p.kappa[k] = float(kap[k] if k < len(kap) else kap[0])
    return p


class OracleSim:
    """One oracle lattice. Arrays crossing this interface are float64, node-major
    in x-fastest order: scalar fields (nz, ny, nx), vector fields (dim, nz, ny, nx),
    populations (Q, nz, ny, nx) in the oracle's own velocity order (see ``e``)."""

    def __init__(self, case):
        self.case = case
        self.params = params_from_case(case)
        self.h = lib().orc_create(C.byref(self.params))
        if not self.h:
            raise ValueError("oracle rejected the problem description")
        nx, ny, nz = case["shape"]
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.dim = self.params.dim
        self.K = self.params.ncomp
        self.Q = lib().orc_Q(self.h)
        e = np.zeros(3 * self.Q, dtype=np.int32)
        w = np.zeros(self.Q)
        lib().orc_velocity_set(self.h, e.ctypes.data_as(C.POINTER(C.c_int)), _dp(w))
        self.e = e.reshape(self.Q, 3)
        self.w = w
        self.solid = np.zeros(self.shape, dtype=np.uint8)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_destroy(h)
            self.h = None

    # set-up -----------------------------------------------------------------
    def set_geometry(self, solid):
        s = np.ascontiguousarray(np.asarray(solid, dtype=np.uint8).reshape(self.shape))
        self.solid = s
        lib().orc_set_geometry(self.h, s.ctypes.data)

    def init_fields(self, k, rho, u=None):
        r = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(self.shape))
        up = None
        if u is not None:
            uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape((self.dim,) + self.shape))
            up = _dp(uu)
        lib().orc_init_fields(self.h, k, _dp(r), up)

    def set_populations(self, k, f):
        a = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape((self.Q,) + self.shape))
        lib().orc_set_populations(self.h, k, _dp(a))

    # stepping and outputs -----------------------------------------------------
    def step(self, n=1):
        lib().orc_step(self.h, int(n))

    @property
    def steps(self):
        return lib().orc_steps(self.h)

    def populations(self, k=0):
        out = np.zeros((self.Q,) + self.shape)
        lib().orc_get_populations(self.h, k, _dp(out))
        return out

    def macroscopic(self, k=0):
        """(rho, u) with u = (sum_i f_i e_i + F/2) / rho; k = -1 for the mixture."""
        rho = np.zeros(self.shape)
        u = np.zeros((self.dim,) + self.shape)
        lib().orc_macroscopic(self.h, k, _dp(rho), _dp(u))
        return rho, u

    def force(self, k=0):
        F = np.zeros((self.dim,) + self.shape)
        lib().orc_force(self.h, k, _dp(F))
        return F

    def psi(self, k=0):
        """(psi, rho incl. virtual densities at boundary solids) at the current time."""
        psi = np.zeros(self.shape)
        rho = np.zeros(self.shape)
        lib().orc_psi(self.h, k, _dp(psi), _dp(rho))
        return psi, rho

    def diagnostics(self):
        mass = np.zeros(2)
        mom = np.zeros(6)
        lib().orc_diagnostics(self.h, _dp(mass), _dp(mom))
        return mass[: self.K], mom.reshape(2, 3)[: self.K]

    def boundary_solids(self):
        out = np.zeros(self.shape, dtype=np.uint8)
        lib().orc_boundary_solids(self.h, out.ctypes.data)
        return out

    # building blocks exposed for pinning ----------------------------------------
    def interaction_force(self, psi, U, rho=None, with_body=False):
        """F^k from given psi/U fields [K, nz, ny, nx] -> [K, nz, ny, nx, 3]."""
        psi = np.ascontiguousarray(np.asarray(psi, dtype=np.float64).reshape((self.K,) + self.shape))
        U = np.ascontiguousarray(np.asarray(U, dtype=np.float64).reshape((self.K,) + self.shape))
        rho = np.ascontiguousarray(np.zeros_like(psi) if rho is None else
                                   np.asarray(rho, dtype=np.float64).reshape(psi.shape))
        F = np.zeros((self.K,) + self.shape + (3,))
        lib().orc_interaction_force(self.h, _dp(psi), _dp(U), _dp(rho), int(with_body), _dp(F))
        return F

    def surface_Q(self, psi, node, k=0):
        """(Qxx, Qyy, Qxy) of the surface-tension adjustment at node (x, y) from a given
        psi field [K, nz, ny, nx] (Section 2.3)."""
        psi = np.ascontiguousarray(np.asarray(psi, dtype=np.float64).reshape((self.K,) + self.shape))
        x, y = node
        out = np.zeros(3)
        lib().orc_surface_Q(self.h, _dp(psi), int(x + self.shape[2] * y), k, _dp(out))
        return out

    def collide_single(self, f, F, k=0):
        fin = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
        Fv = np.ascontiguousarray(np.asarray(F, dtype=np.float64).reshape(3))
        out = np.zeros(self.Q)
        lib().orc_collide_single(self.h, k, _dp(fin), _dp(Fv), _dp(out))
        return out

    def mrt_matrices(self):
        M = np.zeros((self.Q, self.Q))
        Mi = np.zeros((self.Q, self.Q))
        lib().orc_mrt_matrices(self.h, _dp(M), _dp(Mi))
        return M, Mi


# ---------------------------------------------------------------------------
# Equation of state and Maxwell construction
# ---------------------------------------------------------------------------

def eos_Tc(eos, a, b, R=1.0):
    return lib().orc_eos_Tc(EOS[eos], a, b, R)


def eos_pressure(eos, a, b, R, omega, T_red, rho):
    return lib().orc_eos_pressure(EOS[eos], a, b, R, omega, T_red, float(rho))


def maxwell(eos, a, b, R=1.0, omega=0.0, T_red=0.8):
    """Coexistence (rho_g, rho_l, p_sat) of an EOS at T = T_red * Tc."""
    rg, rl, ps = C.c_double(), C.c_double(), C.c_double()
    rc = lib().orc_maxwell_eos(EOS[eos], a, b, R, omega, T_red, C.byref(rg), C.byref(rl),
                               C.byref(ps))
    if rc != 0:
        raise ValueError("no liquid-vapour loop (supercritical?)")
    return rg.value, rl.value, ps.value


def maxwell_bulk(case, k=0, rmin=1e-3, rmax=50.0):
    """Coexistence of the model's own bulk pressure c_s^2 rho + U(rho) of component k."""
    p = params_from_case(case)
    rg, rl, ps = C.c_double(), C.c_double(), C.c_double()
    rc = lib().orc_maxwell_bulk(C.byref(p), k, rmin, rmax, C.byref(rg), C.byref(rl), C.byref(ps))
    if rc != 0:
        raise ValueError("no liquid-vapour loop")
    return rg.value, rl.value, ps.value


def bulk_pressure(case, k, rho):
    p = params_from_case(case)
    return lib().orc_bulk_pressure(C.byref(p), k, float(rho))


def threads():
    return lib().orc_threads()
