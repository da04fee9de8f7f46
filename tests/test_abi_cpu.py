"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/lbm.h, and validates parameters on the host."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_17713_gb300.build import build
    build()
    from paper_2506_17713_gb300 import lbm
    return lbm.library()


def _declared(header="lbm.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    from paper_2506_17713_gb300 import lbm, nn
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(lbm.EXPORTS) == names
    nn_names = _declared("lbm_nn.h")
    assert len(nn_names) == 16
    for n in nn_names:
        assert hasattr(lib, n), n
    assert sorted(nn.EXPORTS) == nn_names


def test_network_entry_points_validate_arguments_on_the_host(lib):
    from paper_2506_17713_gb300 import nn
    L = nn.library()
    assert L.lbm_nn_conv3d(None, 1, 4, 4, 4, None, None, 1, 0, None, None) == 1
    assert L.lbm_nn_avg_pool2(C.c_void_p(256), 1, 3, 4, 4, C.c_void_p(256), None) == 1   # odd size
    assert L.lbm_nn_adam(None, None, None, None, 0, 0.0, 0.0, 0.0, 0.0, 1.0, 1.0, None) == 1
    # tensor-core forms: null pointers, more than 256 output channels, shared memory beyond 227 KB
    fake = C.c_void_p(256)
    assert L.lbm_nn_conv3d_tc(None, 1, 4, 4, 4, fake, None, 1, 0, fake, None) == 1
    assert L.lbm_nn_conv3d_tc(fake, 1, 4, 4, 4, fake, None, 300, 0, fake, None) == 1
    assert L.lbm_nn_conv3d_tc(fake, 256, 4, 4, 4, fake, None, 256, 0, fake, None) == 1
    assert L.lbm_nn_conv3d_tc_grad_input(fake, 300, 4, 4, 4, fake, 8, fake, fake, None) == 1
    assert L.lbm_nn_conv3d_tc_grad_weight(fake, 8, fake, 300, 4, 4, 4, fake, None, 0, fake, None) == 1
    assert L.lbm_nn_tc_error(None) == 1
    done = C.c_int(-1)
    assert L.lbm_nn_wait_selftest(0, C.byref(done), None) == 1               # limit out of range
    assert L.lbm_nn_wait_selftest(5_000_000_000, C.byref(done), None) == 1
    assert L.lbm_nn_wait_selftest(1000, None, None) == 1


def test_status_strings(lib):
    from paper_2506_17713_gb300 import lbm
    for code, name in lbm.STATUS.items():
        assert lbm.lbm_status_str(code) == name


def _case(**kw):
    from synth import cases
    c = cases.droplets_3d_pr(shape=(16, 12, 10), count=1, rmin=3, rmax=4, width=2, seed=1)[0]
    c.update(kw)
    return c


def test_workspace_size_layout(lib):
    from paper_2506_17713_gb300 import lbm
    c = _case()
    n = lbm.lbm_workspace_size(lbm.params_from_case(c))
    N = 16 * 12 * 10
    # two population buffers, psi, rho, mask, boundary list, u snapshot
    assert n >= 2 * 19 * N * 4 + 2 * N * 4 + N + 4 * N + 3 * N * 4
    n64 = lbm.lbm_workspace_size(lbm.params_from_case(dict(c, real="f64")))
    assert n64 > n
    n2 = lbm.lbm_workspace_size(lbm.params_from_case(dict(c, ncomp=2)))
    assert n2 >= n + 2 * 19 * N * 4
    # 16-bit population storage: 2-byte populations plus a staging region for host
    # transfers (Q N floats here)
    for real in ("f16s", "bf16s"):
        nh = lbm.lbm_workspace_size(lbm.params_from_case(dict(c, real=real)))
        assert nh >= 2 * 19 * N * 2 + 2 * N * 4 + N + 4 * N + 3 * N * 4 + 19 * N * 4
        assert nh < n + 19 * N * 4


@pytest.mark.parametrize("bad", [
    dict(tau=[0.5, 0.5]),
    dict(ncomp=3),
    dict(lattice="D2Q9"),                      # nz must be 1 in 2-D
    dict(bc=["periodic", "periodic", "pressure", "pressure", "periodic", "periodic"]),
    dict(bc=["wall", "periodic", "periodic", "periodic", "periodic", "periodic"]),
    dict(bc=["pressure", "pressure", "wall", "wall", "periodic", "periodic"]),  # bc_rho = 0
    dict(g=[[0.0, 0.0], [0.0, 0.0]]),          # EOS pseudopotential needs g_kk != 0
    dict(rho_lo=[2.0, 2.0], rho_hi=[1.0, 1.0]),
    dict(mrt_rates=[[2.5] * 19]),
    dict(T_red=[0.0, 0.0]),
    dict(shape=(2048, 1024, 1024)),            # 2^31 nodes: node indices are 32-bit
    dict(real="f16s", rho_ref=[float("nan"), 1.0]),
    dict(kappa=[0.5, 0.5]),                    # surface-tension source: D2Q9 MRT only
    dict(forcing="moment"),                    # moment-space forcing: D2Q9 only
    dict(lattice="D2Q9", shape=(16, 12, 1), accel=[[0.0, 0.0, 1e-5], [0.0, 0.0, 0.0]]),  # no z in 2-D
])
def test_rejects_invalid_parameters(lib, bad):
    from paper_2506_17713_gb300 import lbm
    c = _case(**bad)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_workspace_size(lbm.params_from_case(c))
    assert ei.value.status == 1


def test_null_arguments(lib):
    from paper_2506_17713_gb300 import lbm
    assert lib.lbm_workspace_size(None, None) == 1
    out = C.c_void_p()
    assert lib.lbm_create(None, None, 0, None, C.byref(out)) == 1
    p = lbm.params_from_case(_case())
    # workspace missing / too small / misaligned
    assert lib.lbm_create(C.byref(p), None, 0, None, C.byref(out)) == 2
    assert lib.lbm_create(C.byref(p), C.c_void_p(256), 16, None, C.byref(out)) == 2
    assert lib.lbm_create(C.byref(p), C.c_void_p(257), 1 << 40, None, C.byref(out)) == 2
    lib.lbm_destroy(None)


def test_params_mapping_roundtrip():
    from paper_2506_17713_gb300 import lbm
    from synth import cases
    c = cases.porous_two_component(shape=(24, 12, 10), buffer=3, porosity=0.7)[0]
    p = lbm.params_from_case(c)
    assert (p.nx, p.ny, p.nz, p.ncomp) == (24, 12, 10, 2)
    assert p.psi_kind[0] == lbm.PSI["rho"] and p.bc[0] == lbm.BC["pressure"]
    assert abs(p.g[0][1] - c["g"][0][1]) < 1e-15
    assert abs(p.bc_rho[0][1] - c["bc_rho"][0][1]) < 1e-15
    p16 = lbm.params_from_case(dict(c, real="bf16s", rho_ref=[0.25, 2.0]))
    assert p16.real == lbm.LBM_BF16S and list(p16.rho_ref) == [0.25, 2.0]


def test_mass_noalloc_rejects_16bit_storage_before_any_device_call(lib):
    # validation happens on the host: the (never dereferenced) device pointer is a dummy
    from paper_2506_17713_gb300 import lbm
    for real in ("f16s", "bf16s"):
        p = lbm.params_from_case(_case(real=real))
        mass = (C.c_double * 2)()
        assert lib.lbm_mass_noalloc(C.byref(p), C.c_void_p(256), mass, None) == 1
