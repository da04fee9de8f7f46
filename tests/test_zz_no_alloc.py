"""lbm_mass_noalloc: the mass reduction for callers that cannot allocate device memory.

It must give the mass that lbm_diagnostics gives for the same lattice, on two calls
in a row (the second reuses the scratch the first left behind), and it must refuse
lattices larger than its fixed scratch covers, 16-bit storage, and a stream that is
being captured into a CUDA graph (without breaking the capture). This file is
collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from synth import cases, random_field, random_solids

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_17713_gb300.build import build
    build()


def _lattice(variant):
    from paper_2506_17713_gb300 import Lattice
    if variant == "pr_f32":
        case, init = cases.droplets_3d_pr(shape=(48, 40, 36), count=1, rmin=10.0, rmax=10.0, seed=5)
        lat = Lattice(case)
        lat.init_fields(0, init["rho"][0])
    elif variant == "d2q9_cs_f64":
        case, init = cases.droplet_2d_cs(n=64, radius=14.0)
        lat = Lattice(case)
        lat.init_fields(0, init["rho"][0])
    else:
        shape = (23, 19, 17)
        case = cases.base_case("D3Q19", shape, ncomp=2, psi=["rho", "rho"], velocity="common", real="f64",
                               g=[[0.0, 0.05], [0.05, 0.0]], wet_phi=[1.1, 1.0])
        lat = Lattice(case)
        lat.set_geometry(random_solids(shape, 0.1, 91))
        lat.init_fields(0, random_field(shape, 0.4, 0.6, 92))
        lat.init_fields(1, random_field(shape, 0.4, 0.6, 93))
    lat.step(30)
    return lat


@pytest.mark.parametrize("variant", ["pr_f32", "d2q9_cs_f64", "two_comp_f64_solids"])
def test_mass_noalloc_matches_diagnostics_twice(variant):
    import torch
    from paper_2506_17713_gb300 import lbm
    lat = _lattice(variant)
    mass_ref, _ = lat.diagnostics()
    f = torch.stack([lat.populations(k) for k in range(lat.K)]).contiguous()
    stream = torch.cuda.current_stream().cuda_stream
    # lbm_diagnostics sums per-node densities that an FP32 lattice has rounded to FP32
    # (half an ulp each), this entry point the populations themselves in FP64: the
    # totals may differ by 2^-24 relative for FP32 lattices; FP64 agrees to rounding.
    rtol = 6e-8 if lat.case.get("real", "f32") == "f32" else 1e-12
    for _ in range(2):
        m = lbm.lbm_mass_noalloc(lat.params, f.data_ptr(), stream)
        assert np.allclose(m, mass_ref, rtol=rtol, atol=0.0), (m, mass_ref)
    lat.close()


def test_mass_noalloc_rejects_oversized_lattice():
    from paper_2506_17713_gb300 import lbm
    p = lbm.params_from_case(cases.base_case("D3Q19", (257, 256, 256)))
    mass = (C.c_double * 2)()
    # rejected before any device work, so a dummy pointer is never touched
    assert lbm.library().lbm_mass_noalloc(C.byref(p), C.c_void_p(256), mass, None) == 1


def test_mass_noalloc_rejects_16bit_storage():
    # the entry point reads populations as FP32 or FP64; shifted 16-bit buffers are refused
    # on the host, before any device work, so the dummy pointer is never touched
    from paper_2506_17713_gb300 import lbm
    for real in ("f16s", "bf16s"):
        p = lbm.params_from_case(cases.base_case("D3Q19", (16, 16, 16), real=real))
        mass = (C.c_double * 2)()
        assert lbm.library().lbm_mass_noalloc(C.byref(p), C.c_void_p(256), mass, None) == 1


def test_mass_noalloc_refuses_a_capturing_stream():
    # the call ends in a copy to host memory and a stream synchronisation, which capture
    # does not allow: it must return LBM_ERR_INVALID_ARG before enqueuing anything, so the
    # caller's capture completes and replays; outside the capture the same call works
    import torch
    from paper_2506_17713_gb300 import lbm
    lat = _lattice("pr_f32")
    mass_ref, _ = lat.diagnostics()
    f = torch.stack([lat.populations(k) for k in range(lat.K)]).contiguous()
    x = torch.zeros(4, device="cuda")
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    mass = (C.c_double * 2)()
    with torch.cuda.graph(g, stream=side):
        x.add_(1.0)
        st = torch.cuda.current_stream().cuda_stream
        code = lbm.library().lbm_mass_noalloc(C.byref(lat.params), C.c_void_p(f.data_ptr()), mass, C.c_void_p(st))
        x.add_(1.0)
    assert code == 1      # LBM_ERR_INVALID_ARG
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(x, torch.full_like(x, 2.0))
    m = lbm.lbm_mass_noalloc(lat.params, f.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert np.allclose(m, mass_ref, rtol=6e-8, atol=0.0)
    lat.close()
