"""The free-streaming bandwidth probe (lbm_stream_probe): each launch moves every
population one link along its direction, f_i(x) <- f_i(x - e_i), with periodic wrap,
bit for bit, and leaves no arithmetic on the values."""
import numpy as np
import pytest

from synth import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_17713_gb300.build import build
    build()


@pytest.mark.parametrize("lattice,shape,real,K", [("D3Q19", (20, 12, 9), "f32", 1), ("D3Q19", (17, 8, 6), "f64", 2),
                                                  ("D2Q9", (33, 21, 1), "f32", 1)])
def test_probe_streams_every_population_one_link(lattice, shape, real, K):
    import torch
    from paper_2506_17713_gb300 import Lattice
    case = cases.base_case(lattice, shape, real=real, ncomp=K, psi=["rho", "rho"], g=[[0.0, 0.0], [0.0, 0.0]])
    lat = Lattice(case)
    nz_, ny_, nx_ = shape[2], shape[1], shape[0]
    rng = np.random.default_rng(3)
    for k in range(K):
        lat.init_fields(k, np.ones((nz_, ny_, nx_)))
    e, _ = lat.velocity_set()
    f0 = []
    for k in range(K):
        f = rng.random((len(e), nz_, ny_, nx_))
        lat.set_populations(k, torch.from_numpy(f))
        f0.append(lat.populations(k).cpu().numpy())
    for steps in (1, 2):
        ms = lat.stream_probe(1)
        assert ms > 0.0
        for k in range(K):
            got = lat.populations(k).cpu().numpy()
            for i, (ex, ey, ez) in enumerate(e):
                ref = np.roll(f0[k][i], (steps * ez, steps * ey, steps * ex), axis=(0, 1, 2))
                assert np.array_equal(got[i], ref), (k, i, steps)
    lat.close()
