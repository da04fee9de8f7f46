"""Batches of lattices (lbm_batch_*): one persistent launch per pass for all
lattices, two steps per CUDA graph replay. The per-node arithmetic is that of
lbm_step, so every lattice of a batch must end bit for bit where the same lattice
stepped on its own ends; one sample is also checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from synth import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_17713_gb300.build import build
    build()


def _lattice(case, init):
    from paper_2506_17713_gb300 import Lattice
    lat = Lattice(case)
    if init.get("solid") is not None:
        lat.set_geometry(init["solid"])
    for k, r in enumerate(init["rho"]):
        lat.init_fields(k, r)
    return lat


def _twins(samples):
    return [_lattice(c, i) for c, i in samples], [_lattice(c, i) for c, i in samples]


def _same(batched, single):
    import torch
    for a, b in zip(batched, single):
        for k in range(a.K):
            assert torch.equal(a.populations(k), b.populations(k))
        ma, pa = a.diagnostics()
        mb, pb = b.diagnostics()
        assert np.array_equal(ma, mb) and np.array_equal(pa, pb)


def _sphere_packs(count=4, real="f32"):
    return cases.sphere_pack_batch(count=count, edge_lo=24, edge_hi=40, seed=31, real=real)


@pytest.mark.parametrize("steps", [1, 6, 7])
def test_sphere_pack_batch_matches_single_lattices_bitwise(steps):
    from paper_2506_17713_gb300 import Batch
    samples = _sphere_packs()
    lats, refs = _twins(samples)
    batch = Batch(lats)
    batch.step(steps)
    for r in refs:
        r.step(steps)
    _same(lats, refs)


def test_batch_then_single_steps_continue_the_same_state():
    # an odd batch step count swaps every lattice's buffers; single steps afterwards
    # and further batch steps must continue from the right buffer
    from paper_2506_17713_gb300 import Batch
    lats, refs = _twins(_sphere_packs(3))
    batch = Batch(lats)
    batch.step(5)
    lats[1].step(1)
    batch.step(4)
    for i, r in enumerate(refs):
        r.step(10 if i == 1 else 9)
    _same(lats, refs)


def test_periodic_lattices_without_solids_bitwise():
    # no fluid list: the batched kernels index every node and rebuild (x, y, z)
    from paper_2506_17713_gb300 import Batch
    samples = []
    for i, shape in enumerate([(37, 29, 23), (48, 20, 33), (30, 30, 30)]):
        case, init = cases.droplets_3d_pr(shape=shape, count=1, rmin=6.0, rmax=8.0, width=4.0, seed=40 + i)
        samples.append((case, init))
    lats, refs = _twins(samples)
    Batch(lats).step(6)
    for r in refs:
        r.step(6)
    _same(lats, refs)


def test_two_component_pressure_faces_bitwise():
    from paper_2506_17713_gb300 import Batch
    samples = [cases.porous_two_component(shape=s, porosity=0.6, corr_length=3.0, buffer=3, seed=50 + i)
               for i, s in enumerate([(36, 16, 14), (28, 20, 12)])]
    lats, refs = _twins(samples)
    Batch(lats).step(8)
    for r in refs:
        r.step(8)
    _same(lats, refs)


def test_sixteen_bit_storage_bitwise():
    from paper_2506_17713_gb300 import Batch
    samples = _sphere_packs(3, real="f16s")
    for c, _ in samples:
        c["rho_ref"] = [c["bc_rho"][1][0]] * 2
    lats, refs = _twins(samples)
    Batch(lats).step(6)
    for r in refs:
        r.step(6)
    _same(lats, refs)


def test_autotune_keeps_results_and_reports_launch_shapes():
    from paper_2506_17713_gb300 import Batch
    lats, refs = _twins(_sphere_packs())
    batch = Batch(lats)
    cfg = batch.autotune()
    assert len(cfg) == 3
    for block, grid in cfg:
        assert block in (128, 256) and grid >= 1
    batch.step(6)
    for r in refs:
        r.step(6)
    _same(lats, refs)


def test_launch_count_and_graph_replays():
    from paper_2506_17713_gb300 import Batch
    lats, _ = _twins(_sphere_packs(2))
    batch = Batch(lats)
    n0 = batch.launches()
    batch.step(6)
    # three passes per step (the packs have boundary solids), one launch each for the
    # whole batch
    assert batch.launches() - n0 == 6 * 3


def test_sample_against_oracle():
    from paper_2506_17713_gb300 import Batch
    samples = _sphere_packs(2)
    lats = [_lattice(c, i) for c, i in samples]
    Batch(lats).step(20)
    case, init = samples[1]
    orc = oracle.OracleSim(case)
    orc.set_geometry(init["solid"])
    orc.init_fields(0, init["rho"][0])
    orc.step(20)
    rg, ug = lats[1].macroscopic_host(0)
    ro, uo = orc.macroscopic(0)
    assert np.abs(rg - ro).max() / np.abs(ro).max() <= 1e-5
    for d in range(3):
        assert np.abs(ug[d] - uo[d]).max() / np.abs(uo[d]).max() <= 1e-5


def test_incompatible_or_repeated_lattices_are_rejected():
    from paper_2506_17713_gb300 import Batch, LbmError
    a = _lattice(*_sphere_packs(1)[0])
    c2, i2 = cases.porous_two_component(shape=(24, 12, 10), porosity=0.6, corr_length=3.0, buffer=3)
    b = _lattice(c2, i2)
    with pytest.raises(LbmError) as ei:
        Batch([a, b])
    assert ei.value.status == 1
    with pytest.raises(LbmError) as ei:
        Batch([a, a])
    assert ei.value.status == 1


def test_full_size_batch_matches_single_lattices_bitwise():
    # the 64-sample benchmark batch (edges U[64, 192]) in its benchmark launch
    # configuration (autotuned, graph replays); the smallest and the largest sample
    # are stepped on their own as well and must end bit for bit equal
    from paper_2506_17713_gb300 import Batch
    samples = cases.sphere_pack_batch(count=64)
    lats = [_lattice(c, i) for c, i in samples]
    sizes = [l.N for l in lats]
    pick = [int(np.argmin(sizes)), int(np.argmax(sizes))]
    refs = [_lattice(*samples[j]) for j in pick]
    batch = Batch(lats)
    batch.autotune()
    batch.step(4)
    for r in refs:
        r.step(4)
    _same([lats[j] for j in pick], refs)
    m, _ = lats[pick[1]].diagnostics()
    assert np.isfinite(m).all()
