"""Host-side logic of bench.py, without a GPU: the byte model of the roofline,
the max-over-ranks aggregation of the N > 1 path (two gloo ranks) and the
reference arm's JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_algorithmic_bytes():
    import bench
    from synth import cases
    c = cases.droplets_3d_pr(shape=(8, 8, 8), count=1, rmin=2, rmax=2)[0]
    b = bench.algorithmic_bytes(c)
    # FP32 D3Q19, one component, periodic: 19*4 read + 19*4 write + psi read; 19*4 read + psi write
    assert b == {"collide": 156, "density": 80, "step": 236}
    c2 = cases.porous_two_component(shape=(20, 10, 10), porosity=0.7, corr_length=2.0, buffer=2)[0]
    b2 = bench.algorithmic_bytes(c2)
    assert b2["collide"] == 2 * 2 * 19 * 4 + 2 * 4 + 1
    assert b2["density"] == 2 * 19 * 4 + 2 * 4 + 2 * 4 + 1
    b3 = bench.algorithmic_bytes(c2, fluid_list=True)      # per fluid node: list + slot map, no mask
    assert b3["collide"] == b2["collide"] - 1 + 8 and b3["density"] == b2["density"] - 1 + 8


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), BENCH_BACKEND="gloo")
    import bench
    w, r, _ = bench.dist_setup()
    secs = 1.0 + r  # rank 1 is the slow one
    bench.barrier(w)
    m = bench.reduce_max(secs, w)
    q.put((r, m, bench.aggregate(100.0, m, w)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_gloo_max_and_aggregate():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the max time (2 s); whole-job units / max time
    assert [o[1] for o in out] == [2.0, 2.0]
    assert [o[2] for o in out] == [100.0, 100.0]


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "24",
                        "--steps", "2", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_committed_traffic_is_gated_by_kernel_source_hash(monkeypatch):
    import bench
    path = os.path.join(ROOT, "profiles", "dram_traffic_pr256_n256.md")
    if not os.path.exists(path):
        pytest.skip("no committed DRAM traffic summary")
    digest = next(l.split(":", 1)[1].strip() for l in open(path) if l.startswith("kernel sources sha256:"))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: digest)
    t = bench.committed_traffic("k_collide", "pr256", 256)
    assert isinstance(t, int) and t > 0
    assert bench.committed_traffic("k_collide", "pr256", 128) is None      # no summary for that size
    # the FP32 instantiation's bytes are not those of the 16-bit storage kernels
    assert bench.committed_traffic("k_collide", "pr256", 256, "f16s") is None
    assert bench.committed_traffic("k_collide", "pr256", 256, "bf16s") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 64)
    assert bench.committed_traffic("k_collide", "pr256", 256) is None      # kernels changed since the capture


def test_macroscopic_output_layout_follows_the_lattice():
    # lbm_macroscopic writes doubles for FP64 lattices and D velocity rows: the end-to-end
    # host buffers of the benchmark must match, or the copy overruns them
    import bench
    assert bench.macroscopic_layout(bench.make_case("cs128")[0]) == ("float64", 2)
    assert bench.macroscopic_layout(bench.make_case("pr256", 32)[0]) == ("float32", 3)
    c = dict(bench.make_case("pr256", 32)[0], real="f16s")
    assert bench.macroscopic_layout(c) == ("float32", 3)
