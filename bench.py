"""Throughput of the D3Q19 Shan-Chen multiphase step on GB300 (MLUPS, % HBM roofline).

Workload (default): D3Q19 single-component Shan-Chen, Peng-Robinson EOS
(a = 2/49, b = 2/21, R = 1, omega = 0.344, T = 0.6 Tc), MRT collision, 256^3
periodic lattice, FP32, 8 droplets with seeded radii U[12, 40] at random
non-overlapping centres. A step is one lattice time step over the whole
lattice (density pass + collide pass). MLUPS = components * nx * ny * nz *
steps / (seconds * 1e6).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun) every rank advances its own lattice (independent
replicas, weak scaling); ranks only meet at the timing barriers.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "pr256": "D3Q19 Shan-Chen PR T=0.6Tc MRT 256^3 FP32, 8 droplets (seed 1234)",
    "exp256": "D3Q19 Shan-Chen psi=exp(-1/rho) BGK 256^3 FP32, droplet R=30",
    "cs128": "D2Q9 Shan-Chen CS T=0.7Tc BGK 128^2 FP64, droplet R=25 (the small parity case; L2-resident)",
    "porous400": "D3Q19 two-component Shan-Chen 400^3 FP32, GRF porous medium (porosity 0.15, "
                 "corr. length 6, seed 7), wetting, constant-density x faces",
    "warmstart": "learned warm start of single-phase steady-state runs: D3Q19 BGK, periodic GRF porous "
                 "samples (porosity U[0.1,0.35], corr. length 6), body force; 3-D U-Net trained on LBM steady states",
    "conv3d": "one periodic 3x3x3 convolution layer of the warm-start U-Net (FP32 activations): forward, "
              "adjoint and weight gradient, BF16 tensor cores vs FP32 CUDA cores",
    "warmstart_errors": "which errors of a warm start cost relaxation steps: the warm-start samples started from "
                        "their converged field with a scaled magnitude, white or smooth velocity noise, or density "
                        "noise, and from the run's own early field rescaled to the exact flux",
    "batch64": "64 D3Q19 sphere-pack drainage samples, box edges U[64,192] (seed 2024), overlapping spheres "
               "r U[8,12] to porosity 0.38, PR T=0.8Tc MRT FP32, wetting solids, per-sample inlet pressure step",
    "drainage400": "the porous400 drainage as configured: non-wetting phase injected through the constant-density "
                   "inlet into the wetting-saturated 400^3 GRF medium (45-degree wetting), 20000 steps, FP32 "
                   "storage and FP16 / BF16 shifted storage; saturation history and breakthrough",
}


# populations as stored; compute is FP32 except for f64
STORAGE = {"f32": "f32", "f64": "f64", "f16s": "f16 deviations f_i - w_i rho_ref",
           "bf16s": "bf16 deviations f_i - w_i rho_ref"}


def ref_density(workload):
    """Default reference density of 16-bit storage: the vapour coexistence density of
    the droplet workloads (vapour populations are then stored almost exactly and liquid
    ones round relative to their own size), 1 (the lattice weights) otherwise."""
    from synth import cases
    return {"pr256": cases.COEX[("PR", 0.6)][0], "exp256": cases.EXP_COEX[0]}.get(workload, 1.0)


def make_case(name, n=256):
    from synth import cases
    if name == "pr256":
        if n == 256:
            case, init = cases.droplets_3d_pr(n=n)
        else:  # smaller cubes (profiling captures, tests): radii and width scaled with the edge
            f = n / 256.0
            case, init = cases.droplets_3d_pr(n=n, rmin=12.0 * f, rmax=40.0 * f,
                                              width=max(2.0, cases.PR06_WIDTH * f))
    elif name == "exp256":
        case, init = cases.droplet_3d_exp(n=n, radius=30.0 * n / 256)
    elif name == "cs128":
        case, init = cases.droplet_2d_cs(n=128 if n == 256 else n)
    elif name == "batch64":   # the oracle-timed stand-in: the first sample of the batch
        case, init = cases.sphere_pack_batch(count=1)[0]
    elif name == "porous400":
        m = 400 if n == 256 else n
        case, init = cases.porous_two_component(shape=(m, m, m))
    else:
        raise SystemExit("unknown workload " + name)
    return case, init


def macroscopic_layout(case):
    """(element type name, velocity rows) of what lbm_macroscopic writes: the compute
    type (double for FP64 lattices, float otherwise) and D velocity components"""
    return ("float64" if case.get("real") == "f64" else "float32"), (3 if case["lattice"] == "D3Q19" else 2)


def l2_note(case, K, N):
    Q = 19 if case["lattice"] == "D3Q19" else 9
    ep = {"f16s": 2, "bf16s": 2, "f64": 8}.get(case.get("real", "f32"), 4)
    gb = K * Q * N * ep / 1e9
    if 2 * gb > 0.129:
        return "inputs larger than L2 (two %.2f GB population buffers)" % gb
    return ("inputs L2-resident (two %.1f MB population buffers): a launch- and latency-bound case, "
            "not an HBM measurement" % (gb * 1e3))


def algorithmic_bytes(case, fused=False, fluid_list=False):
    """Bytes each kernel must move per lattice update of one node it processes (DRAM,
    each value once). Two-pass schedule -- collide: read K*Q populations + K psi
    [+ 1 B mask], write K*Q populations; density: read K*Q populations [+ 1 B mask],
    write K psi [+ K rho next to solids]. With solids the kernels run over the fluid-node
    list: the units are fluid nodes, whose populations sit at fluid slots, and each reads
    its 4 B list entry and 4 B node -> slot map entry instead of the mask. Single-pass
    schedule (k_fused): read and write K*Q populations."""
    Q = 19 if case["lattice"] == "D3Q19" else 9
    e = 8 if case.get("real") == "f64" else 4                       # scalars (psi, rho)
    ep = 2 if case.get("real") in ("f16s", "bf16s") else e          # stored populations
    K = int(case.get("ncomp", 1))
    geom = any(b != "periodic" for b in case.get("bc", ["periodic"] * 6)) or fluid_list
    if fused:
        return {"collide": 2 * K * Q * ep, "density": 0, "step": 2 * K * Q * ep}
    # with solids: populations at fluid slots, a 4 B list entry and a 4 B node -> slot map
    # entry per fluid node replace the 1 B mask
    lst, mask = (8, 0) if fluid_list else (0, 1 if geom else 0)
    collide = 2 * K * Q * ep + K * e + mask + lst
    density = K * Q * ep + K * e + (K * e + mask if geom else 0) + lst
    return {"collide": collide, "density": density, "step": collide + density}


KERNEL_SOURCES = ("args.h", "kernels.cuh", "lattice.cuh")


def kernel_source_hash():
    """sha256 over the sources that define the step kernels (order fixed)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2506_17713_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


# compute and storage types in a step kernel's template arguments, per population storage
KERNEL_TYPES = {"f32": "float, float", "f64": "double, double", "f16s": "float, __half",
                "bf16s": "float, __nv_bfloat16"}


def committed_traffic(kernel, workload, n, real="f32"):
    """DRAM bytes per launch of `kernel` (dram__bytes_read.sum + dram__bytes_write.sum)
    from the committed ncu summary of this workload, for the instantiation of this
    population storage, or None when there is none or the kernel sources have changed
    since it was captured."""
    path = os.path.join(ROOT, "profiles", "dram_traffic_%s_n%d.md" % (workload, n))
    if not os.path.exists(path):
        return None
    digest, value = None, None
    with open(path) as fh:
        for line in fh:
            if line.startswith("kernel sources sha256:"):
                digest = line.split(":", 1)[1].strip()
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) >= 5 and cells[0].startswith(kernel + "<") and \
                    (", %s," % KERNEL_TYPES[real]) in cells[0]:
                try:
                    value = int(cells[4])
                except ValueError:
                    pass
    if digest != kernel_source_hash():
        return None
    return value


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples taken while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def reduce_max(value, world, device=None):
    """Maximum of a float over ranks (the timing rule of the benchmark)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def aggregate(units_per_rank, seconds_per_rank_max, world):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / seconds_per_rank_max


# ---------------------------------------------------------------------------
# Reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_sample(case, init, steps=None, seconds=None):
    """Time oracle steps on the given lattice; returns (MLUPS, seconds, threads, steps).
    With `seconds`, one untimed warm-up step and one timed step size the sample to about
    that much CPU time."""
    import oracle
    s = oracle.OracleSim(case)
    if init.get("solid") is not None:
        s.set_geometry(init["solid"])
    for k, r in enumerate(init["rho"]):
        s.init_fields(k, r)
    dt = 0.0
    if seconds is not None:
        s.step(1)                                  # untimed: threads start, pages fault in
        t0 = time.perf_counter()
        s.step(1)
        dt = time.perf_counter() - t0
        steps = int(min(200000, max(1, round(seconds / max(dt, 1e-6)))))
        steps_left = steps - 1
    else:
        steps_left = steps
    t0 = time.perf_counter()
    s.step(steps_left)
    dt += time.perf_counter() - t0
    K = int(case.get("ncomp", 1))
    nx, ny, nz = case["shape"]
    return K * nx * ny * nz * steps / dt / 1e6, dt, oracle.threads(), steps


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    case, init = make_case(args.workload, args.n)
    steps = max(1, min(args.steps, args.ref_steps))
    oracle_sample(case, init, 1)                                  # warm-up (page-in)
    mlups, dt, threads, _ = oracle_sample(case, init, steps)
    nx, ny, nz = case["shape"]
    sample = "%d oracle steps on the full %dx%dx%d lattice (FP64, OpenMP)" % (steps, nx, ny, nz)
    line = {
        "impl": "reference", "metric": "%s Shan-Chen MLUPS" % case["lattice"], "value": round(mlups, 3),
        "unit": "MLUPS", "n_gpus": args.gpus, "steps": steps, "warmup": 1,
        "ms_per_step": round(1e3 * dt / steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "shape": [nx, ny, nz], "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def run_batch(args):
    """Many lattices in one batch (one persistent launch per pass, two steps per CUDA
    graph replay), against the same lattices stepped one after another."""
    import torch
    from paper_2506_17713_gb300 import Batch, Lattice
    from synth import cases

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    count = args.batch_count
    samples = cases.sphere_pack_batch(count=count, edge_lo=args.batch_edge_lo, edge_hi=args.batch_edge_hi)
    lats = []
    for case, init in samples:
        case["real"] = args.real
        if args.real in ("f16s", "bf16s"):
            case["rho_ref"] = [case["bc_rho"][1][0]] * 2
        lat = Lattice(case)
        lat.set_geometry(init["solid"])
        lat.init_fields(0, init["rho"][0])
        lats.append(lat)
    N = sum(l.N for l in lats)
    n_fluid = sum(int(np.count_nonzero(init["solid"] == 0)) for _, init in samples)
    stream = lats[0].stream
    batch = Batch(lats)
    cfg = batch.autotune()
    batch.step(args.warmup + (args.warmup & 1))
    torch.cuda.synchronize()

    def timed(fn, steps):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier(world, dev)
        torch.cuda.synchronize()
        ev0.record(stream)
        fn(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / 1e3

    steps = args.steps + (args.steps & 1)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    n0 = batch.launches()
    t_batch = timed(batch.step, steps)
    launches = batch.launches() - n0
    clk = clocks.stop()

    def sequential(k):
        for _ in range(k):
            for lat in lats:
                lat.step(1)
    seq_steps = max(2, min(steps, args.batch_seq_steps))
    t_seq = timed(sequential, seq_steps)
    t_max = reduce_max(t_batch, world, dev)
    mlups = aggregate(N * steps, t_max, world) / 1e6
    seq_mlups = N * seq_steps / t_seq / 1e6
    # bytes per fluid node of one step: density (K Q + psi + rho + mask + list) and collide
    ab = algorithmic_bytes(samples[0][0] | {"real": args.real}, fluid_list=True)
    step_gbs = ab["step"] * n_fluid * steps / t_batch / 1e9
    peak, peak_kind = load_peaks()
    if rank != 0:
        barrier(world, dev)
        return
    line = {
        "metric": "D3Q19 Shan-Chen MLUPS", "value": round(mlups, 1), "unit": "MLUPS",
        "n_gpus": world, "steps": steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * t_max / steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS["batch64"].replace("64 D3Q19", "%d D3Q19" % count)
                   .replace("U[64,192]", "U[%d,%d]" % (args.batch_edge_lo, args.batch_edge_hi)),
                   "lattices": count, "nodes": N, "fluid_nodes": n_fluid,
                   "mflups": round(mlups * n_fluid / N, 1), "storage": STORAGE[args.real],
                   "launch": "one persistent launch per pass for all lattices, 2 steps per CUDA graph replay",
                   "autotuned": {"density": cfg[0], "virtual": cfg[1], "collide": cfg[2]},
                   "parallelism": "replicas" if world > 1 else "single-gpu",
                   "l2": "inputs larger than L2 (%.1f GB of populations)" % (
                       2 * 19 * N * (2 if args.real in ("f16s", "bf16s") else 4) / 1e9)},
        "roofline": {"bound": "hbm", "kernel": "batched step (density + virtual + collide passes)",
                     "achieved": round(step_gbs, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(step_gbs / peak, 4), "peak_kind": peak_kind, "traffic": None,
                     "bytes_per_lu": ab["step"], "units_per_launch": n_fluid},
        "sequential": {"value": round(seq_mlups, 1), "unit": "MLUPS", "steps": seq_steps,
                       "ms_per_step": round(1e3 * t_seq / seq_steps, 4),
                       "launch": "lbm_step per lattice, one lattice after another"},
        "speedup_vs_sequential": round(mlups / seq_mlups, 3),
        "cpu_baseline": None, "e2e": None,
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        barrier(world, dev)
    batch.close()


def run_conv3d(args):
    """Throughput of the warm-start network's convolution passes on one layer: the
    tcgen05 implicit GEMMs (BF16 operands, FP32 accumulation) against the FP32
    CUDA-core kernels, 2 * 27 * cin * cout flops per voxel and pass, CUDA events over
    --steps repetitions of each pass after --warmup."""
    import torch
    from paper_2506_17713_gb300 import nn
    torch.cuda.set_device(0)
    cin, cout, n = args.conv_cin, args.conv_cout, args.conv_n
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(cin, n, n, n, device="cuda", generator=g)
    gy = torch.randn(cout, n, n, n, device="cuda", generator=g)
    w = torch.randn(cout, cin, 27, device="cuda", generator=g) * (2.0 / (27 * cin)) ** 0.5
    b = torch.randn(cout, device="cuda", generator=g)
    y = torch.empty(cout, n, n, n, device="cuda")
    gx = torch.empty(cin, n, n, n, device="cuda")
    wt = torch.empty(cin * cout * 27, device="cuda")
    gw = torch.empty(cout, cin, 27, device="cuda")
    gb = torch.empty(cout, device="cuda")
    sc = torch.empty(max(nn.gw_scratch_floats(cin, cout, True), nn.gw_scratch_floats(cin, cout, False)),
                     device="cuda")
    flops = 2.0 * 27 * cin * cout * n ** 3
    passes = {"forward": lambda tc: nn.conv3d(x, w, b, True, y, tc=tc),
              "grad_input": lambda tc: nn.conv3d_grad_input(gy, w, wt, gx, tc=tc),
              "grad_weight": lambda tc: nn.conv3d_grad_weight(x, gy, gw, gb, False, sc, tc=tc)}
    res = {}
    clk_sampler = ClockSampler(0)
    clk_sampler.start()
    for tc in (True, False):
        for name, fn in passes.items():
            for _ in range(args.warmup):
                fn(tc)
            torch.cuda.synchronize()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(args.steps):
                fn(tc)
            e.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(e) / args.steps
            res[("tc_" if tc else "fp32_") + name] = {"ms": round(ms, 4), "tflops": round(flops / ms / 1e9, 2)}
    clk = clk_sampler.stop()
    if nn.tc_error():
        raise RuntimeError("a tensor-core wait gave up")
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
        peak = float(json.load(fh)["bf16_tflops"])
    fwd = res["tc_forward"]
    launches = 3 * (args.steps + args.warmup) + 2 * 2 * (args.steps + args.warmup)   # tc: 1 + 2 + 2 per rep
    print(json.dumps({
        "metric": "conv3d forward TFLOP/s (BF16 tensor cores)", "value": fwd["tflops"], "unit": "TFLOP/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": fwd["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": WORKLOADS["conv3d"], "cin": cin, "cout": cout, "edge": n,
                   "l2": "input %.0f MB and output %.0f MB per pass against a 129 MB L2" % (
                       cin * n ** 3 * 4 / 1e6, cout * n ** 3 * 4 / 1e6)},
        "passes": res,
        "roofline": {"bound": "tensor", "kernel": "k_conv3d_tc", "achieved": fwd["tflops"], "peak": peak,
                     "unit": "TFLOP/s", "frac": round(fwd["tflops"] / peak, 4), "peak_kind": "measured bf16 burst",
                     "traffic": None},
        "gpu_launches": launches, "clocks": clk}))


def _smooth_in_fluid(u, solid, it):
    """`it` Jacobi sweeps of the 7-point mean over fluid nodes (solids stay 0)"""
    fl = (solid == 0).astype(np.float64)
    v = u * fl
    for _ in range(it):
        acc, cnt = v.copy(), fl.copy()
        for ax in (-1, -2, -3):
            for sh in (1, -1):
                acc += np.roll(v, sh, axis=ax)
                cnt += np.roll(fl, sh, axis=ax)
        v = np.where(fl > 0, acc / np.maximum(cnt, 1), 0.0)
    return v


def run_warmstart_errors(args):
    """Steps to the residual criterion from perturbed converged fields of the warm-start
    samples (the first --ws-test held-out seeds, capped at 4): what kind of error in a
    predicted start the relaxation pays for."""
    import torch
    from paper_2506_17713_gb300 import warmstart as ws
    from synth import uniform
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    n, ntrain = args.ws_n, args.ws_train
    phis = [0.10 + 0.25 * float(v) for v in uniform(4242, ntrain + args.ws_test)]
    rng = np.random.default_rng(0)
    rows = []
    for j in range(min(4, args.ws_test)):
        solid = ws.sample_solid(n, 5000 + j, phis[ntrain + j])
        fl = solid == 0
        sp, _, _, _, up, rp = ws.relax(n, solid, None)
        up, rp = up.astype(np.float64), rp.astype(np.float64)
        U = np.abs(up[0][fl]).mean()
        r = {"porosity": round(phis[ntrain + j], 4), "rest": sp}
        r["exact_velocity"] = ws.relax(n, solid, up)[0]
        r["exact_velocity_and_density"] = ws.relax(n, solid, up, rho0=rp)[0]
        r["0.7x_velocity_exact_density"] = ws.relax(n, solid, 0.7 * up, rho0=rp)[0]
        r["1.5x_velocity_exact_density"] = ws.relax(n, solid, 1.5 * up, rho0=rp)[0]
        white = rng.standard_normal(up.shape) * 0.3 * U * fl
        r["velocity_plus_30pct_white_noise_exact_density"] = ws.relax(n, solid, up + white, rho0=rp)[0]
        r["velocity_plus_10pct_white_noise_exact_density"] = ws.relax(n, solid, up + white / 3, rho0=rp)[0]
        r["velocity_plus_3pct_white_noise_exact_density"] = ws.relax(n, solid, up + white / 10, rho0=rp)[0]
        r["velocity_plus_10pct_white_noise_density_1"] = ws.relax(n, solid, up + white / 3)[0]
        sm = _smooth_in_fluid(rng.standard_normal(up.shape) * fl, solid, 6)
        sm *= 0.3 * U / max(np.abs(sm[0][fl]).mean(), 1e-30)
        r["velocity_plus_30pct_smooth_noise_exact_density"] = ws.relax(n, solid, up + sm, rho0=rp)[0]
        dn = 0.01 * (rp - 1.0).std() * rng.standard_normal(rp.shape)
        r["exact_velocity_density_plus_1pct_noise"] = ws.relax(n, solid, up, rho0=rp + dn)[0]
        # the run from rest stopped after m steps, its departure from rest scaled by the exact
        # q_inf / q(m) (a perfect magnitude prediction applied to the LBM's own early field)
        q_inf = float(up[0][fl].mean())
        for m in (200, 800):
            r["rest_%d_steps_then_exact_flux_rescale" % m], r["flux_ratio_at_%d" % m] = \
                ws.relax_scaled_early_field(n, solid, m, q_inf)
        rows.append(r)
    if rank != 0:
        return
    keys = [k for k in rows[0] if k != "porosity" and not k.startswith("flux_ratio")]
    print(json.dumps({
        "metric": "steps to residual <= 1e-6 by start (mean over samples)", "value": float(np.mean([r["rest"] for r in rows])),
        "unit": "steps", "n_gpus": world, "steps": int(sum(sum(r[k] for k in keys) for r in rows)), "warmup": 0,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS["warmstart_errors"], "edge": n, "samples": len(rows),
                   "noise": "relative to the mean |u_x| over the fluid; density noise relative to the std of rho - 1"},
        "mean_steps": {k: float(np.mean([r[k] for r in rows])) for k in keys},
        "per_sample": rows, "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None}), flush=True)


def run_warmstart(args):
    """Time to steady state (residual <= 1e-6) of held-out samples, from the network's
    prediction vs from rest; the network is trained in the same run on steady states
    the LBM produces."""
    import torch
    from paper_2506_17713_gb300 import warmstart as ws
    from synth import uniform

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    n, ntrain, ntest = args.ws_n, args.ws_train, args.ws_test
    u = uniform(4242, ntrain + ntest)
    phis = [0.10 + 0.25 * float(v) for v in u]
    t0 = time.perf_counter()
    solids, us, res = [], [], []
    for b0 in range(0, ntrain, 64):
        sl = slice(b0, min(ntrain, b0 + 64))
        so, uu, rr = ws.steady_states(n, list(range(1000 + sl.start, 1000 + sl.stop)), phis[sl], args.ws_steps)
        for a, b_, c in zip(so, uu, rr):       # train on converged fields only
            if c <= 1e-5:
                solids.append(a)
                us.append(b_)
                res.append(c)
    t_data = time.perf_counter() - t0
    net = ws.UNet(n, channels=(args.ws_c1, 2 * args.ws_c1, 4 * args.ws_c1), seed=0,
                  tensor_cores=not args.ws_fp32)
    t0 = time.perf_counter()
    hist = ws.train(net, solids, us, epochs=args.ws_epochs, batch=8)
    coef = ws.fit_scale(net, solids, us)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    rows, ideal, pred_err, scale_err = [], [], [], []
    for j in range(ntest):
        solid = ws.sample_solid(n, 5000 + j, phis[ntrain + j])
        sp, tp, kp, _, u_plain, rho_plain = ws.relax(n, solid, None)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pred, rho_pred = ws.predict(net, solid, coef)
        t_inf = time.perf_counter() - t0
        sw, tw, kw, _, _, _ = ws.relax(n, solid, pred, rho0=rho_pred)
        rows.append((sp, tp, sw, tw + t_inf, kp, kw))
        # bounds: start from the converged velocity alone, and from velocity and density;
        # diagnostics: the predicted shape at the true scale, and the prediction without density
        true_scale = ws.scale_of(u_plain, solid) / ws.scale_of(pred, solid)
        ideal.append((ws.relax(n, solid, u_plain.astype(np.float64))[0],
                      ws.relax(n, solid, u_plain.astype(np.float64), rho0=rho_plain.astype(np.float64))[0],
                      ws.relax(n, solid, pred * true_scale, rho0=rho_pred)[0],
                      ws.relax(n, solid, pred)[0]))
        pred_err.append(float(np.linalg.norm(pred - u_plain) / np.linalg.norm(u_plain)))
        scale_err.append(ws.scale_of(pred, solid) / ws.scale_of(u_plain, solid))
    r = np.array(rows)
    kerr = np.abs(r[:, 5] - r[:, 4]) / np.abs(r[:, 4])
    if rank != 0:
        return
    line = {
        "metric": "time-to-steady-state speedup (warm start vs plain LBM)",
        "value": round(float(r[:, 1].sum() / r[:, 3].sum()), 3), "unit": "x", "n_gpus": world,
        "steps": int(r[:, 2].sum()), "warmup": 0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS["warmstart"], "edge": n, "train_samples": ntrain, "test_samples": ntest,
                   "network": "3-D U-Net, channels %d/%d/%d, %d parameters, %s" % (
                       args.ws_c1, 2 * args.ws_c1, 4 * args.ws_c1, net.parameters(),
                       "FP32 CUDA-core convolutions" if args.ws_fp32
                       else "BF16 tensor-core convolutions (FP32 accumulation)"),
                   "epochs": args.ws_epochs, "final_train_loss": round(hist[-1], 4),
                   "converged_train_samples": len(solids),
                   "train_residual_max": float(max(res)), "data_seconds": round(t_data, 1),
                   "train_seconds": round(t_train, 1)},
        "steps_to_steady": {"plain_mean": float(r[:, 0].mean()), "warm_mean": float(r[:, 2].mean()),
                            "ratio": round(float(r[:, 0].sum() / r[:, 2].sum()), 3),
                            "from_converged_velocity_mean": float(np.mean([i[0] for i in ideal])),
                            "from_converged_velocity_and_density_mean": float(np.mean([i[1] for i in ideal])),
                            "predicted_shape_and_density_at_true_scale_mean": float(np.mean([i[2] for i in ideal])),
                            "predicted_velocity_without_density_mean": float(np.mean([i[3] for i in ideal]))},
        "prediction_rel_l2_error_mean": round(float(np.mean(pred_err)), 4),
        "predicted_over_true_scale": [round(float(v), 3) for v in scale_err],
        "scale_fit": [round(float(c), 4) for c in coef],
        "wall_seconds": {"plain_total": round(float(r[:, 1].sum()), 3),
                         "warm_total_incl_inference": round(float(r[:, 3].sum()), 3)},
        "permeability": {"max_rel_diff_warm_vs_plain": float(kerr.max()), "plain_mean": float(r[:, 4].mean())},
        "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None,
    }
    print(json.dumps(line), flush=True)


def run_drainage(args):
    """Drainage of the two-component porous workload as configured (400^3 GRF medium,
    porosity 0.15, corr. length 6, 8-lu buffers, wetting phase at 45 degrees through the
    calibrated virtual density, immiscible fluids): the non-wetting phase enters through
    the constant-density inlet. The same run goes once per population storage (FP32, FP16
    and BF16 deviations, FP32 compute). Every `drain_every` steps the non-wetting
    saturation S_nw (fluid nodes between the buffers where the non-wetting density exceeds
    the wetting one) is taken on the device; breakthrough is the first sample with
    non-wetting nodes in the last plane before the outlet buffer. Reported: the histories,
    MLUPS of the stepping alone (CUDA events; the samples excluded) and the 16-bit runs'
    deviation from FP32 (largest |S - S_FP32| over the samples, and the fraction of fluid
    nodes whose phase differs at the end)."""
    import torch
    from paper_2506_17713_gb300 import Lattice
    from synth import cases

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    m = 400 if args.n == 256 else args.n
    case0, init = cases.porous_two_component(shape=(m, m, m))
    solid = init["solid"]
    buf = cases.POROUS_BUFFER
    fluid = torch.from_numpy(solid == 0).cuda()
    core = fluid.clone()
    core[:, :, :buf] = False
    core[:, :, m - buf:] = False
    last = fluid[:, :, m - buf - 1]
    n_core = int(core.sum())
    K = 2
    N = m ** 3
    steps, every = args.drain_steps, args.drain_every
    runs, final = {}, {}
    for real in ("f32", "f16s", "bf16s"):
        case = dict(case0, real=real)
        if real != "f32":
            # each component's reference: the density it has in most of the domain at the start
            # (wetting: the major value, non-wetting: the dissolved one), so that most stored
            # deviations are small
            case["rho_ref"] = list(args.drain_rho_ref)
        lat = Lattice(case)
        lat.set_geometry(solid)
        for k, r in enumerate(init["rho"]):
            lat.init_fields(k, r)
        hist, bt, secs = [], None, 0.0
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        for t in range(every, steps + 1, every):
            ev0.record(lat.stream)
            lat.step(every)
            ev1.record(lat.stream)
            torch.cuda.synchronize()
            secs += ev0.elapsed_time(ev1) / 1e3
            rw, _ = lat.macroscopic(0)
            rn, _ = lat.macroscopic(1)
            nw = rn > rw
            s = float((nw & core).sum()) / n_core
            hist.append([t, round(s, 6)])
            if bt is None and bool((nw[:, :, m - buf - 1] & last).any()):
                bt = t
        m0, _ = lat.diagnostics()
        runs[real] = {"saturation": hist, "breakthrough_step": bt, "mlups": round(K * N * steps / secs / 1e6, 1),
                      "mass": [float(x) for x in m0]}
        final[real] = nw.clone()
        lat.close()
        del lat
        torch.cuda.empty_cache()
    for real in ("f16s", "bf16s"):
        ds = max(abs(a[1] - b[1]) for a, b in zip(runs[real]["saturation"], runs["f32"]["saturation"]))
        runs[real]["max_abs_saturation_diff_vs_f32"] = round(ds, 6)
        runs[real]["phase_mismatch_fraction_vs_f32"] = round(float((final[real] != final["f32"])[fluid].float().mean()), 6)
    if rank != 0:
        return
    line = {
        "metric": "two-component porous drainage: non-wetting saturation after %d steps" % steps,
        "value": runs["f32"]["saturation"][-1][1], "unit": "fraction of pore nodes", "higher_is_better": True,
        "n_gpus": world, "steps": steps, "warmup": 0, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS["drainage400"], "shape": [m, m, m], "fluid_nodes": int(fluid.sum()),
                   "core_nodes": n_core, "sample_every": every,
                   "wet_phi": case0["wet_phi"], "g12": case0["g"][0][1], "tau": case0["tau"],
                   "inlet_rho": case0["bc_rho"][0], "outlet_rho": case0["bc_rho"][1],
                   "rho_ref_16bit": list(args.drain_rho_ref)},
        "runs": runs,
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    from paper_2506_17713_gb300 import Lattice, lbm

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    case, init = make_case(args.workload, args.n)
    case["schedule"] = args.schedule
    if args.real != "f32":
        case["real"] = args.real
        if args.real in ("f16s", "bf16s"):
            rr = args.rho_ref if args.rho_ref is not None else ref_density(args.workload)
            case["rho_ref"] = [rr, rr]
    nx, ny, nz = case["shape"]
    K = int(case.get("ncomp", 1))
    N = nx * ny * nz
    lat = Lattice(case)
    if init.get("solid") is not None:
        lat.set_geometry(init["solid"])
    for k, r in enumerate(init["rho"]):
        lat.init_fields(k, r)
    stream = lat.stream

    # warm-up
    lat.step(args.warmup)
    torch.cuda.synchronize()

    # --- timed region: K steps, device time by CUDA events on the library's stream
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world, dev)
    torch.cuda.synchronize()
    n0 = lat.launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    lat.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = lat.launches() - n0
    secs = ev0.elapsed_time(ev1) / 1e3
    barrier(world, dev)
    clk = clocks.stop()
    secs_max = reduce_max(secs, world, dev)
    mlups = aggregate(K * N * args.steps, secs_max, world) / 1e6

    # --- per-kernel device time (events between the kernels of every step)
    ms, cnt = lat.profile_step(args.steps)
    fused = cnt[0] == 0
    solid = init.get("solid")
    n_fluid = int(N - np.count_nonzero(solid)) if solid is not None else N
    units = n_fluid if solid is not None and n_fluid < N else N   # nodes the two kernels process
    abytes = algorithmic_bytes(case, fused, fluid_list=units < N)
    t_col = ms[2] / max(cnt[2], 1) / 1e3
    t_den = ms[0] / max(cnt[0], 1) / 1e3
    peak, peak_kind = load_peaks()
    ach_col = abytes["collide"] * units / t_col / 1e9
    ach_den = abytes["density"] * units / t_den / 1e9 if not fused else 0.0
    step_gbs = abytes["step"] * units * args.steps / secs / 1e9

    # --- end to end through the C ABI with pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        rho_h = [torch.from_numpy(np.ascontiguousarray(r, dtype=np.float64)).pin_memory() for r in init["rho"]]
        out_t, dims = macroscopic_layout(case)
        out_t = getattr(torch, out_t)
        out_rho = torch.empty((nz, ny, nx), dtype=out_t).pin_memory()
        out_u = torch.empty((dims, nz, ny, nx), dtype=out_t).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k, r in enumerate(rho_h):
            lbm.lbm_init_fields(lat.ctx, k, r.data_ptr(), None, lbm.LBM_HOST)
        lat.step(args.e2e_steps)
        lbm.lbm_macroscopic(lat.ctx, -1 if K > 1 else 0, out_rho.data_ptr(), out_u.data_ptr(), lbm.LBM_HOST)
        mass, mom = lat.diagnostics()
        te = time.perf_counter() - t0
        te_max = reduce_max(te, world, dev)
        e2e = {"value": round(aggregate(K * N * args.e2e_steps, te_max, world) / 1e6, 1), "unit": "MLUPS",
               "h2d_bytes_per_step": int(sum(r.numel() for r in rho_h) * 8 // args.e2e_steps),
               "d2h_bytes_per_step": int((out_rho.numel() + out_u.numel()) * out_rho.element_size()
                                         // args.e2e_steps + 48 * K),
               "steps": args.e2e_steps,
               "note": "init_fields from pinned host + steps + macroscopic to pinned host + diagnostics"}

    # --- ceiling of the collide pass's access pattern: free streaming with the same gather,
    # launch shape and population traffic, no arithmetic and no psi (replaces the state)
    pattern = None
    if not fused and args.probe_steps > 0:
        t_str = lat.stream_probe(args.probe_steps) / args.probe_steps / 1e3
        sbytes = abytes["collide"] - K * (8 if case.get("real") == "f64" else 4)   # without the psi read
        ach_str = sbytes * units / t_str / 1e9
        pattern = {"kernel": "k_stream", "bytes_per_lu": sbytes, "ms_per_launch": round(t_str * 1e3, 4),
                   "achieved": round(ach_str, 1), "frac_of_peak": round(ach_str / peak, 4),
                   "collide_frac_of_pattern": round(ach_col / ach_str, 4)}

    if rank != 0:
        barrier(world, dev)
        return

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        ccase, cinit, what = case, init, "the full %dx%dx%d lattice" % (nx, ny, nz)
        if N > 256 ** 3:   # host memory: time the oracle on a 32-plane slab of the same lattice
            ccase = dict(case, shape=(nx, ny, 32))
            cinit = dict(init, rho=[r[:32] for r in init["rho"]])
            if init.get("solid") is not None:
                cinit["solid"] = init["solid"][:32]
            what = "a %dx%dx32 slab (first 32 z planes, periodic in z) of the lattice" % (nx, ny)
        cpu_mlups, cpu_dt, threads, csteps = oracle_sample(ccase, cinit, seconds=args.cpu_seconds)
        cpu = {"value": round(cpu_mlups, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": "%d FP64 oracle steps on %s (%.1f s, after one untimed step)" % (csteps, what, cpu_dt)}

    line = {
        "metric": "%s Shan-Chen MLUPS" % case["lattice"], "value": round(mlups, 1), "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * secs_max / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if case.get("real") == "f64" else "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload] if args.n == 256 else
                   WORKLOADS[args.workload].replace("256^3", "%d^3" % args.n), "shape": [nx, ny, nz], "components": K,
                   "schedule": "single-pass" if fused else (
                       "slab-overlapped two-pass" if args.schedule == "slab_overlap" else "two-pass"),
                   "parallelism": "replicas" if world > 1 else "single-gpu",
                   "fluid_nodes": n_fluid, "mflups": round(mlups * n_fluid / N, 1),
                   "storage": STORAGE[case.get("real", "f32")] + (
                       " (rho_ref %.6g)" % case["rho_ref"][0] if "rho_ref" in case else ""),
                   "l2": l2_note(case, K, N)},
        "roofline": {"bound": "hbm", "kernel": "k_fused" if fused else "k_collide", "achieved": round(ach_col, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(ach_col / peak, 4),
                     "peak_kind": peak_kind,
                     "traffic": committed_traffic("k_fused" if fused else "k_collide", args.workload, args.n,
                                                  case.get("real", "f32")),
                     "bytes_per_lu": abytes["collide"], "units_per_launch": units,
                     "ms_per_launch": round(t_col * 1e3, 4),
                     "density_kernel": {"achieved": round(ach_den, 1), "frac": round(ach_den / peak, 4),
                                        "bytes_per_lu": abytes["density"],
                                        "ms_per_launch": round(t_den * 1e3, 4)},
                     "step": {"bytes_per_lu": abytes["step"], "achieved": round(step_gbs, 1),
                              "frac": round(step_gbs / peak, 4)},
                     "access_pattern_ceiling": pattern},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        barrier(world, dev)
    lat.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pr256", choices=sorted(WORKLOADS))
    ap.add_argument("--schedule", default="auto", choices=["auto", "two_pass", "single_pass", "slab_overlap"])
    ap.add_argument("--real", default="f32", choices=["f32", "f64", "f16s", "bf16s"],
                    help="population storage (f16s / bf16s: 16-bit deviations, FP32 compute)")
    ap.add_argument("--rho-ref", type=float, default=None,
                    help="reference density of 16-bit storage (default: per workload)")
    ap.add_argument("--n", type=int, default=256, help="cube edge (256 = the benchmark workload; "
                    "smaller edges are for profiling captures)")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--probe-steps", type=int, default=50,
                    help="launches of the free-streaming probe of the collide access pattern (0: skip)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="CPU time of the oracle sample behind cpu_baseline")
    ap.add_argument("--ref-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ws-n", type=int, default=48, help="warmstart: sample edge")
    ap.add_argument("--ws-train", type=int, default=96)
    ap.add_argument("--ws-test", type=int, default=16)
    ap.add_argument("--ws-steps", type=int, default=40000,
                    help="warmstart: step limit of the training steady states")
    ap.add_argument("--ws-epochs", type=int, default=40)
    ap.add_argument("--ws-c1", type=int, default=8)
    ap.add_argument("--ws-fp32", action="store_true", help="warm-start network on FP32 CUDA cores")
    ap.add_argument("--conv-cin", type=int, default=32, help="conv3d: input channels")
    ap.add_argument("--conv-cout", type=int, default=32, help="conv3d: output channels")
    ap.add_argument("--conv-n", type=int, default=128, help="conv3d: cube edge")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-edge-lo", type=int, default=64)
    ap.add_argument("--batch-edge-hi", type=int, default=192)
    ap.add_argument("--batch-seq-steps", type=int, default=50,
                    help="steps of the sequential comparison (batch64)")
    ap.add_argument("--drain-steps", type=int, default=20000, help="drainage400: steps per storage mode")
    ap.add_argument("--drain-every", type=int, default=1000, help="drainage400: steps between saturation samples")
    ap.add_argument("--drain-rho-ref", type=float, nargs=2, default=[1.07, 0.008],
                    help="drainage400: 16-bit reference densities of the wetting and non-wetting components")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "warmstart":
        run_warmstart(args)
    elif args.workload == "warmstart_errors":
        run_warmstart_errors(args)
    elif args.workload == "conv3d":
        run_conv3d(args)
    elif args.workload == "drainage400":
        run_drainage(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
