#!/usr/bin/env python
"""Throughput of the DG residual + exact Jacobian-vector product (DOFs/s) on one GB300.

Workload (default): cubed-sphere shell 6 x 16 x 16 surface cells x 8 radial layers (12,288 hexes),
p = 4 (125 GLL nodes per element, 7,680,000 unknowns), Bates + hydrostatic base state with 1 % T
and 10 m/s seeded perturbations, rotation, radial gravity, mu ~ T^0.69, wall bottom / outflow top.
One step = one fused evaluation of r(u) and J(u) v (dg_jvp, exact mode) in FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank evaluates its own replica of the workload (independent problems, no
collective on the data path); `value` = all ranks' unknowns / max over ranks of the step time.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DG residual+Jv DOFs/s"
UNIT = "DOF/s"
CONFIG_NAME = "shell16x8_p4"
L2_BYTES = 129 * 2 ** 20


def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


HBM_PEAK_GBS = _hbm_peak()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default=CONFIG_NAME)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-worker", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--implicit", action="store_true",
                    help="time the implicit DIRK step variants instead (configs shell32x16_p2_euv, shell48x16_p3_euv)")
    ap.add_argument("--variants", default="plain_bj,mixed_bj,mixed_mlp,plain_none",
                    help="comma list for --implicit: plain_bj, mixed_bj, plain_none, mixed_mlp")
    ap.add_argument("--f32", action="store_true",
                    help="time the FP32 fused residual + exact Jv (dg_jvp_f32) instead of the FP64 one")
    ap.add_argument("--precision", action="store_true",
                    help="contraction precision study (FP32 / bf16 / fp16 and split variants) instead")
    ap.add_argument("--mlp-steps", type=int, default=2, help="plain steps whose blocks train the network")
    ap.add_argument("--mlp-epochs", type=int, default=20)
    return ap.parse_args()


# ----------------------------------------------------------------------------------------------
# oracle timing (cpu_baseline leg and --impl reference): the oracle as it stands, one thread
# ----------------------------------------------------------------------------------------------
def oracle_sample(desc, block):
    """A contiguous block of elements (panel 0, block x block cells, all layers) of the shell, or
    the first block^2 * nz elements of a box."""
    import numpy as np
    if desc.kind == 1:
        nz, n = desc.nz, desc.nx
        return np.array([k + nz * (i + n * j) for j in range(block) for i in range(block) for k in range(nz)])
    return np.arange(min(desc.n_elem, block * block * desc.nz))


def cpu_worker(config, steps, block):
    """Time the oracle's residual + Jv on a sample of elements; prints JSON (runs in a child)."""
    import numpy as np
    from oracle import dg as OD
    from oracle import mesh as OM
    from paper_2306_01085_gb300 import workloads as W
    desc = W.CONFIGS[config][0]()
    om = OM.OracleMesh(desc)
    u = W.state_for(desc, om.X, 2)
    v = W.unit_vector(102, u.shape)
    sample = oracle_sample(desc, block)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        OD.residual(om, u, None, 0.0, elems=sample)
        OD.jvp(om, u, v, 0.0, elems=sample)
        times.append(time.perf_counter() - t0)
    dof = len(sample) * 5 * om.Np
    print(json.dumps({"times": times, "dof": dof, "elements": int(len(sample))}))


def run_cpu_worker(config, steps, block):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", str(block), "--config", config,
           "--steps", str(steps)]
    res = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    if res.returncode != 0:
        raise RuntimeError(res.stderr[-2000:])
    return json.loads(res.stdout.strip().splitlines()[-1])


# ----------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------------
# FP64 work of the kernels: (2 DFMA + DMUL + DADD) per element from one ncu capture of each kernel
# (profiles/fp64_residual_jv_shell16x8_p4.md); only valid for the kernels of that capture, so the
# table is keyed by the source digest of the library it was measured on.
# ----------------------------------------------------------------------------------------------
def grad_flops_per_element(N, NC=2):
    """FP64 flops of the sum-factorised LDG gradient (k_grad) per element, counted from the
    algorithm (an FMA is 2 flops): per component c, at each of the N^3 Gauss points G u (9),
    the lifting sum over 6 faces and 3 directions (36), the weak derivative D^T over 3 axes and 3
    directions (18 N) and the 1/(w |J|) scaling (3); at each of the 6 N^2 face points the trace
    average (2), (w n dS) u_hat (3) and the extrapolation of the 3 new gradient components (6 N)."""
    NP, NF = N ** 3, N ** 2
    return 5 * NC * (NP * (48 + 18 * N) + 6 * NF * (5 + 6 * N))


# FP64 flops per element: k_grad from the algorithm; k_volume and k_faces (pointwise physics
# dominated) as executed, (2 DFMA + DMUL + DADD) thread instructions of the ncu capture of the
# residual kernels whose source digest is CAPTURE_DIGEST (profiles/fp64_residual_jv_shell16x8_p4.md)
FP64_FLOPS_PER_ELEMENT = {("k_grad", 5): float(grad_flops_per_element(5)), ("k_volume", 5): 210000.0,
                          ("k_faces", 5): 85028.1}
FLOPS_KIND = {"k_grad": "algorithmic (sum-factorisation count)", "k_volume": "executed (ncu instruction counts)",
              "k_faces": "executed (ncu instruction counts)"}
DRAM_BYTES_PER_LAUNCH = {("k_grad", 5): 1206108672.0, ("k_volume", 5): 912022272.0, ("k_faces", 5): 755261952.0}
CAPTURE_DIGEST = "a3a5ace70bb03005accaf9eafe37c37425512c87388f0f7d4384474e5ccbcaba"
RESIDUAL_SOURCES = ("dg_kernels.cuh", "dg_internal.cuh", "dg_map.cuh", "dg_kernels_n5.cu")


def residual_kernel_digest():
    """sha256 of the sources of the p = 4 residual kernels and the compile flags."""
    import hashlib
    from paper_2306_01085_gb300 import build as B
    h = hashlib.sha256()
    for f in RESIDUAL_SOURCES:
        with open(os.path.join(B.CSRC, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    h.update(" ".join(B.ARCH + B.FLAGS).encode())
    return h.hexdigest()


# FP64 peak from unit counts: 2 DFMA lanes/SM/cycle x 152 SMs x 2 flops x 2.07 GHz
FP64_PEAK_TFLOPS = 2 * 152 * 2 * 2.07e9 / 1e12


def rank_aggregate(ms, n_dof, world, device="cuda"):
    """Max over ranks of a per-step time and the whole-job throughput. Every rank evaluates its own
    replica of n_dof unknowns (no collective on the data path), so value = world * n_dof / max."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * n_dof / (ms_max * 1e-3)


def main_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2306_01085_gb300 import build as B
    from paper_2306_01085_gb300 import dg as DG
    from paper_2306_01085_gb300 import workloads as W

    B.build()
    desc = W.CONFIGS[args.config][0]()
    mesh = DG.Mesh(desc)
    x = mesh.nodes().cpu().numpy()
    u = W.state_for(desc, x, 2 + rank)
    v = W.unit_vector(102 + rank, u.shape)
    ug = torch.from_numpy(u).cuda()
    vg = torch.from_numpy(v).cuda()
    r = torch.empty_like(ug)
    jv = torch.empty_like(ug)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        if args.f32:
            mesh.jvp_f32(ug, vg, t=0.0, out=jv, r_out=r)
        else:
            mesh.jvp(ug, vg, t=0.0, out=jv, r_out=r)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if not (torch.isfinite(r).all() and torch.isfinite(jv).all()):
        raise RuntimeError("non-finite residual or Jv")

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    mesh.profile_start(capacity=64 * args.steps + 64)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)                 # write 2x L2 between steps (outside the events)
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    prof, launches = mesh.profile_stop()
    clk = clocks.stop()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms_mean = sum(ms) / len(ms)
    ms_max, value = rank_aggregate(ms_mean, mesh.n_dof, world)

    # dominant kernel and its FP64 roofline
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_cnt) = dom
    per_launch_ms = dom_ms / dom_cnt
    key = (dom_name, desc.p + 1)
    fpe = None if args.f32 else FP64_FLOPS_PER_ELEMENT.get(key)
    flops = fpe * mesh.n_elem if fpe else None
    achieved = flops / (per_launch_ms * 1e-3) / 1e12 if flops else None
    probe = DG.probe_fp64()
    fresh = residual_kernel_digest() == CAPTURE_DIGEST
    traffic = DRAM_BYTES_PER_LAUNCH.get(key) if (args.config == CONFIG_NAME and fresh and not args.f32) else None
    roofline = {"bound": "alu", "kernel": dom_name, "achieved": round(achieved, 4) if achieved else None,
                "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                "frac": round(achieved / FP64_PEAK_TFLOPS, 4) if achieved else None, "traffic": traffic,
                "peak_kind": "FP64 from unit counts x max SM clock (2 DFMA/SM/cycle, 152 SMs, 2.07 GHz)",
                "flops_kind": FLOPS_KIND.get(dom_name),
                "peak_probe": round(probe, 4), "launch_ms": round(per_launch_ms, 4), "fp64_flops_per_launch": flops,
                "share": round(dom_ms / sum(v[0] for v in prof.values()), 4),
                "counters": "ncu capture of these kernel sources" if fresh else "ncu capture of earlier kernel sources (flops as then)",
                "dram_gbs": round(traffic / (per_launch_ms * 1e-3) / 1e9, 1) if traffic else None}

    # the whole step against HBM: the two-pass minimum of 144 B/DOF (u, v in; q, q_dot out; u, q,
    # v, q_dot in; r, Jv out)
    roofline["hbm_context"] = {"bytes_per_dof": 144, "achieved_gbs": round(144 * mesh.n_dof / (ms_max * 1e-3) / 1e9, 1),
                               "peak_gbs": HBM_PEAK_GBS, "frac": round(144 * mesh.n_dof / (ms_max * 1e-3) / 1e9 / HBM_PEAK_GBS, 4)}

    # end to end through the public API: every step copies its inputs from pinned host memory and
    # its results back to pinned host memory. The copies run on their own streams with two device
    # buffer sets, so step k + 1's inputs and step k - 1's results move while step k computes.
    e2e = None
    if not args.no_e2e:
        uh = torch.from_numpy(u).pin_memory()
        vh = torch.from_numpy(v).pin_memory()
        rh = [torch.empty_like(uh).pin_memory() for _ in range(2)]
        jh = [torch.empty_like(uh).pin_memory() for _ in range(2)]
        ud, vd = [ug, torch.empty_like(ug)], [vg, torch.empty_like(vg)]
        rd, jd = [r, torch.empty_like(r)], [jv, torch.empty_like(jv)]
        h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()

        def pipelined(n_steps, start=None):
            """n_steps steps; start (an event on the compute stream) gates the first copy."""
            h2d_done = [torch.cuda.Event() for _ in range(2)]
            comp_done = [torch.cuda.Event() for _ in range(2)]
            d2h_done = [torch.cuda.Event() for _ in range(2)]

            def load(k):
                b = k % 2
                if start is not None:
                    h2d.wait_event(start)
                if k >= 2:
                    h2d.wait_event(comp_done[b])       # step k - 2 has read this buffer set
                with torch.cuda.stream(h2d):
                    ud[b].copy_(uh, non_blocking=True)
                    vd[b].copy_(vh, non_blocking=True)
                h2d_done[b].record(h2d)

            load(0)
            for k in range(n_steps):
                b = k % 2
                if k + 1 < n_steps:
                    load(k + 1)
                stream.wait_event(h2d_done[b])
                if k >= 2:
                    stream.wait_event(d2h_done[b])     # step k - 2's results have left this set
                if args.f32:
                    mesh.jvp_f32(ud[b], vd[b], t=0.0, out=jd[b], r_out=rd[b])
                else:
                    mesh.jvp(ud[b], vd[b], t=0.0, out=jd[b], r_out=rd[b])
                comp_done[b].record(stream)
                d2h.wait_event(comp_done[b])
                with torch.cuda.stream(d2h):
                    rh[b].copy_(rd[b], non_blocking=True)
                    jh[b].copy_(jd[b], non_blocking=True)
                d2h_done[b].record(d2h)
            stream.wait_stream(d2h)

        pipelined(args.warmup)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        pipelined(args.steps, start=ev0)
        ev1.record(stream)
        torch.cuda.synchronize()
        if not (torch.isfinite(rh[(args.steps - 1) % 2]).all() and torch.isfinite(jh[(args.steps - 1) % 2]).all()):
            raise RuntimeError("non-finite end-to-end result")
        e2e_ms = ev0.elapsed_time(ev1) / args.steps
        _, e2e_value = rank_aggregate(e2e_ms, mesh.n_dof, world)
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": 2 * 8 * mesh.n_dof, "d2h_bytes_per_step": 2 * 8 * mesh.n_dof}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res = run_cpu_worker(args.config, 1, 4)
        cpu = {"value": res["dof"] / min(res["times"]), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"residual + complex-step Jv of {res['elements']} contiguous elements "
                         f"({res['dof']} DOF; panel 0, 4x4 cells, all layers) of the same shell, one thread"}

    if world > 1:
        dist.barrier()
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32" if args.f32 else "f64", "data": "synthetic",
               "config": {"workload": f"{args.config}: {W.CONFIGS[args.config][1]}", "n_elem": mesh.n_elem,
                          "p": desc.p, "n_dof": mesh.n_dof, "step": "fused residual + exact Jv (dg_jvp_f32)" if args.f32 else "fused residual + exact Jv (dg_jvp)",
                          "l2": "2x L2 buffer written between timed steps", "parallelism": f"replicas x{world}"},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
               "kernels": {k: {"ms": round(v[0], 4), "launches": v[1]} for k, v in prof.items()},
               "clocks": clk, "wall_s_timed": round(wall, 4)}
        print(json.dumps(out), flush=True)
    mesh.close()
    if world > 1:
        dist.destroy_process_group()


def main_reference(args):
    """The oracle (this repository's CPU reference of the method) on the same workload, one thread."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sys.path.insert(0, ROOT)
    from paper_2306_01085_gb300 import workloads as W
    res = run_cpu_worker(args.config, args.warmup + args.steps, 2)
    times = res["times"][args.warmup:] or res["times"]
    ms = 1e3 * sum(times) / len(times)
    value = res["dof"] / (ms * 1e-3)
    sample = (f"residual + complex-step Jv of {res['elements']} contiguous elements ({res['dof']} DOF) of the "
              f"same shell per step, one thread")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{args.config}: {W.CONFIGS[args.config][1]}"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main_implicit(args):
    """Wall time per implicit DIRK(3,3) step of 60 s for the solver variants (1 GPU).

    plain_bj:   FP64 residual and exact FP64 Jv, block-Jacobi on exact blocks (FP32 LU)
    mixed_bj:   FP64 residual, FP32 inner Jv and FP32-assembled blocks (FP32 LU)
    plain_none: FP64 unpreconditioned GMRES(30)
    mixed_mlp:  mixed precision with the learned diagonal + low-rank preconditioner, trained first on
                the exact blocks of --mlp-steps plain steps (training time reported separately)
    mixed_rb_bj: mixed precision, the reduced basis of the last 8 Newton updates (Sec. 3.2) over
                block-Jacobi, with the RB initial guess
    mixed_rb:   mixed precision, the reduced basis over the mass matrix (nothing assembled)
    mixed_bj16: mixed_bj with the inverses stored as FP16 (power-of-two column scales)
    Every variant starts from the same state; the final states are compared with plain_bj.
    """
    import numpy as np
    import torch
    from paper_2306_01085_gb300 import build as B
    from paper_2306_01085_gb300 import dg as DG
    from paper_2306_01085_gb300 import workloads as W

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    B.build()
    config = args.config if args.config != CONFIG_NAME else "shell32x16_p2_euv"
    desc = W.CONFIGS[config][0]()
    mesh = DG.Mesh(desc)
    u0 = torch.from_numpy(W.state_for(desc, mesh.nodes().cpu().numpy(), 2)).cuda()
    dt = 60.0 / W.shell_reference().t0
    variants = {
        "plain_bj": dict(precond="bj", jv_prec="f64"),
        "mixed_bj": dict(precond="bj", jv_prec="f32"),
        "plain_none": dict(precond="none", jv_prec="f64"),
    }
    variants["mixed_mlp"] = dict(precond="mlp", jv_prec="f32")
    variants["mixed_rb_bj"] = dict(precond="rb_bj", jv_prec="f32")
    variants["mixed_rb"] = dict(precond="rb", jv_prec="f32")
    variants["mixed_bj16"] = dict(precond="bj16", jv_prec="f32")
    results, finals = {}, {}
    training = None
    if "mixed_mlp" in args.variants.split(","):
        # harvest exact blocks from plain steps (each step's initial state, coefficient dt a_ii),
        # then train the network with the library's own kernels
        gamma = float(DG.dirk_tableau(3)[0][0, 0])
        n_harvest = max(1, args.mlp_steps)
        mesh.mlp_init(hidden=256, rank=16, max_samples=n_harvest * mesh.n_elem, seed=11)
        u = u0.clone()
        t_h = time.perf_counter()
        for k in range(n_harvest):
            mesh.mlp_harvest(u, k * dt, dt * gamma, stride=1)
            mesh.implicit_step(u, k * dt, dt, stages=3, precond="bj", jv_prec="f32")
        t_h = time.perf_counter() - t_h
        torch.cuda.synchronize()
        t_t = time.perf_counter()
        first, last = mesh.mlp_train(epochs=args.mlp_epochs, batch=1024, lr=1e-3)
        torch.cuda.synchronize()
        training = {"samples": mesh.mlp_sizes()["n_samples"], "harvest_steps": n_harvest,
                    "harvest_s": round(t_h, 2), "train_s": round(time.perf_counter() - t_t, 2),
                    "epochs": args.mlp_epochs, "loss_first_epoch": first, "loss_last_epoch": last,
                    "params": mesh.mlp_sizes()["n_params"]}
    for name in args.variants.split(","):
        kw = variants[name]
        u = u0.clone()
        mesh.rb_reset()
        steps = []
        rc = 0
        kernels = None
        for k in range(args.steps):
            last = k == args.steps - 1
            if last:
                mesh.profile_start(capacity=200000)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = mesh.implicit_step(u, k * dt, dt, stages=3, check=False, **kw)
            torch.cuda.synchronize()
            st["wall_s"] = time.perf_counter() - t0
            if last:
                prof, _ = mesh.profile_stop()
                kernels = {kn: {"ms": round(v[0], 2), "launches": v[1]} for kn, v in prof.items()}
            steps.append(st)
            rc = st["rc"]
            if rc != 0:
                break
        finals[name] = u.cpu().numpy() if rc == 0 else None
        newton = [sum(st["newton"]) for st in steps]
        gmres = [sum(st["gmres"]) for st in steps]
        results[name] = {"rc": rc, "steps_done": sum(1 for st in steps if st["rc"] == 0),
                         "wall_s_per_step": [round(st["wall_s"], 4) for st in steps],
                         "precond_s_per_step": [round(st["precond_ms"] / 1e3, 4) for st in steps],
                         "newton_per_step": newton, "gmres_per_step": gmres,
                         "gmres_per_newton": round(sum(gmres) / max(1, sum(newton)), 2),
                         "kernels_last_step": kernels}
    ref = finals.get("plain_bj")
    if ref is not None:
        du = np.abs(ref - u0.cpu().numpy()).max(axis=(0, 2))
        for name, fin in finals.items():
            if fin is not None and name != "plain_bj":
                results[name]["final_diff_rel_to_change"] = (np.abs(fin - ref).max(axis=(0, 2)) / du).tolist()
    base = results.get("plain_bj", {}).get("wall_s_per_step")
    out = {"metric": "implicit DIRK(3,3) step wall time at Newton 1e-8", "unit": "s/step", "config": config,
           "n_elem": mesh.n_elem, "n_dof": mesh.n_dof, "dt_s": 60.0, "steps": args.steps, "variants": results,
           "mlp_training": training}
    for name in ("mixed_bj", "mixed_mlp", "mixed_rb_bj", "mixed_rb"):
        if base and results.get(name, {}).get("rc") == 0:
            out[f"speedup_{name}_vs_plain_bj"] = round(np.mean(base) / np.mean(results[name]["wall_s_per_step"]), 3)
    print(json.dumps(out), flush=True)
    mesh.close()


def main_precision(args):
    """Precision study of the basis contractions on one GPU: the fused residual + exact Jv with the
    contractions in FP32, bfloat16 and binary16 operands (FP32 accumulation), and their hi + lo
    three-product splits, each timed (2x L2 written between steps) and compared per variable with
    the FP64 path on the same input (the FP64 path itself agrees with the oracle to 1e-12)."""
    import numpy as np
    import torch
    from paper_2306_01085_gb300 import build as B
    from paper_2306_01085_gb300 import dg as DG
    from paper_2306_01085_gb300 import workloads as W

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    B.build()
    config = args.config if args.config != CONFIG_NAME else "shell32x16_p2_euv"
    desc = W.CONFIGS[config][0]()
    mesh = DG.Mesh(desc)
    u = W.state_for(desc, mesh.nodes().cpu().numpy(), 2)
    v = W.unit_vector(102, u.shape)
    ug = torch.from_numpy(u).cuda()
    vg = torch.from_numpy(v).cuda()
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    r64, j64 = mesh.empty(), mesh.empty()
    mesh.jvp(ug, vg, t=0.0, out=j64, r_out=r64)
    ref_r = np.moveaxis(r64.cpu().numpy(), 1, 0).reshape(5, -1)
    ref_j = np.moveaxis(j64.cpu().numpy(), 1, 0).reshape(5, -1)
    r, jv = mesh.empty(), mesh.empty()
    modes = {"fp64": lambda: mesh.jvp(ug, vg, t=0.0, out=jv, r_out=r)}
    for name in DG.CM:
        modes[name] = (lambda nm: lambda: mesh.eval_precision(nm, ug, vg, t=0.0, r=r, jv=jv))(name)
    out = {"metric": "fused residual + Jv DOFs/s and relative error per variable by contraction precision",
           "config": config, "n_elem": mesh.n_elem, "n_dof": mesh.n_dof, "steps": args.steps,
           "reference": "FP64 path on the same input", "modes": {}}
    clocks = ClockSampler(0)
    clocks.start()
    for name, fn in modes.items():
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            fn()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        gr = np.moveaxis(r.cpu().numpy(), 1, 0).reshape(5, -1)
        gj = np.moveaxis(jv.cpu().numpy(), 1, 0).reshape(5, -1)
        with np.errstate(invalid="ignore"):
            er = (np.abs(gr - ref_r).max(1) / np.abs(ref_r).max(1)).tolist()
            ej = (np.abs(gj - ref_j).max(1) / np.abs(ref_j).max(1)).tolist()
        out["modes"][name] = {"ms": round(ms, 4), "dof_per_s": mesh.n_dof / (ms * 1e-3),
                              "rel_err_r": [float(f"{x:.3e}") for x in er],
                              "rel_err_jv": [float(f"{x:.3e}") for x in ej]}
    out["clocks"] = clocks.stop()
    print(json.dumps(out), flush=True)
    mesh.close()


if __name__ == "__main__":
    a = parse()
    if a.implicit:
        main_implicit(a)
        sys.exit(0)
    if a.precision:
        main_precision(a)
        sys.exit(0)
    if a.cpu_worker:
        cpu_worker(a.config, a.steps, a.cpu_worker)
    elif a.impl == "reference":
        main_reference(a)
    else:
        main_ours(a)
