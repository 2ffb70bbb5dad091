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
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default=CONFIG_NAME)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--interp", choices=["fp64", "tc"], default="fp64",
                    help="nodes -> Gauss values step: FP64 sum-factorised passes, or the tensor-core "
                         "contraction with FP64-accurate digit slicing")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-implicit", action="store_true", help="leave the implicit-step comparison off the line")
    ap.add_argument("--no-radial", action="store_true", help="leave the radial 1D ensemble off the line")
    ap.add_argument("--radial", action="store_true", help="time the radial 1D ensemble alone")
    ap.add_argument("--radial-columns", type=int, default=16384)
    ap.add_argument("--implicit-config", default="shell32x16_p2_euv")
    ap.add_argument("--implicit-chosen", default="mixed_bj16")
    ap.add_argument("--implicit-steps", type=int, default=3)
    ap.add_argument("--dt", type=float, default=60.0, help="--implicit: the DIRK step in seconds")
    ap.add_argument("--cpu-worker", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-procs", type=int, default=1, help=argparse.SUPPRESS)
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
# oracle timing (cpu_baseline leg and --impl reference): the oracle as it stands, on one thread and
# on every host core (the sample's elements split across processes)
# ----------------------------------------------------------------------------------------------
SAMPLE_BLOCK = 4   # panel 0, 4 x 4 angular cells, all layers: 128 elements of the 12,288-element shell


def oracle_sample(desc, block):
    """A contiguous block of elements (panel 0, block x block cells, all layers) of the shell, or
    the first block^2 * nz elements of a box."""
    import numpy as np
    if desc.kind == 1:
        nz, n = desc.nz, desc.nx
        return np.array([k + nz * (i + n * j) for j in range(block) for i in range(block) for k in range(nz)])
    return np.arange(min(desc.n_elem, block * block * desc.nz))


def cpu_model():
    """The host CPU's model name and its core count."""
    name = None
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu model"):
                    name = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not name:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.split(":")[0].strip() in ("Model name", "Vendor ID"):
                    name = ln.split(":", 1)[1].strip()
                    if ln.startswith("Model name"):
                        break
        except (OSError, subprocess.SubprocessError):
            pass
    return name or "unknown", os.cpu_count() or 1


_W = {}


def _worker_init(config):
    from oracle import mesh as OM
    from paper_2306_01085_gb300 import workloads as W
    desc = W.CONFIGS[config][0]()
    om = OM.OracleMesh(desc)
    _W.update(om=om, u=W.state_for(desc, om.X, 2), v=W.unit_vector(102, (desc.n_elem, 5, om.Np)))


def _worker_chunk(elems):
    from oracle import dg as OD
    OD.residual(_W["om"], _W["u"], None, 0.0, elems=elems)
    OD.jvp(_W["om"], _W["u"], _W["v"], 0.0, elems=elems)
    return len(elems)


def cpu_worker(config, steps, block, procs):
    """Time the oracle's residual + Jv on a sample of elements with `procs` processes (forked after
    the mesh is built; this process never touches a GPU); prints JSON (runs in a child)."""
    import multiprocessing as mp
    import numpy as np
    _worker_init(config)
    desc_n = _W["om"].desc
    sample = oracle_sample(desc_n, block)
    chunks = [c for c in np.array_split(sample, procs) if len(c)]
    times = []
    if procs == 1:
        for _ in range(steps):
            t0 = time.perf_counter()
            _worker_chunk(sample)
            times.append(time.perf_counter() - t0)
    else:
        with mp.get_context("fork").Pool(procs) as pool:
            pool.map(_worker_chunk, chunks)              # warm the workers
            for _ in range(steps):
                t0 = time.perf_counter()
                pool.map(_worker_chunk, chunks)
                times.append(time.perf_counter() - t0)
    dof = len(sample) * 5 * _W["om"].Np
    print(json.dumps({"times": times, "dof": dof, "elements": int(len(sample)), "procs": procs}))


def run_cpu_worker(config, steps, block, procs=1):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", str(block), "--cpu-procs", str(procs),
           "--config", config, "--steps", str(steps)]
    res = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    if res.returncode != 0:
        raise RuntimeError(res.stderr[-2000:])
    return json.loads(res.stdout.strip().splitlines()[-1])


def cpu_baseline_leg(config, steps=2):
    """The oracle on the same element sample on one thread and on every core: both values, the
    cores used and the CPU model."""
    model, ncpu = cpu_model()
    one = run_cpu_worker(config, steps, SAMPLE_BLOCK, 1)
    allc = run_cpu_worker(config, steps, SAMPLE_BLOCK, ncpu) if ncpu > 1 else one
    v1 = one["dof"] / min(one["times"])
    vn = allc["dof"] / min(allc["times"])
    sample = (f"residual + complex-step Jv of {one['elements']} contiguous elements ({one['dof']} DOF; panel 0, "
              f"{SAMPLE_BLOCK}x{SAMPLE_BLOCK} cells, all layers) of the same shell per step, best of {steps}")
    return {"value": vn, "unit": UNIT, "cores": allc["procs"], "kind": "oracle", "sample": sample,
            "one_thread": {"value": v1, "cores": 1}, "all_cores": {"value": vn, "cores": allc["procs"]},
            "cpu_model": model, "nproc": ncpu}


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
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark(self):
        """Index of the next sample (to summarise a part of the loaded window)."""
        return len(self.lines)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.proc = None
        return self.summary()

    def summary(self, start=0, end=None):
        """Median SM clock, max clock and throttle reasons of the samples [start, end)."""
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[start:end]:
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
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm),
                "interval_ms": 50}


# ----------------------------------------------------------------------------------------------
# algorithmic work of the step's kernels
# ----------------------------------------------------------------------------------------------
# HBM bytes of the method per unknown for one fused residual + exact Jv in two passes, geometry
# recomputed: pass 1 reads u, v and writes q, q_dot (8 + 8 + 24 + 24 B); pass 2 reads u, q, v, q_dot
# and writes r, Jv (64 + 16 B).
ALGO_BYTES_PER_DOF = 144

# FP64 flops (value, exact tangent) of the pointwise physics of the shell16x8_p4 workload (mu, kappa
# ~ T^0.69, no heating), counted on the oracle's own expressions with shared primitives:
# tests/test_flop_counts.py recomputes these numbers. Transcendental calls (exp, pow) are listed
# apart and not converted to flops.
PHYS_FLOPS = {"volume_point": (262, 480), "face_interior": (437, 721), "face_wall": (225, 376),
              "face_outflow": (143, 229)}
PHYS_TRANSCENDENTALS = {"volume_point": 3, "face_interior": 8, "face_wall": 6, "face_outflow": 3}


def grad_flops_per_element(N, NC=2):
    """FP64 flops of the sum-factorised LDG gradient (k_grad) per element, counted from the
    algorithm (an FMA is 2 flops): per component c, at each of the N^3 Gauss points G u (9),
    the lifting sum over 6 faces and 3 directions (36), the weak derivative D^T over 3 axes and 3
    directions (18 N) and the 1/(w |J|) scaling (3); at each of the 6 N^2 face points the trace
    average (2), (w n dS) u_hat (3) and the extrapolation of the 3 new gradient components (6 N)."""
    NP, NF = N ** 3, N ** 2
    return 5 * NC * (NP * (48 + 18 * N) + 6 * NF * (5 + 6 * N))


def kernel_flops(N, n_elem, n_interior, n_wall, n_outflow):
    """Algorithmic FP64 flops per launch of each kernel of the fused residual + exact Jv (value and
    tangent planes):
      k_interp  3 passes of N-point contractions per Gauss point and one per face point, 5 variables;
      k_grad    grad_flops_per_element;
      k_volume  pointwise flux and source, plus per plane and Gauss point the reference fluxes
                (15 x 3 FMA = 90), the source weighting (5), the weak derivative (5 x 3 x N FMA),
                the face lifting (5 x 6 FMA = 60) and the projection B^T (5 x 3 x N FMA);
      k_faces   the numerical flux of Eq. LDG2 per interior, wall and outflow face point."""
    NP, NF = N ** 3, N ** 2
    interp = 2 * 5 * (NP * 3 * 2 * N + 6 * NF * 2 * N)
    volume = NP * (sum(PHYS_FLOPS["volume_point"]) + 2 * (155 + 60 * N))
    faces = NF * (n_interior * sum(PHYS_FLOPS["face_interior"]) + n_wall * sum(PHYS_FLOPS["face_wall"])
                  + n_outflow * sum(PHYS_FLOPS["face_outflow"]))
    return {"k_interp": interp * n_elem, "k_grad": grad_flops_per_element(N) * n_elem,
            "k_volume": volume * n_elem, "k_faces": faces}


def face_kinds(desc):
    """(interior, wall, outflow) faces of a workload mesh: 6 face slots per element, each interior
    face shared by two elements; shells have 6 nx^2 faces on each sphere, boxes nx ny on each z end
    unless z is periodic."""
    E = desc.n_elem
    nb = 6 * desc.nx * desc.nx if desc.kind == 1 else (desc.nx * desc.ny if desc.bc_lo else 0)
    kinds = {0: 0, 1: 0, 2: 0}
    if nb:
        kinds[desc.bc_lo] += nb
        kinds[desc.bc_hi] += nb
    return 3 * E - nb, kinds[1], kinds[2]


# DRAM bytes per launch of each kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the kernel sources whose digest is CAPTURE_DIGEST; on other sources the
# traffic is reported as null.
DRAM_BYTES_PER_LAUNCH = {"k_interp": 332595968.0, "k_grad": 1202171392.0, "k_faces": 752034816.0,
                         "k_volume": 909457664.0}
CAPTURE_DIGEST = "966fdfbcd34bba688dffe5843a34eba029307f0500bcd0fc3921510afc235bbf"
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


def roofline_of(mesh, desc, config, prof, ms_step, f32, interp="fp64"):
    """The step against the HBM roofline (the method's 144 B per unknown), with each kernel's
    algorithmic FP64 work against the FP64 peak beside it (the tensor-core interpolation does no
    FP64 arithmetic and is left out of that list)."""
    achieved = ALGO_BYTES_PER_DOF * mesh.n_dof / (ms_step * 1e-3) / 1e9
    fresh = (not f32 and interp == "fp64" and config == CONFIG_NAME and CAPTURE_DIGEST is not None
             and residual_kernel_digest() == CAPTURE_DIGEST)
    traffic = sum(DRAM_BYTES_PER_LAUNCH.values()) if fresh and DRAM_BYTES_PER_LAUNCH else None
    total_ms = sum(v[0] for v in prof.values())
    dom_name, (dom_ms, dom_cnt) = max(prof.items(), key=lambda kv: kv[1][0])
    out = {"bound": "hbm", "scope": "the fused residual + exact Jv step (k_interp, k_grad, k_faces, k_volume)",
           "achieved": round(achieved, 2), "peak": HBM_PEAK_GBS, "unit": "GB/s", "frac": round(achieved / HBM_PEAK_GBS, 5),
           "peak_kind": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
           "bytes_per_dof": ALGO_BYTES_PER_DOF, "traffic": traffic,
           "traffic_kind": "DRAM bytes per step, ncu dram__bytes_read.sum + dram__bytes_write.sum of these sources"
           if traffic else None,
           "dominant_kernel": {"name": dom_name, "launch_ms": round(dom_ms / dom_cnt, 4),
                               "share": round(dom_ms / total_ms, 4)}}
    if f32 or config != CONFIG_NAME:
        return out
    n_int, n_wall, n_out = face_kinds(desc)
    flops = kernel_flops(desc.p + 1, mesh.n_elem, n_int, n_wall, n_out)
    fp64 = {}
    for k, fl in flops.items():
        if k in prof and not (interp == "tc" and k == "k_interp"):
            ms_launch = prof[k][0] / prof[k][1]
            tf = fl / (ms_launch * 1e-3) / 1e12
            fp64[k] = {"flops_per_launch": fl, "launch_ms": round(ms_launch, 4), "tflops": round(tf, 4),
                       "frac": round(tf / FP64_PEAK_TFLOPS, 4)}
    step_flops = sum(flops.values())
    out["fp64"] = {"peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                   "peak_kind": "FP64 from unit counts x max SM clock (2 DFMA/SM/cycle, 152 SMs, 2.07 GHz)",
                   "peak_probe": round(float(__import__("paper_2306_01085_gb300.dg", fromlist=["x"]).probe_fp64()), 4),
                   "flops_kind": "algorithmic: the oracle's pointwise expressions counted on an operation-"
                                 "counting scalar (value + forward-mode tangent), transcendental calls not "
                                 "included; sum-factorised contractions counted from the algorithm",
                   "step_flops": step_flops, "step_tflops": round(step_flops / (ms_step * 1e-3) / 1e12, 4),
                   "step_frac": round(step_flops / (ms_step * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, 4),
                   "kernels": fp64}
    return out


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
    mesh.set_interp(args.interp)
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

    # clocks sampled every 50 ms over the whole loaded window (warm-up, timed steps, end-to-end leg
    # and the implicit steps)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if not (torch.isfinite(r).all() and torch.isfinite(jv).all()):
        raise RuntimeError("non-finite residual or Jv")

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    mesh.profile_start(capacity=64 * args.steps + 64)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    mark0 = clocks.mark()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)                 # write 2x L2 between steps (outside the events)
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    mark1 = clocks.mark()
    if world > 1:
        dist.barrier()
    prof, launches = mesh.profile_stop()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms_mean = sum(ms) / len(ms)
    ms_max, value = rank_aggregate(ms_mean, mesh.n_dof, world)
    roofline = roofline_of(mesh, desc, args.config, prof, ms_max, args.f32, args.interp)

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
    mesh.close()
    del flush

    # the radial 1D ensemble (Sec. 4.3)
    radial = None
    if not args.no_radial and not args.f32:
        radial = radial_leg(clocks=clocks)

    # the implicit-step half of the metric: plain FP64 against the chosen mixed-precision variant
    implicit = None
    if not args.no_implicit and not args.f32:
        names = ["plain_bj", args.implicit_chosen]
        if args.implicit_chosen == "mixed_bj16":
            names.append("mixed_bj16_lag3")   # the chosen variant with its preconditioner built every 3 steps
        implicit = implicit_variants(args.implicit_config, names, args.implicit_steps, clocks=clocks)
        implicit = implicit_summary(implicit, args.implicit_chosen)
    clk_all = clocks.stop()
    clk_timed = clocks.summary(mark0, mark1)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(args.config)

    if world > 1:
        dist.barrier()
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32" if args.f32 else "f64", "data": "synthetic",
               "config": {"workload": f"{args.config}: {W.CONFIGS[args.config][1]}", "n_elem": mesh.n_elem,
                          "p": desc.p, "n_dof": mesh.n_dof, "step": "fused residual + exact Jv (dg_jvp_f32)" if args.f32 else "fused residual + exact Jv (dg_jvp)",
                          "l2": "2x L2 buffer written between timed steps", "parallelism": f"replicas x{world}",
                          "interp": "FP64 sum-factorised passes" if args.interp == "fp64" else
                          "tensor cores (tcgen05, FP16 digits, FP64-accurate)"},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
               "kernels": {k: {"ms": round(v[0], 4), "launches": v[1]} for k, v in prof.items()},
               "clocks": clk_timed, "clocks_loaded_window": clk_all, "wall_s_timed": round(wall, 4),
               "implicit": implicit, "radial": radial}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main_reference(args):
    """The oracle (this repository's CPU statement of the method) on the same workload: the element
    sample of the cpu_baseline leg, split across every host core."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sys.path.insert(0, ROOT)
    from paper_2306_01085_gb300 import workloads as W
    model, ncpu = cpu_model()
    res = run_cpu_worker(args.config, args.warmup + args.steps, SAMPLE_BLOCK, ncpu)
    times = res["times"][args.warmup:] or res["times"]
    ms = 1e3 * sum(times) / len(times)
    value = res["dof"] / (ms * 1e-3)
    sample = (f"residual + complex-step Jv of {res['elements']} contiguous elements ({res['dof']} DOF; panel 0, "
              f"{SAMPLE_BLOCK}x{SAMPLE_BLOCK} cells, all layers) of the same shell per step, split across "
              f"{res['procs']} processes")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{args.config}: {W.CONFIGS[args.config][1]}"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": res["procs"], "kind": "oracle", "sample": sample,
                            "cpu_model": model, "nproc": ncpu},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


IMPLICIT_VARIANTS = {
    "plain_bj": dict(precond="bj", jv_prec="f64"),
    "mixed_bj": dict(precond="bj", jv_prec="f32"),
    "plain_none": dict(precond="none", jv_prec="f64"),
    "mixed_mlp": dict(precond="mlp", jv_prec="f32"),
    "mixed_rb_bj": dict(precond="rb_bj", jv_prec="f32"),
    "mixed_rb": dict(precond="rb", jv_prec="f32"),
    "mixed_bj16": dict(precond="bj16", jv_prec="f32"),
    # the same with the preconditioner built once every 3 steps (lagged)
    "mixed_bj16_lag3": dict(precond="bj16", jv_prec="f32", precond_refresh="lagged", refresh_every=3),
}


def implicit_variants(config, names, n_steps, clocks=None, mlp_steps=2, mlp_epochs=20, dt_s=60.0):
    """Wall time per implicit DIRK(3,3) step of dt_s seconds for the solver variants (1 GPU), every variant
    from the same state; final states compared with plain_bj. With clocks (a running ClockSampler)
    each variant's steps get their own clock summary."""
    import numpy as np
    import torch
    from paper_2306_01085_gb300 import build as B
    from paper_2306_01085_gb300 import dg as DG
    from paper_2306_01085_gb300 import workloads as W

    B.build()
    desc = W.CONFIGS[config][0]()
    mesh = DG.Mesh(desc)
    u0 = torch.from_numpy(W.state_for(desc, mesh.nodes().cpu().numpy(), 2)).cuda()
    dt = dt_s / W.shell_reference().t0
    results, finals = {}, {}
    training = None
    if "mixed_mlp" in names:
        # harvest exact blocks from plain steps (each step's initial state, coefficient dt a_ii),
        # then train the network with the library's own kernels
        gamma = float(DG.dirk_tableau(3)[0][0, 0])
        n_harvest = max(1, mlp_steps)
        mesh.mlp_init(hidden=256, rank=16, max_samples=n_harvest * mesh.n_elem, seed=11)
        u = u0.clone()
        t_h = time.perf_counter()
        for k in range(n_harvest):
            mesh.mlp_harvest(u, k * dt, dt * gamma, stride=1)
            mesh.implicit_step(u, k * dt, dt, stages=3, precond="bj", jv_prec="f32")
        t_h = time.perf_counter() - t_h
        torch.cuda.synchronize()
        t_t = time.perf_counter()
        first, last = mesh.mlp_train(epochs=mlp_epochs, batch=1024, lr=1e-3)
        torch.cuda.synchronize()
        training = {"samples": mesh.mlp_sizes()["n_samples"], "harvest_steps": n_harvest,
                    "harvest_s": round(t_h, 2), "train_s": round(time.perf_counter() - t_t, 2),
                    "epochs": mlp_epochs, "loss_first_epoch": first, "loss_last_epoch": last,
                    "params": mesh.mlp_sizes()["n_params"]}
    for name in names:
        kw = IMPLICIT_VARIANTS[name]
        # one untimed step first: the variant's one-time allocations (block storage, FP32 workspace)
        u = u0.clone()
        mesh.rb_reset()
        # (a lagged variant warms up with a per-step build, so its timed steps start with a build)
        warm = dict(kw, precond_refresh="step") if kw.get("precond_refresh") == "lagged" else kw
        mesh.implicit_step(u, 0.0, dt, stages=3, check=False, **warm)
        torch.cuda.synchronize()
        u = u0.clone()
        mesh.rb_reset()
        steps = []
        rc = 0
        kernels = None
        mark = clocks.mark() if clocks else None
        for k in range(n_steps):
            last = k == n_steps - 1
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
                         "kernels_last_step": kernels,
                         "clocks": clocks.summary(mark, clocks.mark()) if clocks else None}
    ref = finals.get("plain_bj")
    if ref is not None:
        du = np.abs(ref - u0.cpu().numpy()).max(axis=(0, 2))
        for name, fin in finals.items():
            if fin is not None and name != "plain_bj":
                results[name]["final_diff_rel_to_change"] = (np.abs(fin - ref).max(axis=(0, 2)) / du).tolist()
    out = {"metric": "implicit DIRK(3,3) step wall time at Newton 1e-8", "unit": "s/step",
           "config": f"{config}: {W.CONFIGS[config][1]}", "n_elem": mesh.n_elem, "n_dof": mesh.n_dof, "dt_s": dt_s,
           "steps": n_steps, "warmup_steps": 1, "variants": results, "mlp_training": training}
    base = results.get("plain_bj", {}).get("wall_s_per_step")
    for name in names:
        if name != "plain_bj" and base and results.get(name, {}).get("rc") == 0:
            out[f"speedup_{name}_vs_plain_bj"] = round(np.mean(base) / np.mean(results[name]["wall_s_per_step"]), 3)
    mesh.close()
    return out


def implicit_summary(res, chosen):
    """The implicit-step comparison as it goes on the benchmark line."""
    v = res["variants"]
    return {"metric": res["metric"], "unit": "s/step", "config": res["config"], "n_dof": res["n_dof"],
            "dt_s": res["dt_s"], "steps": res["steps"], "warmup_steps": 1, "newton_rtol": 1e-8, "chosen": chosen,
            "chosen_means": "FP32 inner Jv, FP32 Gram-Schmidt arithmetic on an FP32 Krylov basis, exact element "
                            "block-Jacobi with FP16-stored inverses built every step; FP64 Newton residual",
            "plain_means": "FP64 Jv and Gram-Schmidt, exact element block-Jacobi with FP32 inverses built "
                           "every step",
            "speedup_chosen_vs_plain": res.get(f"speedup_{chosen}_vs_plain_bj"),
            "speedup_lagged_vs_plain": res.get("speedup_mixed_bj16_lag3_vs_plain_bj"),
            "lagged_means": "the chosen variant with its preconditioner built on the first of every 3 steps "
                            "(DG_REFRESH_LAGGED); the timed steps hold one build",
            "variants": {k: {kk: vv for kk, vv in d.items() if kk != "kernels_last_step"} for k, d in v.items()}}


def main_implicit(args):
    """The implicit-step variants on one workload (--variants), one JSON line."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    config = args.config if args.config != CONFIG_NAME else args.implicit_config
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.2)
    out = implicit_variants(config, args.variants.split(","), args.steps, clocks=clocks,
                            mlp_steps=args.mlp_steps, mlp_epochs=args.mlp_epochs, dt_s=args.dt)
    out["clocks_loaded_window"] = clocks.stop()
    print(json.dumps(out), flush=True)


RADIAL_COLUMNS = 16384


def radial_leg(n_col=RADIAL_COLUMNS, steps=20, warmup=3, implicit_steps=3, clocks=None):
    """The radial 1D ensemble (Sec. 4.3's 28-element p = 2 column, DIRK(2,2) at 30 s) on one GPU:
    n_col independent columns, each with its own site, EUV efficiency and conductivity factor.
    Times the fused residual + exact Jv of the whole ensemble (2x L2 written between steps) and
    whole DIRK(2,2) steps; reports DOF/s and column-steps/s."""
    import numpy as np
    import torch
    from paper_2306_01085_gb300 import dg as DG
    from paper_2306_01085_gb300 import workloads as W
    d = W.radial_desc(n_col=n_col)
    params = W.radial_params(n_col)
    rad = DG.Radial(d, params)
    u0 = W.radial_state(d, seed=3)
    ug = torch.from_numpy(u0).cuda()
    vg = torch.from_numpy(W.unit_vector(17, u0.shape)).cuda()
    r, jv = rad.empty(), rad.empty()
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        rad.jvp(ug, vg, 0.0, out=jv, r_out=r)
    torch.cuda.synchronize()
    mark = clocks.mark() if clocks else None
    rad.profile_start(64 * steps + 64)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        rad.jvp(ug, vg, 0.0, out=jv, r_out=r)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    prof, launches = rad.profile_stop()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    if not (torch.isfinite(r).all() and torch.isfinite(jv).all()):
        raise RuntimeError("non-finite radial residual or Jv")
    clk_rj = clocks.summary(mark, clocks.mark()) if clocks else None
    # implicit steps (each a whole DIRK(2,2) step of every column, host-synchronised Newton)
    dt = 30.0 / W.shell_reference().t0
    u = ug.clone()
    rad.step(u, 0.0, dt, stages=2)                      # warm-up step (first-call costs)
    torch.cuda.synchronize()
    mark = clocks.mark() if clocks else None
    rad.profile_start(100000)
    walls, newton = [], []
    for k in range(implicit_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = rad.step(u, (k + 1) * dt, dt, stages=2, newton_rtol=1e-8)
        torch.cuda.synchronize()
        walls.append(time.perf_counter() - t0)
        newton.append(st["newton"][:2])
    sprof, slaunch = rad.profile_stop()
    clk_st = clocks.summary(mark, clocks.mark()) if clocks else None
    rad.close()
    step_s = float(np.mean(walls))
    n_dof = d.n_dof
    return {"workload": f"radial1d_p2: {n_col} columns x 28 elements, p = 2 (the paper's 1D mesh: first layer "
                        f"2.5 km, geometric growth, 100-600 km), EUVAC heating, 25 (epsilon, alpha0) pairs at "
                        f"seeded sites", "n_col": n_col, "n_dof": n_dof, "dtype": "f64",
            "residual_jv": {"metric": "DG residual+Jv DOFs/s", "value": n_dof / (ms * 1e-3), "unit": "DOF/s",
                            "ms_per_step": round(ms, 4), "steps": steps, "warmup": warmup,
                            "l2": "2x L2 buffer written between timed steps",
                            "kernels": {k: {"ms": round(v[0], 4), "launches": v[1]} for k, v in prof.items()},
                            "gpu_launches": launches, "clocks": clk_rj},
            "implicit": {"metric": "DIRK(2,2) column-steps/s at Newton 1e-8 (dt = 30 s)",
                         "value": n_col / step_s, "unit": "column-steps/s", "s_per_step": round(step_s, 5),
                         "steps": implicit_steps, "newton_per_stage": newton,
                         "jacobian": "FP32, colored tangent probing, banded LU per column; Newton on the FP64 residual",
                         "kernels": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in sprof.items()},
                         "gpu_launches": slaunch, "clocks": clk_st}}


def main_radial(args):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_2306_01085_gb300 import build as B
    B.build()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.2)
    out = radial_leg(n_col=args.radial_columns, steps=args.steps, warmup=args.warmup, clocks=clocks)
    out["clocks_loaded_window"] = clocks.stop()
    print(json.dumps(out), flush=True)


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
    config = args.config   # the benchmarked 12,288-element p = 4 shell unless --config says otherwise
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
    if a.radial:
        main_radial(a)
        sys.exit(0)
    if a.cpu_worker:
        cpu_worker(a.config, a.steps, a.cpu_worker, a.cpu_procs)
    elif a.impl == "reference":
        main_reference(a)
    else:
        main_ours(a)
