#!/usr/bin/env python3
"""Benchmark: SES grid points/s (labels + edge intersections) on one GB300.

Workload: the 5,000-atom synthetic globule (C-alpha walk compacted to 0.0125
atoms/A^3), r_p 1.4 A, h 0.25 A, margin 0.8 A -- 44.7 M grid points.  A step
is one eses_run: cell binning, patch construction, classification of every
point, crossing edges, roots and normals, area and volume.

  value      points/s with the atoms resident in HBM (CUDA events around
             eses_run on the library's stream; L2 flushed between steps)
  e2e        points/s through the public C ABI with host buffers: create from
             pinned host atoms, run, copy labels and intersections back
  plain_fp64 the same step with every stage in FP64 and no proposer (the
             plain GPU form), and the filtered step's labels, edges,
             intersections and normals against its outputs
  proposer_study  the 50,000-atom globule (h 0.2) with the proposer off, the
             certificate on every tile, and the trained MLP + certificate
  roofline   the dominant kernel (by event-timed duration; the other heavy
             kernel beside it) against the FP32 ALU peak, with the algorithmic
             flops of the oracle-counted flop model
  exterior   the headline step with the exterior-only surface (cavities
             filled by flood-fill sweeps; eager, host-synchronised sweeps)
  batch      the 256-molecule workload (log-uniform 300-20,000 atoms, h 0.5)
             in one batched context: persistent tile kernels with a device
             work queue, replayed as one CUDA graph, autotuned launch shapes
  assembly   the 1,000,000-atom assembly (60 rotated 16,667-atom globules,
             h 0.3, ~1.3e10 points) in one context: labels and intersections
             stay in HBM (13 GB of labels), graph replay
  cpu_baseline  the FP64 CPU oracle on a seeded sample of blocks, all cores

--impl reference times the oracle (the reference arm of this build) on the
same workload.  Under torchrun every rank computes its own molecule (weak
scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SES grid points/s (labels+edge intersections)"
UNIT = "points/s"
N_SM = 152
FP32_LANES = 128  # FP32 FMA lanes per SM
WORKLOAD = 2


# DRAM bytes per step (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the globule workload: the root solve's six launches summed
# (profiles/root-solve_globule-5000.md), the classification's two tiers
# (profiles/k_classify_globule-5000.md); reported only while the kernels'
# sources are the ones that were captured
TRAFFIC = {
    "edge_solve": (739_858_432, {"eses_edges.cu": "caf97df99fe6129f", "eses_tile.cuh": "0665160bfe8f347d",
                                 "eses_internal.cuh": "9c0bf5106d8efdeb"}),
    "classify": (10_196_736, {"eses_classify.cu": "71fc2607bb299d7e", "eses_tile.cuh": "0665160bfe8f347d",
                              "eses_internal.cuh": "9c0bf5106d8efdeb"}),
}


def captured_traffic(kernel):
    import hashlib
    entry = TRAFFIC.get(kernel)
    if entry is None:
        return None
    nbytes, shas = entry
    for f, sha in shas.items():
        with open(os.path.join(ROOT, "paper_1809_04352_gb300", "csrc", f), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest()[:16] != sha:
                return None
    return nbytes


def measure_fma_peaks(stream_ptr=0):
    """FP32 and FP64 FMA throughput of this device, measured by the package's
    FMA microbenchmark (libpeaks.so, CUDA events, best of 5 launches)."""
    import ctypes

    from paper_1809_04352_gb300 import build as libbuild
    lib = ctypes.CDLL(libbuild.PEAKS_LIB)
    lib.peaks_fma.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    lib.peaks_fma.restype = ctypes.c_int
    out = (ctypes.c_double * 4)()
    if lib.peaks_fma(5, ctypes.c_void_p(stream_ptr) if stream_ptr else None, out) != 0:
        return None
    return {"fp32_tflops": out[0], "fp32_kernel_ms": out[1], "fp64_tflops": out[2], "fp64_kernel_ms": out[3],
            "how": "FMA microbenchmark: 8 independent FMA chains per thread, 8 blocks of 256 threads per SM, "
                   "2 flops per FMA, best of 5 launches timed with CUDA events"}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        idx = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
        if not idx.isdigit():
            idx = "0"
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", idx, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                    power.append(float(p[3]))
                except ValueError:
                    continue
                for n, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    from paper_1809_04352_gb300.scaling import rank_env
    return rank_env()


def block_atom_counts(xyz, rad, wl, dims, lo, block_pts):
    """Per block of the oracle's block layout (block_pts points, shared faces):
    the number of atoms whose reach r + 2 r_p meets the block's box (a host
    count used only to stratify the timing sample)."""
    import numpy as np

    import oracle
    nb = [oracle.block_count(int(d), block_pts) for d in dims]
    cells = block_pts - 1
    edge = cells * wl.h
    reach = rad + 2.0 * wl.r_p
    b0 = np.clip(np.floor((xyz - reach[:, None] - lo) / edge).astype(np.int64), 0, np.array(nb) - 1)
    b1 = np.clip(np.floor((xyz + reach[:, None] - lo) / edge).astype(np.int64), 0, np.array(nb) - 1)
    cnt = np.zeros(nb, np.int64)
    for i in range(xyz.shape[0]):
        cnt[b0[i, 0]:b1[i, 0] + 1, b0[i, 1]:b1[i, 1] + 1, b0[i, 2]:b1[i, 2] + 1] += 1
    return cnt.reshape(-1)


def cpu_sample(xyz, rad, wl, seed, per_stratum=None, block_pts=32):
    """The oracle's whole-grid time on the host cores, extrapolated from a
    stratified sample: blocks (block_pts points) split into three strata by
    the atoms that reach them (none; up to the median; more), per_stratum
    seeded blocks of each timed on all cores, the whole grid's time taken as
    the sum over strata of (blocks in the stratum) x (measured time per
    block).  Returns (grid points, estimated seconds, cores, blocks timed,
    measured seconds)."""
    import numpy as np

    import oracle
    cores = oracle.num_threads()
    dims, lo = oracle.grid(xyz, rad, wl.h, wl.margin)
    cnt = block_atom_counts(np.asarray(xyz), np.asarray(rad), wl, dims, lo, block_pts)
    nz = cnt[cnt > 0]
    med = float(np.median(nz)) if len(nz) else 0.0
    strata = [np.flatnonzero(cnt == 0), np.flatnonzero((cnt > 0) & (cnt <= med)), np.flatnonzero(cnt > med)]
    per_stratum = per_stratum or cores
    rng = np.random.default_rng(seed)
    est, measured, timed = 0.0, 0.0, 0
    for ids in strata:
        if len(ids) == 0:
            continue
        pick = np.sort(rng.choice(ids, size=min(per_stratum, len(ids)), replace=False))
        t0 = time.perf_counter()
        oracle.run(xyz, rad, wl.r_p, wl.h, wl.margin, block_pts=block_pts, block_ids=pick, nthreads=cores)
        dt = time.perf_counter() - t0
        # dt is the wall time of len(pick) blocks on min(len(pick), cores) threads
        cpu_per_block = dt * min(len(pick), cores) / len(pick)
        est += len(ids) * cpu_per_block / cores
        measured += dt
        timed += len(pick)
    return int(np.prod(dims)), est, cores, timed, measured


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from paper_1809_04352_gb300 import inputs
    wl = inputs.WORKLOADS[WORKLOAD]
    xyz, rad = inputs.workload_atoms(WORKLOAD)
    for w in range(args.warmup):
        cpu_sample(xyz, rad, wl, seed=100 + w, per_stratum=args.ref_blocks)
    pts, secs, meas = 0, 0.0, 0.0
    cores = blocks = 0
    for k in range(args.steps):
        p, dt, cores, blocks, m = cpu_sample(xyz, rad, wl, seed=200 + k, per_stratum=args.ref_blocks)
        pts += p
        secs += dt
        meas += m
    value = pts / secs
    sample = (f"extrapolated: per step, a stratified sample of {blocks} seeded 32^3-point blocks of {wl.name} "
              f"(three strata by the atoms reaching a block) timed on {cores} cores, the whole grid's time "
              f"estimated from the time per block of each stratum; {args.steps} steps, {meas:.1f} s measured")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(wl, xyz, pts // max(args.steps, 1)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def profile_batch(args, eses, inputs, torch):
    """--profile-only on the 256-molecule batch: one context, W + K runs (the
    first plans, the rest replay its graph), one JSON line with the mean step
    and stage times of the last K."""
    bwl = inputs.WORKLOADS[3]
    mols = [inputs.workload_atoms(3, molecule=m) for m in range(len(inputs.batch_sizes()))]
    stream = torch.cuda.current_stream()
    ctx = eses.eses_create_batch(mols, bwl.r_p, bwl.h, bwl.margin)
    try:
        eses.eses_set_option(ctx, eses.ESES_OPT_STREAM, stream.cuda_stream)
        eses.eses_set_option(ctx, eses.ESES_OPT_GRAPH, 0 if args.no_graph else 1)
        eses.eses_set_option(ctx, eses.ESES_OPT_PROFILE, 1)
        times, stages = [], []
        for k in range(args.warmup + args.steps):
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            eses.eses_run(ctx)
            s1.record(stream)
            s1.synchronize()
            if k >= args.warmup:
                times.append(s0.elapsed_time(s1))
                stages.append(eses.eses_stage_times(ctx))
        st = eses.eses_stats(ctx)
        print(json.dumps({"profile_only": True, "workload": bwl.name, "ms_per_step": statistics.mean(times),
                          "stages_ms": {k: statistics.mean(x[k] for x in stages) for k in stages[0]},
                          "kernel_launches_per_step": st["kernel_launches"], "points": st["points"],
                          "crossing_edges": st["crossing_edges"]}))
    finally:
        eses.eses_destroy(ctx)


def config_of(wl, xyz, npts):
    return {"workload": f"{wl.name}: synthetic C-alpha-walk globule, {xyz.shape[0]} atoms, "
                        f"r_p {wl.r_p} A, h {wl.h} A, margin {wl.margin} A",
            "n_atoms": int(xyz.shape[0]), "r_p": wl.r_p, "h": wl.h, "margin": wl.margin,
            "grid_points": npts, "precision": "fp32-filtered, fp64 band and roots",
            "l2": "flushed between steps (256 MiB device write)"}


def fp_compare(eses, ctx, n_mol, h, set_prop, prop_mode, k_steps, labels=True):
    """The context's FP32-filtered results (already run) against its plain
    FP64 form (every stage FP64, no proposer): labels, crossing edges, the
    largest intersection and normal differences, and the FP64 form's step
    time.  Restores the filtered precision and the proposer."""
    import numpy as np

    def grab():
        return [[eses.eses_mol_intersections(ctx, m, a, fp32=False) for a in range(3)] for m in range(n_mol)]

    a32 = grab()
    lab32 = [eses.eses_mol_labels(ctx, m) for m in range(n_mol)] if labels else None
    in32 = eses.eses_stats(ctx)["inside_points"]
    eses.eses_set_option(ctx, eses.ESES_OPT_PRECISION, eses.ESES_PREC_FP64)
    set_prop(ctx, "off")
    eses.eses_run(ctx)
    t = []
    for _ in range(k_steps):
        t0 = time.perf_counter()
        eses.eses_run(ctx)
        t.append(time.perf_counter() - t0)
    a64 = grab()
    same_lab = None
    if labels:
        same_lab = all(np.array_equal(lab32[m], eses.eses_mol_labels(ctx, m)) for m in range(n_mol))
    in64 = eses.eses_stats(ctx)["inside_points"]
    same_edges, dtau, dnrm = True, 0.0, 0.0
    for m in range(n_mol):
        for a in range(3):
            x, y = a32[m][a], a64[m][a]
            if not np.array_equal(x["idx"], y["idx"]):  # same tiles, same order when the edges agree
                same_edges = False
                continue
            if len(x["idx"]):
                dtau = max(dtau, float(np.abs(x["tau"] - y["tau"]).max()) * h)
                dnrm = max(dnrm, float(np.abs(x["normal"] - y["normal"]).max()))
    eses.eses_set_option(ctx, eses.ESES_OPT_PRECISION, eses.ESES_PREC_FP32_FILTERED)
    set_prop(ctx, prop_mode)
    return {"labels_equal": same_lab, "inside_points_equal": bool(in32 == in64), "edges_equal": same_edges,
            "max_intersection_diff_A": dtau, "max_normal_diff": dnrm,
            "fp64_form_ms_per_step": 1e3 * statistics.mean(t), "fp64_form_steps": k_steps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-blocks", type=int, default=None, help="reference arm: blocks timed per stratum")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-only", action="store_true",
                    help="only the warm-up and device-resident steps (for ncu captures); prints stage times")
    ap.add_argument("--profile-workload", default="globule", choices=["globule", "paper-density", "batch-256"],
                    help="with --profile-only: the headline globule, the paper-density globule at h 0.25, or the "
                         "256-molecule batch (h 0.5, one context)")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes instead of the autotuner's")
    ap.add_argument("--no-graph", action="store_true", help="eager launches instead of CUDA-graph replay")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-molecule batched workload")
    ap.add_argument("--no-exterior", action="store_true", help="skip the exterior-only surface step")
    ap.add_argument("--no-assembly", action="store_true", help="skip the 1,000,000-atom assembly")
    ap.add_argument("--proposer", default="mlp", choices=["off", "mlp", "certify"],
                    help="tile proposer of the headline step (default: the trained MLP with the exact certificate)")
    ap.add_argument("--no-proposer-study", action="store_true",
                    help="skip the proposer comparison on the 50,000-atom globule")
    ap.add_argument("--no-density", action="store_true", help="skip the paper-density globule")
    ap.add_argument("--no-precision-study", action="store_true",
                    help="skip the FP32-filtered vs plain FP64 comparison on the larger workloads")
    ap.add_argument("--no-stream", action="store_true",
                    help="skip the assembly at h 0.1 streamed in slabs (3.1e11 points, beyond device memory)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    from paper_1809_04352_gb300 import build as libbuild
    from paper_1809_04352_gb300 import eses, inputs, scaling

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    if rank == 0:
        libbuild.build()
    barrier()
    libbuild.build()
    eses.load()
    if args.profile_only and args.profile_workload == "batch-256":
        profile_batch(args, eses, inputs, torch)
        return
    wl = inputs.WORKLOADS[WORKLOAD]
    xyz, rad = inputs.workload_atoms(WORKLOAD, molecule=rank)
    if args.profile_only and args.profile_workload == "paper-density":
        xyz, rad = inputs.paper_density(5000, 2200)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed_runs(ctx, k):
        times, stages = [], []
        for _ in range(k):
            flush.zero_()
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record(stream)
            eses.eses_run(ctx)
            e.record(stream)
            e.synchronize()
            times.append(s.elapsed_time(e))
            stages.append(eses.eses_stage_times(ctx))
        return times, stages

    # ---- device-resident step (value) --------------------------------------
    from paper_1809_04352_gb300 import proposer as prop
    prop_modes = {"off": eses.ESES_PROPOSER_OFF, "mlp": eses.ESES_PROPOSER_MLP,
                  "certify": eses.ESES_PROPOSER_CERTIFY}
    params = prop.load_params()

    def set_prop(c, mode):
        eses.eses_set_proposer(c, prop_modes[mode], params if mode == "mlp" else None, 0.5)

    ctx = eses.eses_create(xyz, rad, wl.r_p, wl.h, wl.margin)
    eses.eses_set_option(ctx, eses.ESES_OPT_STREAM, stream.cuda_stream)
    eses.eses_set_option(ctx, eses.ESES_OPT_PROFILE, 1)
    set_prop(ctx, args.proposer)
    use_graph = not args.no_graph
    eses.eses_set_option(ctx, eses.ESES_OPT_GRAPH, 1 if use_graph else 0)
    tuned = None
    if not args.no_autotune and not args.profile_only:
        cls_ms, edge_ms = eses.eses_autotune(ctx, 3)
        tuned = {k: eses.eses_get_option(ctx, v) for k, v in (
            ("cls_ctas_per_sm", eses.ESES_OPT_CLS_CTAS), ("cls_tiles_per_pop", eses.ESES_OPT_CLS_TILES),
            ("edge_ctas_per_sm", eses.ESES_OPT_EDGE_CTAS), ("edge_tiles_per_pop", eses.ESES_OPT_EDGE_TILES),
            ("root_threads", eses.ESES_OPT_ROOT_THREADS))}
    for _ in range(args.warmup):
        eses.eses_run(ctx)
    dims, _ = eses.eses_grid(ctx)
    npts = int(np.prod(dims))
    torch.cuda.synchronize()
    barrier()
    clocks = Clocks()
    clocks.start()
    times, stages = timed_runs(ctx, args.steps)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    st = eses.eses_stats(ctx)
    if args.profile_only:
        print(json.dumps({"profile_only": True, "ms_per_step": statistics.mean(times),
                          "stages_ms": {k: statistics.mean(s[k] for s in stages) for k in stages[0]},
                          "kernel_launches_per_step": st["kernel_launches"], "points": npts}))
        eses.eses_destroy(ctx)
        return
    total_s, all_pts = scaling.job_totals(sum(times) / 1e3, float(npts), "cuda")
    value = scaling.throughput(all_pts, args.steps, total_s)
    stage_ms = {k: statistics.mean(s[k] for s in stages) for k in stages[0]}

    # ---- plain FP64 form (same step, every stage FP64) ----------------------
    lab32 = eses.eses_labels(ctx)
    out32 = [eses.eses_intersections(ctx, a) for a in range(3)]
    eses.eses_set_option(ctx, eses.ESES_OPT_PRECISION, eses.ESES_PREC_FP64)
    set_prop(ctx, "off")
    eses.eses_run(ctx)
    t64, s64 = timed_runs(ctx, max(2, min(args.steps, 5)))
    plain_ms = statistics.mean(t64)
    # the FP32-filtered step's outputs against the plain FP64 step's
    out64 = [eses.eses_intersections(ctx, a) for a in range(3)]
    same_edges = all(np.array_equal(np.sort(out32[a]["idx"]), np.sort(out64[a]["idx"])) for a in range(3))
    dtau = dnrm = d32 = 0.0
    if same_edges:
        for a in range(3):
            o1, o2 = np.argsort(out32[a]["idx"]), np.argsort(out64[a]["idx"])
            if len(o1):
                dtau = max(dtau, float(np.abs(out32[a]["tau"][o1] - out64[a]["tau"][o2]).max()) * wl.h)
                dnrm = max(dnrm, float(np.abs(out32[a]["normal"][o1] - out64[a]["normal"][o2]).max()))
                d32 = max(d32, float(np.abs(out32[a]["tau32"].astype(np.float64) - out32[a]["tau"]).max()) * wl.h)
    precision_check = {"labels_equal": bool(np.array_equal(lab32, eses.eses_labels(ctx))),
                       "edges_equal": bool(same_edges), "max_intersection_diff_A": dtau,
                       "max_normal_diff": dnrm, "tau32_rounding_A": d32}
    del lab32, out32, out64
    eses.eses_set_option(ctx, eses.ESES_OPT_PRECISION, eses.ESES_PREC_FP32_FILTERED)
    eses.eses_destroy(ctx)

    # ---- buried-patch pre-culling on the headline molecule -------------------
    culling = None
    if not args.no_density:
        cctx = eses.eses_create(xyz, rad, wl.r_p, wl.h, wl.margin)
        eses.eses_set_option(cctx, eses.ESES_OPT_STREAM, stream.cuda_stream)
        eses.eses_set_option(cctx, eses.ESES_OPT_PROFILE, 1)
        set_prop(cctx, args.proposer)
        culling = {}
        labs = {}
        for cull in (1, 0):
            eses.eses_set_option(cctx, eses.ESES_OPT_CULL, cull)
            for _ in range(2):
                eses.eses_run(cctx)
            ct, cs = timed_runs(cctx, max(3, min(args.steps, 5)))
            labs[cull] = eses.eses_labels(cctx)
            culling["culled" if cull else "unculled"] = {
                "ms_per_step": statistics.mean(ct), "stages_ms": {k: statistics.mean(v[k] for v in cs) for k in cs[0]},
                "big_tier_tiles": int(eses.eses_stats(cctx)["big_tier_tiles"])}
        npair, nfree, nvert = eses.eses_patch_counts(cctx)
        culling.update(workload=wl.name, circle_pairs=npair, free_arc_pairs=nfree, free_vertices=nvert,
                       labels_equal=bool(np.array_equal(labs[0], labs[1])), graph=False,
                       gain=culling["unculled"]["ms_per_step"] / culling["culled"]["ms_per_step"])
        del labs
        eses.eses_destroy(cctx)

    # ---- end to end through the C ABI with host buffers ---------------------
    xyz_pin = torch.from_numpy(np.ascontiguousarray(xyz)).pin_memory()
    rad_pin = torch.from_numpy(np.ascontiguousarray(rad)).pin_memory()
    lab_pin = torch.empty(npts, dtype=torch.int8).pin_memory()
    caps = [0, 0, 0]
    bufs = None
    h2d = xyz.nbytes + rad.nbytes + (params.nbytes if args.proposer == "mlp" else 0)
    d2h = 0
    e2e_times = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = eses.eses_create(xyz_pin.numpy(), rad_pin.numpy(), wl.r_p, wl.h, wl.margin)
        set_prop(c2, args.proposer)
        eses.eses_run(c2)
        eses.eses_labels(c2, lab_pin.numpy().reshape(tuple(int(v) for v in dims)))
        ne = [eses.eses_num_intersections(c2, a) for a in range(3)]
        if bufs is None or any(ne[a] > caps[a] for a in range(3)):
            caps = [int(v * 1.2) + 16 for v in ne]
            bufs = [(torch.empty(c, dtype=torch.int64).pin_memory(), torch.empty(c, dtype=torch.float64).pin_memory(),
                     torch.empty(3 * c, dtype=torch.float64).pin_memory()) for c in caps]
        lib = eses.load()
        for a in range(3):
            lib.eses_intersections(c2, a, bufs[a][0].data_ptr(), bufs[a][1].data_ptr(), bufs[a][2].data_ptr(), None,
                                   None)
        area_vol = eses.eses_area_volume(c2)
        eses.eses_destroy(c2)
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_times.append(t1 - t0)
        d2h = npts + sum(ne) * (8 + 8 + 24) + 16
    e2e_s = scaling.job_max(sum(e2e_times), "cuda")
    e2e_value = scaling.throughput(all_pts, args.steps, e2e_s)

    # ---- roofline of the dominant kernel ------------------------------------
    peaks, psrc = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fma = measure_fma_peaks(stream.cuda_stream)
    if fma is not None:
        fp32_peak = fma["fp32_tflops"]
        psrc_txt = "measured: " + fma["how"]
    else:
        fp32_peak = N_SM * FP32_LANES * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
        psrc_txt = f"derived: {N_SM} SMs x {FP32_LANES} FP32 lanes x 2 flops x {sm_max:.0f} MHz (sm_max_mhz {psrc})"
    with open(os.path.join(ROOT, "tests", "golden", "flop_model.json")) as f:
        fm = json.load(f)[wl.name]
    # algorithmic flops per launch (oracle-counted flop model) and the kernel's
    # mean event-timed duration over the timed steps
    kernels = {
        "classify": ("k_classify<float,true> (FP32-filtered classification, every grid point)",
                     fm["model_flops"], stage_ms["classify"],
                     {"flops_per_point": fm["flops_per_point"]}),
        "edge_solve": ("root solve: k_edge_stage, k_roots_sphere, k_roots_torus, k_roots_torus_exact, k_edge_pick, "
                       "k_edge_hard "
                       "<float,true> (first root and its patch of every crossing edge)",
                       fm["edge_counts"]["model_flops"], stage_ms["edge_solve"],
                       {"flops_per_edge": fm["edge_flops_per_edge"], "edges": fm["edge_counts"]["edges"]}),
    }
    rl = {}
    for name, (kname, flops, ms, extra) in kernels.items():
        achieved = flops / (ms / 1e3) / 1e12
        rl[name] = dict({"bound": "alu", "kernel": kname, "achieved": achieved, "peak": fp32_peak,
                         "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": captured_traffic(name),
                         "peak_source": psrc_txt, "flops_per_launch": flops, "kernel_ms": ms}, **extra)
    dominant = max(rl, key=lambda k: rl[k]["kernel_ms"])
    roofline = rl[dominant]
    roofline_others = {k: v for k, v in rl.items() if k != dominant}

    # ---- proposer study: the 50,000-atom globule, h 0.2, three modes ---------
    study = None
    if not args.no_proposer_study:
        swl = inputs.WORKLOADS[4]
        sxyz, srad = inputs.workload_atoms(4)
        sctx = eses.eses_create(sxyz, srad, swl.r_p, swl.h, swl.margin)
        eses.eses_set_option(sctx, eses.ESES_OPT_STREAM, stream.cuda_stream)
        eses.eses_set_option(sctx, eses.ESES_OPT_PROFILE, 1)
        eses.eses_set_option(sctx, eses.ESES_OPT_GRAPH, 1 if use_graph else 0)
        study = {"workload": f"{swl.name}: synthetic globule, {sxyz.shape[0]} atoms, r_p {swl.r_p} A, h {swl.h} A, "
                             f"margin {swl.margin} A"}
        ref_labels = None
        for mode in ("off", "certify", "mlp"):
            set_prop(sctx, mode)
            for _ in range(2):
                eses.eses_run(sctx)
            ts, sts = timed_runs(sctx, max(2, min(args.steps, 5)))
            sst = eses.eses_stats(sctx)
            # identical labels in every mode (the certificate keeps them exact)
            same = None
            cur = eses.eses_labels(sctx).reshape(-1)
            if ref_labels is None:
                ref_labels = cur
            else:
                same = bool(np.array_equal(cur, ref_labels))
            study[mode] = {"ms_per_step": statistics.mean(ts),
                           "classify_ms": statistics.mean(x["classify"] for x in sts),
                           "points_per_s": sst["points"] / (statistics.mean(ts) / 1e3),
                           "tiles": int(sst["tiles"]), "tiles_proposed_far": int(sst["tiles_proposed_far"]),
                           "tiles_certified": int(sst["tiles_certified"]), "labels_equal_off": same}
        study["points"] = int(sst["points"])
        study["mlp_gain_vs_off"] = study["off"]["ms_per_step"] / study["mlp"]["ms_per_step"]
        study["mlp_gain_vs_certify"] = study["certify"]["ms_per_step"] / study["mlp"]["ms_per_step"]
        if not args.no_precision_study:
            study["fp32_filtered_vs_fp64"] = fp_compare(eses, sctx, 1, swl.h, set_prop, "mlp", 2)
        eses.eses_destroy(sctx)

    # ---- exterior-only surface on the headline molecule -----------------------
    exterior = None
    if not args.no_exterior:
        xctx = eses.eses_create(xyz, rad, wl.r_p, wl.h, wl.margin)
        eses.eses_set_option(xctx, eses.ESES_OPT_STREAM, stream.cuda_stream)
        eses.eses_set_option(xctx, eses.ESES_OPT_PROFILE, 1)
        set_prop(xctx, args.proposer)
        eses.eses_set_option(xctx, eses.ESES_OPT_EXTERIOR, 1)
        eses.eses_run(xctx)
        torch.cuda.synchronize()
        barrier()
        xt, xs = timed_runs(xctx, max(3, min(args.steps, 5)))
        torch.cuda.synchronize()
        barrier()
        xst = eses.eses_stats(xctx)
        xav = eses.eses_area_volume(xctx)
        exterior = {"ms_per_step": statistics.mean(xt), "points_per_s": npts / (statistics.mean(xt) / 1e3),
                    "band_and_fill_ms": statistics.mean(v["band"] for v in xs),
                    "cavity_points": int(xst["cavity_points"]), "sweeps": int(xst["exterior_sweeps"]),
                    "crossing_edges": int(xst["crossing_edges"]), "area_A2": xav[0], "volume_A3": xav[1],
                    "graph": False}
        eses.eses_destroy(xctx)

    # ---- the paper-density globule (0.1 atoms/A^3), h 0.25 and 0.4 ---------------
    density = None
    if not args.no_density:
        dxyz, drad = inputs.paper_density(5000, 2200)
        density = {"workload": "paper-density-5000: synthetic globule at 0.1 atoms/A^3 (eight atoms per residue), "
                               f"{dxyz.shape[0]} atoms, r_p 1.4 A, margin 0.8 A"}
        for dh in (0.25, 0.4):
            dctx = eses.eses_create(dxyz, drad, 1.4, dh, 0.8)
            eses.eses_set_option(dctx, eses.ESES_OPT_STREAM, stream.cuda_stream)
            eses.eses_set_option(dctx, eses.ESES_OPT_PROFILE, 1)
            eses.eses_set_option(dctx, eses.ESES_OPT_GRAPH, 1 if use_graph else 0)
            set_prop(dctx, args.proposer)
            for _ in range(args.warmup):
                eses.eses_run(dctx)
            torch.cuda.synchronize()
            barrier()
            dt, ds = timed_runs(dctx, max(3, min(args.steps, 10)))
            dst = eses.eses_stats(dctx)
            density[f"h{dh}"] = {"value": dst["points"] / (statistics.mean(dt) / 1e3), "unit": UNIT,
                                 "ms_per_step": statistics.mean(dt), "points": int(dst["points"]),
                                 "crossing_edges": int(dst["crossing_edges"]),
                                 "root_failures": int(dst["root_failures"]),
                                 "stages_ms": {k: statistics.mean(v[k] for v in ds) for k in ds[0]}}
            if not args.no_precision_study:
                density[f"h{dh}"]["fp32_filtered_vs_fp64"] = fp_compare(eses, dctx, 1, dh, set_prop, args.proposer, 2)
            # buried-patch pre-culling (§5 of the paper): the same step with every circle and face staged
            npair, nfree, nvert = eses.eses_patch_counts(dctx)
            eses.eses_set_option(dctx, eses.ESES_OPT_CULL, 0)
            try:
                eses.eses_run(dctx)
                unculled = "runs"
            except eses.EsesError as e:
                unculled = f"fails: {e}"
            density[f"h{dh}"]["culling"] = {"circle_pairs": npair, "free_arc_pairs": nfree, "free_vertices": nvert,
                                            "without_culling": unculled}
            eses.eses_destroy(dctx)

    # ---- batched workload: 256 molecules in one context ---------------------
    batch = None
    if not args.no_batch:
        bwl = inputs.WORKLOADS[3]
        mols = [inputs.workload_atoms(3, molecule=m) for m in range(len(inputs.batch_sizes()))]
        bctx = eses.eses_create_batch(mols, bwl.r_p, bwl.h, bwl.margin)
        eses.eses_set_option(bctx, eses.ESES_OPT_STREAM, stream.cuda_stream)
        eses.eses_set_option(bctx, eses.ESES_OPT_GRAPH, 1 if use_graph else 0)
        if not args.no_autotune:
            eses.eses_autotune(bctx, 2)
        for _ in range(args.warmup):
            eses.eses_run(bctx)
        bpts = eses.eses_stats(bctx)["points"]
        torch.cuda.synchronize()
        barrier()
        bt = []
        for _ in range(args.steps):
            flush.zero_()
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            eses.eses_run(bctx)
            s1.record(stream)
            s1.synchronize()
            bt.append(s0.elapsed_time(s1))
        torch.cuda.synchronize()
        barrier()
        bst = eses.eses_stats(bctx)
        btot, bpts_all = scaling.job_totals(sum(bt) / 1e3, float(bpts), "cuda")
        batch = {"workload": f"{bwl.name}: {len(mols)} synthetic globules, atom counts log-uniform in [300, 20000] "
                             f"({sum(len(r) for _, r in mols)} atoms), r_p {bwl.r_p} A, h {bwl.h} A, "
                             f"margin {bwl.margin} A, one context",
                 "value": scaling.throughput(bpts_all, args.steps, btot), "unit": UNIT,
                 "ms_per_step": 1e3 * btot / args.steps,
                 "points": int(bpts), "crossing_edges": int(bst["crossing_edges"]),
                 "root_failures": int(bst["root_failures"]), "kernel_launches_per_step": int(bst["kernel_launches"]),
                 "graph": use_graph}
        if not args.no_precision_study:
            batch["fp32_filtered_vs_fp64"] = fp_compare(eses, bctx, len(mols), bwl.h, lambda c, m: None, None, 1)
        eses.eses_destroy(bctx)

    # ---- the 1,000,000-atom assembly in one context --------------------------
    assembly = None
    if not args.no_assembly:
        awl = inputs.WORKLOADS[5]
        axyz, arad = inputs.workload_atoms(5)
        actx = eses.eses_create(axyz, arad, awl.r_p, awl.h, awl.margin)
        eses.eses_set_option(actx, eses.ESES_OPT_STREAM, stream.cuda_stream)
        eses.eses_set_option(actx, eses.ESES_OPT_GRAPH, 1 if use_graph else 0)
        set_prop(actx, args.proposer)
        for _ in range(2):  # planning run, then the graph capture
            eses.eses_run(actx)
        torch.cuda.synchronize()
        barrier()
        at = []
        for _ in range(2):  # inputs and outputs far larger than L2
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            eses.eses_run(actx)
            a1.record(stream)
            a1.synchronize()
            at.append(a0.elapsed_time(a1))
        torch.cuda.synchronize()
        barrier()
        ast = eses.eses_stats(actx)
        atot, apts_all = scaling.job_totals(sum(at) / 1e3, float(ast["points"]), "cuda")
        assembly = {"workload": f"{awl.name}: 60 copies of a 16,667-atom globule on an icosahedral shell of radius "
                                f"300 A ({axyz.shape[0]} atoms), r_p {awl.r_p} A, h {awl.h} A, margin {awl.margin} A",
                    "value": scaling.throughput(apts_all, len(at), atot), "unit": UNIT,
                    "ms_per_step": 1e3 * atot / len(at), "steps": len(at), "points": int(ast["points"]),
                    "crossing_edges": int(ast["crossing_edges"]), "root_failures": int(ast["root_failures"]),
                    "graph": use_graph, "proposer": args.proposer}
        if not args.no_precision_study:
            assembly["fp32_filtered_vs_fp64"] = fp_compare(eses, actx, 1, awl.h, set_prop, args.proposer, 1,
                                                           labels=False)
        eses.eses_destroy(actx)

    # ---- the assembly at h 0.1 streamed in slabs (beyond device memory) -----
    streamed = None
    if not args.no_stream:
        from paper_1809_04352_gb300 import stream as sstream
        axyz, arad = inputs.workload_atoms(5)
        free_b, total_b = torch.cuda.mem_get_info()
        kept = {"slabs": 0}

        def sink(k, part):
            kept["slabs"] += 1

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tot = sstream.stream(axyz, arad, 1.4, 0.1, 0.8, sink, max_points=6 << 30, block_pts=128,
                             proposer_params=params if args.proposer == "mlp" else None)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        streamed = {"workload": f"assembly-1M at h 0.1 A: {int(np.prod(tot['dims']))} points "
                                f"({int(np.prod(tot['dims'])) / 1e9:.0f} GB of labels, device {total_b / 1e9:.0f} GB), "
                                f"{tot['slabs']} slabs of at most {6 << 30} points, 2 contexts on 2 streams",
                    "value": tot["points"] / wall, "unit": UNIT, "wall_s": wall, "points": int(tot["points"]),
                    "crossing_edges": int(tot["crossing_edges"]), "area_A2": tot["area"], "volume_A3": tot["volume"],
                    "timing": "host wall clock around the whole streamed run: model builds, every slab's run and "
                              "its labels and intersections copied to host memory"}

    # ---- CPU baseline (rank 0, N = 1) ---------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pts, secs, cores, nblk, meas = cpu_sample(xyz, rad, wl, seed=7)
        cpu = {"value": pts / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"extrapolated: a stratified sample of {nblk} seeded 32^3-point blocks of {wl.name} "
                         f"(three strata by the atoms reaching a block, {meas:.1f} s measured on {cores} cores); "
                         f"whole-grid time estimated as {secs:.1f} s for {pts} points"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": config_of(wl, xyz, npts),
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * e2e_s / args.steps},
                "gpu_launches": int(st["kernel_launches"]) * args.steps,
                "roofline": roofline,
                "roofline_other_kernels": roofline_others,
                "peaks": {"fma": fma, "fp32_derived_tflops": N_SM * FP32_LANES * 2 * sm_max * 1e6 / 1e12,
                          "hbm_gbs": peaks.get("hbm_gbs"), "hbm_source": psrc},
                "launch": {"cuda_graph": use_graph, "autotuned": tuned, "proposer": args.proposer},
                "proposer_study": study,
                "exterior": exterior,
                "batch": batch,
                "assembly": assembly,
                "assembly_streamed": streamed,
                "paper_density": density,
                "culling": culling,
                "cpu_baseline": cpu,
                "clocks": clk,
                "plain_fp64": {"value": all_pts / (plain_ms / 1e3), "unit": UNIT, "ms_per_step": plain_ms,
                               "stages_ms": {k: statistics.mean(s[k] for s in s64) for k in s64[0]},
                               "fp32_filtered_vs_fp64": precision_check},
                "stages_ms": stage_ms,
                "stats": {k: st[k] for k in ("crossing_edges", "inside_points", "circle_pairs", "free_vertices",
                                             "root_failures")},
                "area_A2": area_vol[0], "volume_A3": area_vol[1]}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
