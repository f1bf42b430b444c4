"""Throughput of the batched biased-Langevin trial generator with the bias
functional: aggregate atom-steps/s over 64 trials of the 11 040-atom
solvated heteropolymer (one GPU), plus the roofline of the dominant kernel,
the end-to-end number through the C ABI with host buffers, and the FP64
oracle on the host cores.

One bench "step" = one list interval: nstlist (10) MD steps of every trial,
i.e. one pass over every stage of the hot path (cell/list rebuild, pair and
bonded forces, reaction coordinate and ratchet bias, Langevin update,
functional accumulation).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "aggregate atom-steps/s (batched biased Langevin + functional) vs plain; % HBM roofline"
WORKLOAD = "64 trials x 11040-atom heteropolymer in flexible water (4.8 nm box), RF cut-off 1.0 nm, dt 1 fs"
# algorithmic model of one atom-step at this density (r_list = 1.1 nm, 99.8 atoms/nm^3):
BYTES_PER_ATOM_STEP = 1224.0         # 112 B of state + 278 int32 half-list entries
PAIRS_PER_ATOM_STEP = 209.0          # half pairs inside r_cut = 1.0 nm
FLOPS_PER_PAIR = 35.0                # LJ + reaction field, FP32
# DRAM traffic of one pair-kernel launch on this workload (dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture) per captured variant, and the
# sources it was taken on (the kernel and its headers): reported as
# roofline.traffic only for the variant the run timed and while those sources
# are unchanged
PAIR_TRAFFIC = {"bytes": {7: 209.478144e6 + 7.621120e6},
                "sources": ["vp_pair.cu", "vp_pair_dev.cuh", "vp_internal.cuh", "vp_dev.cuh"],
                "source_sha256": "86bf29a2be4c3f89a6b649ade11c513d8430aa27292543f9b5049b829ba28b94"}


def pair_traffic(variant):
    import hashlib
    if variant not in PAIR_TRAFFIC["bytes"]:
        return None
    h = hashlib.sha256()
    try:
        for f in PAIR_TRAFFIC["sources"]:
            h.update(open(os.path.join(ROOT, "paper_1405_6104_gb300", "csrc", f), "rb").read())
    except OSError:
        return None
    return PAIR_TRAFFIC["bytes"][variant] if h.hexdigest() == PAIR_TRAFFIC["source_sha256"] else None


def rank_info():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms from before
    the warm-up to after the kernel-timing pass; summarised over the samples
    whose timestamps fall inside the timed region (or, when that region is
    shorter than three sampling periods, over the whole loaded window)."""

    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        # wait (bounded) for the first sample so that the window is covered
        t0 = time.time()
        while self.p is not None and time.time() - t0 < 5.0 and os.path.getsize(self.f.name) == 0:
            time.sleep(0.05)

    @staticmethod
    def _stamp(text: str):
        import datetime
        try:
            return datetime.datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self, t_begin: float, t_end: float):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = []
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((self._stamp(parts[0]), float(parts[1]), float(parts[2]),
                             {nm for nm, v in zip(self.NAMES, parts[5:9]) if v.lower().startswith("active")}))
            except ValueError:
                continue
        os.unlink(self.f.name)
        inside = [r for r in rows if r[0] is not None and t_begin <= r[0] <= t_end]
        window = "timed region"
        if len(inside) < 3:
            inside, window = rows, "warm-up + timed region + kernel-timing pass (timed region < 3 samples)"
        if not inside:
            return None
        reasons = set().union(*[r[3] for r in inside])
        return {"sm_mhz": statistics.median([r[1] for r in inside]), "sm_max_mhz": inside[-1][2],
                "reasons": sorted(reasons), "samples": len(inside), "window": window}


def equilibrate(B, S, s, p, steps: int = 3000, gamma: float = 20.0):
    """Relaxes the generated start (random water orientations are hot) with
    strong friction and no bias on the GPU; returns the system with the
    relaxed positions (velocities are then drawn per trial)."""
    pe = S.Params(**{**p.__dict__, "gamma": gamma, "k_ratchet": 0.0})
    with B.TrialBatch(s, pe, [1], trial_seeds=[7]) as b:
        b.step(steps)
        pos, _, _ = b.get_state(0)
    out = s.copy()
    out.pos = pos.astype(np.float32).astype(np.float64)
    out.vel = None
    return out


def make_batch(B, S, prep_steps: int, stream_ptr=0, rank: int = 0, world: int = 1):
    """This rank's 64 trials of the weak-scaling batch: global trials
    rank*64 .. rank*64+63 (shard_trials), Philox seeds 1000 + global index."""
    from paper_1405_6104_gb300.shard import shard_trials
    s, p, seeds = S.batched_64(1)
    trials = shard_trials(len(seeds) * world, world, rank)
    seeds = [1000 + int(t) for t in trials]
    if prep_steps > 0:
        s = equilibrate(B, S, s, p, steps=prep_steps)
    batch = B.TrialBatch(s, p, [len(seeds)], trial_seeds=seeds, cuda_stream=stream_ptr)
    batch.global_trials = trials
    return s, p, seeds, batch


def cpu_baseline(S, steps: int = 60, one_core_steps: int = 0):
    """The FP64 oracle as it stands on the host cores: one trial of the same
    11 040-atom system for a bounded number of MD steps, on all cores and
    (one_core_steps > 0) on one core."""
    import oracle as O
    s, p = S.plain_single(1)
    O.run(s, p, 1000, 1)  # build and warm
    t0 = time.perf_counter()
    r = O.run(s, p, 1000, steps)
    dt = time.perf_counter() - t0
    assert r["status"] == 0
    out = {"value": s.n_atoms * steps / dt, "unit": "atom-steps/s", "cores": O.num_threads(), "kind": "oracle",
           "sample": f"1 trial x {steps} MD steps of the 11040-atom system (FP64; its O(N^2) list rebuild at the "
                     "displacement rule)", "seconds": dt}
    if one_core_steps > 0:
        all_cores = O.num_threads()
        O.set_num_threads(1)
        try:
            t1 = time.perf_counter()
            O.run(s, p, 1000, one_core_steps)
            d1 = time.perf_counter() - t1
        finally:
            O.set_num_threads(all_cores)
        out["one_core"] = {"value": s.n_atoms * one_core_steps / d1, "unit": "atom-steps/s", "cores": 1,
                           "sample": f"1 trial x {one_core_steps} MD steps", "seconds": d1}
    return out


def run_reference(args):
    from paper_1405_6104_gb300 import systems as S
    r, w, _ = rank_info()
    if r != 0:
        return 0
    steps_per = 10
    vals = []
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(S, steps=steps_per)
        if k >= args.warmup:
            vals.append(cb)
    total_t = sum(v["seconds"] for v in vals)
    value = 11040 * steps_per * len(vals) / total_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "atom-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / len(vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (oracle: one trial per step sample)", "global_batch": 1,
                       "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": "atom-steps/s", "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": f"each step: 1 trial x {steps_per} MD steps of the 11040-atom system"},
            "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import torch
    import torch.distributed as dist

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    import __graft_entry__
    if world > 1:  # one rank per node compiles (the others would race on the object files)
        if local == 0:
            __graft_entry__.build()
        dist.barrier()
    __graft_entry__.build()
    from paper_1405_6104_gb300 import binding as B
    from paper_1405_6104_gb300 import systems as S

    s, p, seeds, batch = make_batch(B, S, args.prep_steps, rank=rank, world=world)
    n_trials = len(seeds)
    atoms = n_trials * s.n_atoms
    nst = p.nstlist
    stream = torch.cuda.ExternalStream(batch.stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # launch shapes picked by the project's autotuner on this batch (untimed),
    # or fixed from the command line (through the autotuner's cache format)
    if args.pair_variant is None and args.cv_variant is None:
        tuned = B.sim_autotune(batch.h, 5, None)
        step_form = B.sim_autotune_step(batch.h, 2)
    else:
        probe = tempfile.mktemp(suffix=".txt")
        picked = B.sim_autotune(batch.h, 1, probe)
        key = open(probe).read().split()[0]
        with open(probe, "w") as f:
            f.write(f"{key} {args.pair_variant if args.pair_variant is not None else picked[0]} "
                    f"{args.cv_variant if args.cv_variant is not None else picked[1]}\n")
        tuned = B.sim_autotune(batch.h, 1, probe)
        os.unlink(probe)
        step_form = 0
    # the roofline times the pair launches of the timed region: the one-kernel
    # form has none, so it is timed in the kernel-per-phase form
    timed_form = 0 if step_form == 1 else step_form
    B.sim_set_step_mode(batch.h, timed_form)
    clocks = ClockSampler(local) if rank == 0 else None
    # event-record nodes around the pair kernel inside the chunk graph: the
    # roofline's launch duration is measured over the timed region itself
    B.sim_set_timing(batch.h, 2)
    # warm-up (also captures the CUDA graph)
    for _ in range(args.warmup):
        batch.step(nst)
    barrier()
    B.sim_kernel_times(batch.h)  # drop the warm-up's launches
    diag0 = B.sim_diagnostics(batch.h)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_begin = time.time()
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed launches
    ev0.record(stream)
    for _ in range(args.steps):
        batch.step(nst)
    ev1.record(stream)
    barrier()
    torch.cuda.nvtx.range_pop()
    t_end = time.time()
    ms = ev0.elapsed_time(ev1)
    diag1 = B.sim_diagnostics(batch.h)
    in_graph = B.sim_kernel_times(batch.h).get("pair_in_graph", (float("nan"), 0))
    B.sim_set_timing(batch.h, 0)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / args.steps
    value = world * atoms * nst * args.steps / (ms * 1e-3)

    # per-kernel times (direct launches, CUDA events on the library stream)
    B.sim_set_timing(batch.h, True)
    B.sim_kernel_times(batch.h)
    kt_steps = max(2, min(args.steps, 5))
    for _ in range(kt_steps):
        batch.step(nst)
    kt = B.sim_kernel_times(batch.h)
    B.sim_set_timing(batch.h, False)
    clk = clocks.stop(t_begin, t_end) if clocks else None

    # the method's selection over every rank's trials, on the functional
    # accumulated since the start (warm-up, timed region, kernel-timing pass):
    # one double per trial gathered on the host
    from paper_1405_6104_gb300.shard import global_selection
    phi_loc, _ = batch.bias_functional()
    sel_trial, sel_phi = global_selection(phi_loc, batch.global_trials)
    sel_steps = (args.warmup + args.steps + kt_steps) * nst
    phi_all = np.asarray(phi_loc, np.float64)

    # end to end through the C ABI with host buffers: per step the state of
    # every trial is uploaded from pinned memory, nstlist steps are taken and
    # the functional plus the selected trial are read back
    pos0 = torch.empty((atoms, 3), dtype=torch.float64, pin_memory=True)
    vel0 = torch.empty((atoms, 3), dtype=torch.float64, pin_memory=True)
    off = 0
    for t in range(n_trials):
        pp, vv, _ = batch.get_state(t)
        pos0[off:off + s.n_atoms] = torch.from_numpy(pp)
        vel0[off:off + s.n_atoms] = torch.from_numpy(vv)
        off += s.n_atoms
    P, V = pos0.numpy(), vel0.numpy()
    e2e_steps = max(2, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        batch.set_state(-1, P, V)
        batch.step(nst)
        phi, am = batch.bias_functional()
    t1 = time.perf_counter()
    e2e = {"value": world * atoms * nst * e2e_steps / (t1 - t0), "unit": "atom-steps/s",
           "h2d_bytes_per_step": int(P.nbytes + V.nbytes), "d2h_bytes_per_step": int(phi.nbytes + 4 + 4)}
    diag = B.sim_diagnostics(batch.h)
    # 8 x 4 atom pairs per list entry, masked pairs included
    diag["pairs_evaluated_per_atom_step"] = round(8.0 * diag["list_entries"] / atoms, 1)
    # list rebuilds of the timed region: a trial's list is rebuilt when one of
    # its atoms has moved skin/2 - 1e-5 nm since the list was built, or after
    # nstlist steps, so no pair within r_cut is ever missing from it
    trial_steps = n_trials * nst * args.steps
    rb = diag1["trial_rebuilds"] - diag0["trial_rebuilds"]
    diag["timed_region"] = {
        "skin_violations": diag1["skin_violations"] - diag0["skin_violations"],
        "trial_rebuilds": rb, "trial_steps": trial_steps,
        "mean_steps_between_rebuilds": round(trial_steps / max(rb, 1), 2),
        "displacement_triggered": diag1["displacement_rebuilds"] - diag0["displacement_rebuilds"]}
    batch.close()

    # plain: one trial of the same system on the same kernels (graph replay),
    # the single-trial GPU baseline that batching is compared with
    plain = None
    if rank == 0:
        with B.TrialBatch(s, p, [1], trial_seeds=seeds[:1]) as one:
            B.sim_autotune(one.h, 5, None)
            plain_form, plain_forms_ms = B.sim_autotune_step(one.h, 3, times=True)
            ostream = torch.cuda.ExternalStream(one.stream)
            for _ in range(args.warmup):
                one.step(nst)
            torch.cuda.synchronize()
            n_plain = max(10, args.steps)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ostream)
            for _ in range(n_plain):
                one.step(nst)
            e1.record(ostream)
            torch.cuda.synchronize()
            pv = s.n_atoms * nst * n_plain / (e0.elapsed_time(e1) * 1e-3)
            plain = {"value": pv, "unit": "atom-steps/s",
                     "workload": f"1 trial x {s.n_atoms} atoms, same kernels, {n_plain} x {nst} MD steps",
                     "step_form": B.STEP_FORM_NAMES[plain_form],
                     "ms_per_md_step_by_form": dict(zip(B.STEP_FORM_NAMES, plain_forms_ms)),
                     "batching_speedup": value / world / pv}

    if rank == 0:
        pk, src = peaks()
        pair_ms, pair_n = in_graph
        pair_avg_s = pair_ms / max(pair_n, 1) * 1e-3
        # ALU roofline of the pair kernel (dominant): algorithmic FP32 flops per launch
        flops_launch = atoms * PAIRS_PER_ATOM_STEP * FLOPS_PER_PAIR
        sm_mhz = pk.get("sm_max_mhz", 2070.0)
        fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6
        achieved = flops_launch / pair_avg_s
        step_s = ms_per_step * 1e-3 / nst
        hbm_achieved = atoms * BYTES_PER_ATOM_STEP / step_s / 1e9
        try:
            cb = cpu_baseline(S, one_core_steps=10)
        except Exception as exc:  # the baseline must not sink the GPU line
            cb = {"value": None, "unit": "atom-steps/s", "cores": None, "kind": "oracle", "sample": f"failed: {exc}"}
        line = {
            "metric": METRIC, "value": value, "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+i64-fixed+ff-cv", "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": n_trials * world, "atoms_per_trial": s.n_atoms,
                       "start": f"generated, relaxed {args.prep_steps} steps at gamma 20/ps (untimed)",
                       "md_steps_per_bench_step": nst, "parallelism": f"replicas x{world}",
                       "autotuned": {"pair_variant": tuned[0], "cv_variant": tuned[1],
                                     "step_form": B.STEP_FORM_NAMES[step_form],
                                     "timed_form": B.STEP_FORM_NAMES[timed_form]},
                       "l2": "working set > L2 (lists + state ~0.5 GB)"},
            "roofline": {"bound": "alu", "kernel": "pair", "achieved": achieved / 1e12, "peak": fp32_peak / 1e12,
                         "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": pair_traffic(tuned[0]),
                         "traffic_unit": f"bytes per launch (ncu, variant {tuned[0]})",
                         "launch_ms": pair_avg_s * 1e3, "launches_timed": pair_n,
                         "launch_timing": "event-record nodes around each pair launch inside the replayed graphs of the timed region",
                         "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (SM max clock: {src})",
                         "work": f"{PAIRS_PER_ATOM_STEP:.0f} half pairs x {FLOPS_PER_PAIR:.0f} flops per atom-step"},
            "hbm_model": {"bytes_per_atom_step": BYTES_PER_ATOM_STEP, "achieved": hbm_achieved,
                          "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": hbm_achieved / pk["hbm_gbs"],
                          "peak_source": src},
            "kernel_ms": {k: v[0] / v[1] for k, v in kt.items() if v[1] > 0},
            "plain": plain,
            "cpu_baseline": cb,
            "e2e": e2e,
            "gpu_launches": int(round(args.steps * sum(v[1] for v in kt.values()) / kt_steps)),
            "clocks": clk,
            "diagnostics": diag,
            "selection": {"trial": sel_trial, "phi": sel_phi, "over_trials": n_trials * world,
                          "md_steps": sel_steps,
                          "phi_quartiles_rank0": [float(x) for x in np.percentile(phi_all, [0, 25, 50, 75, 100])]},
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# the toy model: the section's rMD protocol (2000 trials of 30 000 steps per
# K_R) over a scan of twelve K_R values spanning two and a half decades
TOY_K = [0.25 * 2 ** (i / 1.5) for i in range(12)]  # 0.25 .. 40
TOY_TRIALS, TOY_STEPS = 2000, 30000
# FP64 operations of one trial-step as the equations state them (normals 12,
# B-A-O-A-B 26, force 51, z 4, ratchet 9, functional 5, sum 2; a division,
# square root, logarithm or sincos counts as one)
TOY_FLOPS_PER_STEP = 109.0


def toy_cpu_baseline(S, tp, ks, seeds, per_k: int = 2):
    import oracle as O
    idx = [i for k in TOY_K for i in np.where(ks == k)[0][:per_k]]
    O.toy2d_run(tp, ks[idx[0]], int(seeds[idx[0]]), 100)
    t0 = time.perf_counter()
    steps = 0
    for i in idx:
        n, _, _, _ = O.toy2d_run(tp, ks[i], int(seeds[i]), TOY_STEPS)
        steps += n if n >= 0 else TOY_STEPS
    dt = time.perf_counter() - t0
    return {"value": steps / dt, "unit": "trial-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(idx)} trials ({per_k} per K_R) of up to {TOY_STEPS} steps, one core", "seconds": dt}


def run_toy(args):
    """The two-dimensional toy model: one bench step = one toy2d_run over the
    whole K_R scan (12 x 2000 trials of up to 30 000 steps, each to first
    passage)."""
    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1405_6104_gb300 import binding as B
    from paper_1405_6104_gb300 import systems as S
    tp, ks, seeds = S.toy2d_rmd_batch(TOY_TRIALS, TOY_K)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    for _ in range(args.warmup):
        passage, phi, _, _ = B.toy2d_run(tp, ks, seeds, TOY_STEPS, want_state=False, cuda_stream=sp)
    executed = float(np.where(passage >= 0, passage, TOY_STEPS).sum())
    clocks = ClockSampler(local) if rank == 0 else None
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_begin = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        B.toy2d_run(tp, ks, seeds, TOY_STEPS, want_state=False, cuda_stream=sp)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_end = time.time()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop(t_begin, t_end) if clocks else None
    value = executed * args.steps / (ms * 1e-3)
    pk, src = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    fp64_peak = 152 * 2 * 2 * sm_mhz * 1e6  # 2 FP64 FMA per SM per clock
    achieved = TOY_FLOPS_PER_STEP * executed / (ms * 1e-3 / args.steps)
    best = {}
    for k in TOY_K:
        sel = np.where((ks == k) & (passage >= 0))[0]
        best[f"{k:.3g}"] = {"reached": float(len(sel) / TOY_TRIALS),
                            "best_phi": float(phi[sel].min()) if len(sel) else None}
    line = {
        "metric": "trial-steps/s (2-D toy model: rMD trials + functional, K_R scan)", "value": value,
        "unit": "trial-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"2-D toy model, {len(TOY_K)} K_R values x {TOY_TRIALS} rMD trials x up to "
                               f"{TOY_STEPS} steps (each to first passage)", "trial_steps_executed": executed,
                   "l2": "state in registers; no inputs beyond 32 B per trial"},
        "roofline": {"bound": "alu", "kernel": "k_toy2d", "achieved": achieved / 1e12, "peak": fp64_peak / 1e12,
                     "unit": "TFLOP/s (FP64)", "frac": achieved / fp64_peak, "traffic": None,
                     "peak_source": f"152 SMs x 2 FP64 FMA x 2 x {sm_mhz:.0f} MHz",
                     "work": f"{TOY_FLOPS_PER_STEP:.0f} FP64 operations per trial-step"},
        "cpu_baseline": toy_cpu_baseline(S, tp, ks, seeds),
        "gpu_launches": args.steps,
        "clocks": clk,
        "per_k": best,
    }
    print(json.dumps(line))
    return 0


def run_adjoint(args):
    """Row a9 at its configuration: the functional's gradient along a
    500-frame path of the 30 000-atom system (1800-atom solute), checkpoints
    every 50 steps.  One bench step = forward 500 steps with checkpoints,
    the coefficients, the reverse sweep (each segment restored and replayed
    with the frame recorder, then the adjoint kernels)."""
    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1405_6104_gb300 import binding as B
    from paper_1405_6104_gb300 import systems as S
    from paper_1405_6104_gb300.adjoint import trajectory_adjoint
    s, p = S.adjoint_30k(3)
    p.k_ratchet = 5.0
    n_frames, every = 500, 50
    with B.TrialBatch(s, p, [1], trial_seeds=[3]) as b:
        B.sim_autotune(b.h, 3, None)
        fwd_form, fwd_forms_ms = B.sim_autotune_step(b.h, 2, times=True)
        stream = torch.cuda.ExternalStream(b.stream)
        for _ in range(args.warmup):
            trajectory_adjoint(b, 0, n_frames, every=every)
        clocks = ClockSampler(local) if rank == 0 else None
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_begin = time.time()
        t0 = time.perf_counter()
        ev0.record(stream)
        for _ in range(args.steps):
            phi, G, _ = trajectory_adjoint(b, 0, n_frames, every=every)
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        t_end = time.time()
        ms = ev0.elapsed_time(ev1)
        clk = clocks.stop(t_begin, t_end) if clocks else None
        # where the time goes: one more run with per-kernel timing on the
        # batch and on the batch that replays the segments side by side
        handles = [b.h] + [rb.h for rb in b.__dict__.get("_replay_batches", {}).values()]
        forms = [B.sim_step_mode(hh) for hh in handles]
        for hh in handles:
            B.sim_set_step_mode(hh, 0)  # per-kernel times need the kernel-per-phase form
            B.sim_set_timing(hh, 1)
            B.sim_kernel_times(hh)
        t1 = time.perf_counter()
        trajectory_adjoint(b, 0, n_frames, every=every)
        t_kt = time.perf_counter() - t1
        kt, kt_fwd = {}, None
        for hh in handles:
            for k, (t_ms, cnt) in B.sim_kernel_times(hh).items():
                a0, c0 = kt.get(k, (0.0, 0))
                kt[k] = (a0 + t_ms, c0 + cnt)
            if kt_fwd is None:
                kt_fwd = dict(kt)
            B.sim_set_timing(hh, 0)
        for hh, f in zip(handles, forms):
            B.sim_set_step_mode(hh, f)
    md_ms = sum(v[0] for v in kt.values())
    pk, _ = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6
    pair_ms = kt_fwd["pair"][0] / kt_fwd["pair"][1]  # the single trial's launches (the forward run)
    pair_flops = s.n_atoms * PAIRS_PER_ATOM_STEP * FLOPS_PER_PAIR
    n_seg = n_frames // every
    line = {
        "metric": "adjoint frames/s (gradient of the functional along a path, checkpointed replay)",
        "value": n_frames * args.steps / (ms * 1e-3), "unit": "frames/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+i64-fixed+ff-cv", "data": "synthetic",
        "config": {"workload": f"30 000 atoms (1800-atom solute, 9400 waters), {n_frames} frames (1 per step), "
                               f"checkpoints every {every} steps, k_R 5", "phi": float(phi),
                   "grad_max": float(np.abs(G).max()),
                   "forward_step_form": B.STEP_FORM_NAMES[fwd_form],
                   "forward_ms_per_md_step_by_form": dict(zip(B.STEP_FORM_NAMES, fwd_forms_ms))},
        "wall_s_per_step": wall / args.steps,
        "md_kernels_ms_per_step": md_ms,
        "md_kernel_share": md_ms / (t_kt * 1e3),
        "kernel_ms": {k: v[0] / v[1] for k, v in kt.items() if v[1] > 0},
        "note": "per bench step: 500 MD steps of the 30 000-atom trial forward, then its 10 segments replayed side by "
                "side (one batch of 10 trials, 50 steps) and the adjoint kernels; the rest is checkpoint transfers "
                "and the host loop",
        "roofline": {"bound": "alu", "kernel": "pair (one 30 000-atom trial)", "achieved": pair_flops / (pair_ms * 1e-3) / 1e12,
                     "peak": fp32_peak / 1e12, "unit": "TFLOP/s", "frac": pair_flops / (pair_ms * 1e-3) / fp32_peak,
                     "traffic": None, "launch_ms": pair_ms,
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz",
                     "work": f"{PAIRS_PER_ATOM_STEP:.0f} half pairs x {FLOPS_PER_PAIR:.0f} flops per atom-step",
                     "launch_timing": "direct launches timed by CUDA events in a pass after the timed region"},
        "cpu_baseline": adjoint_cpu_baseline(S, s, p),
        # the step kernels of one gradient (from the timing pass) and the four
        # adjoint kernels of each segment, over the timed gradients
        "gpu_launches": args.steps * (int(sum(v[1] for v in kt.values())) + 4 * n_seg),
        "clocks": clk,
    }
    print(json.dumps(line))
    return 0


def adjoint_cpu_baseline(S, s, p, n_md: int = 10, n_grad: int = 10):
    """The FP64 oracle on the host cores for one adjoint frame: two MD steps
    (forward run and replay) and the gradient of Phi at one frame, from a
    bounded sample (n_md MD steps, n_grad frames) of the same system."""
    import oracle as O
    t0 = time.perf_counter()
    r = O.run(s, p, 3, n_md, record_every=1)
    t_md = (time.perf_counter() - t0) / n_md
    frames = np.asarray(r["frames"])[:n_grad] if "frames" in r else np.repeat(np.asarray(s.pos)[None], n_grad, 0)
    t1 = time.perf_counter()
    O.phi_frames_grad(s, p, frames)
    t_grad = (time.perf_counter() - t1) / len(frames)
    return {"value": 1.0 / (2 * t_md + t_grad), "unit": "frames/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{n_md} MD steps and the gradient at {len(frames)} frames of the 30 000-atom system; "
                      "one frame = 2 MD steps + its gradient"}


def run_similarity(args):
    """Row f3: path similarity of every pair of 64 trial paths of the
    11 040-atom system (23 160 native contacts), from formation times
    tracked on the GPU during 100 steps."""
    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1405_6104_gb300 import binding as B
    from paper_1405_6104_gb300 import systems as S
    s, p, seeds = S.batched_64(1)
    with B.TrialBatch(s, p, [len(seeds)], trial_seeds=seeds) as b:
        B.sim_contact_tracking(b.h, 10)
        b.step(100)
        n_c = len(B.sim_native_contacts(b.h, 0))
        T = np.stack([B.sim_contact_times(b.h, t, n_c) for t in range(len(seeds))])
    pairs = [(a, c) for a in range(len(seeds)) for c in range(a + 1, len(seeds))]
    stream = torch.cuda.Stream()
    for _ in range(args.warmup):
        B.path_similarity(T, pairs, cuda_stream=stream.cuda_stream)
    clocks = ClockSampler(local) if rank == 0 else None
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_begin = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        sim = B.path_similarity(T, pairs, cuda_stream=stream.cuda_stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_end = time.time()
    clk = clocks.stop(t_begin, t_end) if clocks else None
    ms = ev0.elapsed_time(ev1) / args.steps
    import oracle as O
    t0 = time.perf_counter()
    O.path_similarity(T[0], T[1])
    t_or = time.perf_counter() - t0
    comparisons = float(len(pairs)) * n_c * (n_c - 1)
    line = {
        "metric": "path-pair similarities/s (every pair of trial paths)",
        "value": len(pairs) / (ms * 1e-3), "unit": "path pairs/s", "n_gpus": 1, "steps": args.steps,
        "definition_rate": {"value": comparisons / (ms * 1e-3), "unit": "ordered contact pairs/s",
                            "note": "the definition's n_c (n_c - 1) comparisons per path pair / time"},
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"{len(seeds)} trials x 11 040 atoms, {n_c} native contacts, {len(pairs)} path pairs "
                               f"(formation times from 100 tracked steps)", "s_mean": float(np.mean(sim)),
                   "s_min": float(np.min(sim)), "s_max": float(np.max(sim))},
        "note": "one call ranks the times on the host, uploads the ranks, counts the agreeing ordered contact pairs "
                "of every path pair (joint histogram of the ranks when the paths hold few distinct times) and reads back s",
        "cpu_baseline": {"value": 1.0 / t_or, "unit": "path pairs/s", "cores": 1, "kind": "oracle",
                         "sample": f"one path pair, all {n_c * (n_c - 1)} ordered contact pairs (the definition)"},
        "gpu_launches": args.steps * (1 if all(len(set(r)) * len(set(r)) <= 4096 for r in T) else 2),
        "clocks": clk
    }
    print(json.dumps(line))
    return 0


def equilibrate_batch(B, S, systems, p, steps: int, gamma: float = 20.0):
    """Relaxes every system of a batch together (strong friction, no bias);
    returns copies of the systems with the relaxed FP32 positions."""
    pe = S.Params(**{**p.__dict__, "gamma": gamma, "k_ratchet": 0.0})
    out = []
    with B.TrialBatch(systems, pe, [1] * len(systems), trial_seeds=[7 + k for k in range(len(systems))]) as b:
        b.step(steps)
        for k, s in enumerate(systems):
            pos, _, _ = b.get_state(k)
            c = s.copy()
            c.pos = pos.astype(np.float32).astype(np.float64)
            c.vel = None
            out.append(c)
    return out


def _timed_batch(B, batch, n_calls: int, nst: int, stream):
    """CUDA-event milliseconds of n_calls calls of nst steps on the batch's stream."""
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(n_calls):
        batch.step(nst)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def run_uneven(args):
    """BASELINE configuration of the uneven batch: 32 systems of 5 000 to
    60 000 atoms (solutes of 200 to 2000 atoms, boxes at 33 water-equivalents
    per nm^3), one trial each, 5 000 MD steps (500 bench steps of 10) after a
    relaxation; launch shapes from the autotuner, chosen per size class."""
    import torch
    import torch.distributed as dist
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import __graft_entry__
    if world > 1:  # one rank per node compiles
        if local == 0:
            __graft_entry__.build()
        dist.barrier()
    __graft_entry__.build()
    from paper_1405_6104_gb300 import binding as B
    from paper_1405_6104_gb300 import systems as S
    from paper_1405_6104_gb300.shard import shard_by_cost
    steps = args.steps if args.steps is not None else 500
    all_systems, p = S.uneven_32(2)
    nst = p.nstlist
    atoms_all = int(sum(s.n_atoms for s in all_systems))
    # a fixed ensemble split over the ranks by its cost (atoms x steps): strong scaling
    mine = shard_by_cost([s.n_atoms * steps * nst for s in all_systems], world, rank)
    systems = [all_systems[k] for k in mine]
    if args.prep_steps > 0:
        systems = equilibrate_batch(B, S, systems, p, min(args.prep_steps, 1000))
    atoms = int(sum(s.n_atoms for s in systems))
    seeds = [2000 + int(k) for k in mine]

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    with B.TrialBatch(systems, p, [1] * len(systems), trial_seeds=seeds) as b:
        tuned = B.sim_autotune(b.h, 5, None)
        classes = B.sim_tune_classes(b.h)
        # the roofline times pair launches: the one-kernel form has none
        form = B.sim_autotune_step(b.h, 2)
        timed_form = 0 if form == 1 else form
        B.sim_set_step_mode(b.h, timed_form)
        stream = torch.cuda.ExternalStream(b.stream)
        clocks = ClockSampler(local) if rank == 0 else None
        B.sim_set_timing(b.h, 2)
        for _ in range(args.warmup):
            b.step(nst)
        torch.cuda.synchronize()
        B.sim_kernel_times(b.h)
        diag0 = B.sim_diagnostics(b.h)
        barrier()
        t_begin = time.time()
        ms = _timed_batch(B, b, steps, nst, stream)
        barrier()
        t_end = time.time()
        ms = max_over_ranks(ms)
        diag1 = B.sim_diagnostics(b.h)
        pair_ms, pair_n = B.sim_kernel_times(b.h).get("pair_in_graph", (float("nan"), 0))
        B.sim_set_timing(b.h, 0)
        clk = clocks.stop(t_begin, t_end) if clocks else None
        phi, best = b.bias_functional()
        # end to end with host buffers, as the default line
        P = np.concatenate([b.get_state(k)[0] for k in range(len(systems))])
        V = np.concatenate([b.get_state(k)[1] for k in range(len(systems))])
        e2e_calls = 10
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_calls):
            b.set_state(-1, P, V)
            b.step(nst)
            phi_e, _ = b.bias_functional()
        t1 = t0 + max_over_ranks(time.perf_counter() - t0)
        B.sim_set_timing(b.h, 1)
        B.sim_kernel_times(b.h)
        for _ in range(3):
            b.step(nst)
        kt = B.sim_kernel_times(b.h)
        B.sim_set_timing(b.h, 0)
    value = atoms_all * nst * steps / (ms * 1e-3)
    from paper_1405_6104_gb300.shard import global_selection
    best, best_phi = global_selection(phi, np.asarray(mine, np.int64))
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    pk, src = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6
    pair_avg_s = pair_ms / max(pair_n, 1) * 1e-3
    flops = atoms * PAIRS_PER_ATOM_STEP * FLOPS_PER_PAIR  # the same water density in every system
    # the oracle on the host cores: a bounded sample (the smallest system, a few steps)
    import oracle as O
    small = min(range(len(all_systems)), key=lambda k: all_systems[k].n_atoms)
    O.run(all_systems[small], p, 2000 + small, 1)
    tc = time.perf_counter()
    O.run(all_systems[small], p, 2000 + small, 20)
    t_or = time.perf_counter() - tc
    line = {
        "metric": METRIC, "value": value, "unit": "atom-steps/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "f32+i64-fixed+ff-cv", "data": "synthetic",
        "config": {"workload": f"uneven batch: 32 systems of {min(s.n_atoms for s in all_systems)} to "
                               f"{max(s.n_atoms for s in all_systems)} atoms ({atoms_all} in all), one trial each, "
                               f"{steps * nst} MD steps timed", "md_steps_per_bench_step": nst,
                   "parallelism": f"trials sharded over {world} rank(s) by atoms x steps",
                   "start": f"generated, relaxed {min(args.prep_steps, 1000)} steps at gamma 20/ps (untimed)",
                   "autotuned": {"pair_variant": tuned[0], "cv_variant": tuned[1], "size_classes": classes,
                                 "step_form": B.STEP_FORM_NAMES[form], "timed_form": B.STEP_FORM_NAMES[timed_form]},
                   "l2": "working set > L2"},
        "roofline": {"bound": "alu", "kernel": "pair", "achieved": flops / pair_avg_s / 1e12,
                     "peak": fp32_peak / 1e12, "unit": "TFLOP/s", "frac": flops / pair_avg_s / fp32_peak,
                     "traffic": None, "launch_ms": pair_avg_s * 1e3, "launches_timed": pair_n,
                     "launch_timing": "event-record nodes around the pair launches of each step in the replayed graphs",
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz",
                     "work": f"{PAIRS_PER_ATOM_STEP:.0f} half pairs x {FLOPS_PER_PAIR:.0f} flops per atom-step"},
        "kernel_ms": {k: v[0] / v[1] for k, v in kt.items() if v[1] > 0},
        "cpu_baseline": {"value": all_systems[small].n_atoms * 20 / t_or, "unit": "atom-steps/s",
                         "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"the smallest system ({all_systems[small].n_atoms} atoms), 20 MD steps"},
        "e2e": {"value": atoms_all * nst * e2e_calls / (t1 - t0), "unit": "atom-steps/s",
                "h2d_bytes_per_step": int(P.nbytes + V.nbytes) * atoms_all // atoms,
                "d2h_bytes_per_step": int(phi_e.nbytes + 8) * atoms_all // atoms if world == 1 else
                8 * len(all_systems) + 8 * world},
        "gpu_launches": int(round(steps * sum(v[1] for v in kt.values()) / 3)),
        "clocks": clk,
        "diagnostics": {"skin_violations": diag1["skin_violations"] - diag0["skin_violations"],
                        "trial_rebuilds": diag1["trial_rebuilds"] - diag0["trial_rebuilds"],
                        "trial_steps": len(systems) * nst * steps},
        "selection": {"trial": int(best), "phi": float(best_phi),
                      "phi_per_trial": [float(x) for x in phi] if world == 1 else None},
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_long(args):
    """The stated run lengths: the 64-trial batch for 10 000 MD steps (each
    trial's functional, the selected trial, error flags and list statistics)
    and one trial of the same system for 20 000 MD steps, from the relaxed
    start; timed as a whole (one bench step = the whole run)."""
    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1405_6104_gb300 import binding as B
    from paper_1405_6104_gb300 import systems as S
    s, p, seeds = S.batched_64(1)
    s = equilibrate(B, S, s, p, steps=args.prep_steps) if args.prep_steps > 0 else s
    out = {}
    clocks = ClockSampler(local) if rank == 0 else None
    t_begin = time.time()
    for name, n_trials, n_md in (("batch64_10000", 64, 10000), ("single_20000", 1, 20000)):
        with B.TrialBatch(s, p, [n_trials], trial_seeds=seeds[:n_trials]) as b:
            B.sim_autotune(b.h, 3, None)
            form = B.sim_autotune_step(b.h, 2)
            stream = torch.cuda.ExternalStream(b.stream)
            b.step(p.nstlist)  # captures the chunk graph
            ms = _timed_batch(B, b, (n_md - p.nstlist) // p.nstlist, p.nstlist, stream)
            phi, best = b.bias_functional()
            zs = [b.get_state(k)[2] for k in range(n_trials)]
            diag = B.sim_diagnostics(b.h)
        steps_timed = n_md - p.nstlist
        out[name] = {
            "trials": n_trials, "md_steps": n_md, "atom_steps_per_s": n_trials * s.n_atoms * steps_timed / (ms * 1e-3),
            "ms": ms, "status": "ok (no error flag)", "phi": [float(x) for x in phi], "argmin": int(best),
            "phi_min": float(phi[best]), "z_final": [float(z[0]) for z in zs], "z_min": [float(z[1]) for z in zs],
            "skin_violations": diag["skin_violations"], "trial_rebuilds": diag["trial_rebuilds"],
            "mean_steps_between_rebuilds": round(n_trials * n_md / max(diag["trial_rebuilds"], 1), 2),
            "step_form": B.STEP_FORM_NAMES[form]}
    t_end = time.time()
    clk = clocks.stop(t_begin, t_end) if clocks else None
    line = {"metric": METRIC, "value": out["batch64_10000"]["atom_steps_per_s"], "unit": "atom-steps/s",
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": out["batch64_10000"]["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64-fixed+ff-cv", "data": "synthetic",
            "config": {"workload": "64 trials x 11040 atoms for 10 000 MD steps (10 ps), and 1 trial for 20 000",
                       "start": f"generated, relaxed {args.prep_steps} steps at gamma 20/ps (untimed)"},
            "runs": out, "clocks": clk}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed bench steps (default 60: 60 x 10 MD steps keep the clock sampler inside the timed "
                         "region; uneven: 500, i.e. the configuration's 5 000 MD steps)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="batched64",
                    choices=["batched64", "uneven", "long", "toy2d", "adjoint30k", "similarity"],
                    help="batched64: the 64 x 11 040-atom trial batch (default); uneven: 32 systems of 5k-60k atoms, "
                         "5 000 steps; long: the stated run lengths (64 trials x 10 000 steps, 1 trial x 20 000); "
                         "toy2d: the 2-D toy model's K_R scan; adjoint30k: the functional's gradient along a "
                         "500-frame path of 30 000 atoms; similarity: path similarity over 64 trial paths")
    ap.add_argument("--pair-variant", type=int, default=None, help="fix the pair-kernel variant (skip autotuning)")
    ap.add_argument("--cv-variant", type=int, default=None, help="fix the reaction-coordinate kernel variant")
    ap.add_argument("--prep-steps", type=int, default=3000,
                    help="untimed relaxation steps of the generated start (0: none, e.g. for kernel profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "uneven":
        return run_uneven(args)
    if args.steps is None:
        args.steps = 60
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "toy2d":
        return run_toy(args)
    if args.workload == "adjoint30k":
        return run_adjoint(args)
    if args.workload == "similarity":
        return run_similarity(args)
    if args.workload == "long":
        return run_long(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
