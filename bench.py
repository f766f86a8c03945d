"""Benchmark of the QM/MM-Multipole hot path on GB300.

A step is one V+forces call at one geometry through the C ABI:
    qmmm_set_positions -> qmmm_vpot -> qmmm_ewald -> qmmm_forces
i.e. region I and the region-II potential, the region-I matrix V (Eq. 9), the multipoles and
E_II (Eq. 6, Eq. 10), and the full gradient (region-I adjoint, tensor and Pulay terms).

Metric: shell-pair x charge integrals/s = (screened shell pairs x region-I charges) per step / step
time, plus ms per V+forces call; FP64 is the headline (the active-site workload is quoted in FP64)
and the mixed-precision path is measured beside it with its error against FP64.

Default workload: the largest single-GPU configuration, a large active site of 150 QM atoms with f
shells (1500 shells, 5100 AOs) and 198723 MM charges (TIP3P waters) in an 86 A box, cutoff 12 A,
alpha 0.3 A^-1, kmax 24 (synthetic, seeded); --config c2 is the 60-atom active site.  The L2 is
flushed (256 MiB write) before every timed step, outside the timed interval.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config c1|c2|c4|c5]
(c5: 64 uneven frames through the batch API, one CUDA graph, against a loop of FP64 calls)
N > 1 runs replicas (one per GPU, launched by torch.distributed.run): the path does not shard.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "shell-pair x charge integrals/s; ms per V+forces call, mixed vs FP64 at 1e-6"
UNIT = "integrals/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# plain-ALU peaks at the maximum SM clock (2070 MHz, 152 SMs): FP64 2 FMA/clk/SM (the part's
# 1.25 TFLOP/s FP64 rating), FP32 128 FMA/clk/SM
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def comb(n, k):
    return math.comb(n, k) if n >= k >= 0 else 0


def flops_forward(L):
    """Algorithmic FLOPs per (primitive pair, charge) of the V sweep: Boys 25+3L, R recursion
    2 C(L+4,4), Hermite accumulation 2 C(L+3,3), setup 15."""
    return 25 + 3 * L + 2 * comb(L + 4, 4) + 2 * comb(L + 3, 3) + 15


def flops_adjoint(L):
    """Per (primitive pair, charge) of the adjoint sweep: Boys to L+1 (28+3L), R recursion to L+1
    2 C(L+5,4), the four density contractions (e_0, e_x, e_y, e_z) and the charge sum
    S += q R over the C(L+3,3) Hermite terms 10 C(L+3,3), setup/accumulation/reduction 47.  The
    centre-A derivative coefficients meet S once per pair, not per charge, so they are not
    counted per term (the FP64 kernels of the f-shell classes with L >= 5 contract them per
    charge instead: 4 C(L+3,3) more than counted here)."""
    return 28 + 3 * L + 2 * comb(L + 5, 4) + 10 * comb(L + 3, 3) + 47


CLASS_L = [la + lb for la in range(4) for lb in range(la + 1)]  # class index la(la+1)/2 + lb

# DRAM bytes (read + write) of one adjoint sweep (all angular-class kernels of one call, the mixed
# path's pair records and pair gradients included), per (workload, precision), from one ncu
# capture of the current kernels (dram__bytes_read.sum + dram__bytes_write.sum); a workload or
# precision without a capture of the current kernels reports None.
SWEEP_TRAFFIC = {("c4", "fp64"): 153_470_720, ("c4", "mixed"): 364_729_600}


def sweep_flops(info, adjoint):
    f = flops_adjoint if adjoint else flops_forward
    return sum(n * info["n_region1"] * f(CLASS_L[c]) for c, n in enumerate(info["n_prim_pairs_class"]))


def make_system(name):
    import workloads
    return {"c1": workloads.config1_water, "c2": workloads.config2_active_site,
            "c4": workloads.config4_large_site}[name]()


def describe(s, info):
    A = 0.52917721092
    return (f"{s.name}: {s.natm} QM atoms, {s.nshell} shells, {s.nao} AOs, {s.nmm} MM charges (TIP3P), "
            f"{s.box[0] * A:.1f} A box, cutoff {s.cutoff * A:.1f} A, alpha {s.ewald_alpha / A:.2f} A^-1, "
            f"kmax {s.kmax[0]}, sigma {s.mm_sigma[0] * A:.2f} A; {info['n_shell_pairs']} screened shell pairs, "
            f"{info['n_region1']} region-I charges")


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    def __init__(self, gpu_index):
        self.samples = []
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if len(s) > 3 + k and s[3 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest value of x over all ranks: the job's time is that of its slowest replica."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_step, ms):
    """Whole-job throughput: every replica processes units_per_step per step of ms milliseconds."""
    return world * units_per_step / (ms * 1e-3)


def _shell_subset(s, shells):
    """The workload restricted to a subset of its shells (same atoms, MM charges and Ewald
    parameters; the density is the matching AO block): a bounded sample of the moment work."""
    ao = np.concatenate([[0], np.cumsum([(l + 1) * (l + 2) // 2 for l in s.shell_l])])
    t = s.copy()
    t.shell_atom = np.ascontiguousarray(s.shell_atom[shells])
    t.shell_l = np.ascontiguousarray(s.shell_l[shells])
    t.shell_nprim = np.ascontiguousarray(s.shell_nprim[shells])
    offs, exps, coefs = [], [], []
    for sh in shells:
        o, n = int(s.shell_prim_offset[sh]), int(s.shell_nprim[sh])
        offs.append(len(exps))
        exps += list(s.prim_exp[o:o + n])
        coefs += list(s.prim_coeff[o:o + n])
    t.shell_prim_offset = np.asarray(offs, dtype=s.shell_prim_offset.dtype)
    t.prim_exp, t.prim_coeff = np.asarray(exps), np.asarray(coefs)
    idx = np.concatenate([np.arange(ao[sh], ao[sh + 1]) for sh in shells])
    t.dm = np.ascontiguousarray(s.dm[np.ix_(idx, idx)])
    return t


def _charge_subset(s, sub):
    t = s.copy()
    t.mm_xyz = np.ascontiguousarray(s.mm_xyz[sub])
    t.mm_q = np.ascontiguousarray(s.mm_q[sub])
    t.mm_sigma = np.ascontiguousarray(s.mm_sigma[sub])
    return t


# Screened shell pairs of each seeded workload as the library's planner counts them (reported by
# qmmm_get_info; the GPU arm checks its own count against this): the reference arm, which runs no
# GPU code, needs the same units per step as the GPU arm.
SCREENED_SHELL_PAIRS = {"c1": 78, "c2": 47386, "c4": 172365}


def cpu_baseline(s, seconds=12.0, seed=0, n_shell_pairs=None):
    """The FP64 oracle on the host cores, for the whole V+forces step of the workload, from bounded
    samples scaled to the full step (each piece's cost is linear in what is sampled):
      * region-I V + adjoint (Obara-Saika): a random sample of shell pairs x all region-I charges;
      * Mulliken moments and multipoles: a random subset of the shells (cost per shell pair);
      * region-II potential at the QM sites (real-space + reciprocal Ewald, region-I and Gaussian
        corrections): a random subset of the MM charges;
      * the MM-side Ewald derivatives (dE/dq, dE/dR_MM): a random subset of the MM charges.
      * the Pulay term (moment derivatives): the same shell subset; the QM tensor gradient (O(natm)):
        the whole system.
    Same per-(shell pair, charge) unit as the GPU metric."""
    import oracle
    rng = np.random.default_rng(seed)
    cores = os.cpu_count()
    idx = oracle.region1(s)[0]
    nI = len(idx)
    npairs = s.nshell * (s.nshell + 1) // 2
    units = (n_shell_pairs if n_shell_pairs is not None else npairs) * nI  # the GPU arm's unit count

    # region-I V + adjoint on sampled shell pairs (about half the budget)
    pairs_all = [(i, j) for i in range(s.nshell) for j in range(i, s.nshell)]
    k, t_pairs, n_pairs = 2, 0.0, 0
    while True:
        pick = rng.choice(len(pairs_all), k, replace=False)
        pairs = [pairs_all[p] for p in pick]
        pairs = [(a, b) if s.shell_l[a] >= s.shell_l[b] else (b, a) for a, b in pairs]
        t0 = time.perf_counter()
        oracle.vpot(s, pairs=pairs)
        oracle.vgrad_pairs(s, pairs)
        dt = time.perf_counter() - t0
        t_pairs += dt
        n_pairs += k
        if t_pairs >= 0.5 * seconds or n_pairs >= len(pairs_all):
            break
        k = min(len(pairs_all) - n_pairs, max(2 * k, int(k * (0.5 * seconds - t_pairs) / max(dt, 1e-3))))
    t_region1 = t_pairs * npairs / n_pairs

    # moments and multipoles on a shell subset
    nsh = max(2, min(s.nshell, int(round(s.nshell / 6))))
    shells = np.sort(rng.choice(s.nshell, nsh, replace=False))
    sub_s = _shell_subset(s, shells)
    t0 = time.perf_counter()
    M_sub = oracle.multipoles(sub_s)
    t_mult_s = time.perf_counter() - t0
    t_mult = t_mult_s * npairs / (nsh * (nsh + 1) // 2)
    # the Pulay term (moment derivatives, per shell pair) on the same subset, and the QM tensor
    # gradient (per QM atom) on the whole system; their cost does not depend on the values
    phi_r = rng.standard_normal((s.natm, 20))
    t0 = time.perf_counter()
    oracle.pulay_grad(sub_s, phi_r)
    t_pul_s = time.perf_counter() - t0
    t_pulay = t_pul_s * npairs / (nsh * (nsh + 1) // 2)
    t0 = time.perf_counter()
    oracle.tensor_grad_qm(s, M_sub, phi_r)
    t_tg = time.perf_counter() - t0
    del M_sub

    # region-II potential at the QM sites, on a charge subset
    nsub = max(1, min(s.nmm, 1500))
    sub = np.sort(rng.choice(s.nmm, nsub, replace=False))
    t0 = time.perf_counter()
    oracle.ewald_phi(_charge_subset(s, sub))
    t_phi_s = time.perf_counter() - t0
    t_phi = t_phi_s * s.nmm / nsub

    # MM-side Ewald derivatives for a charge subset (multipoles of the full density)
    M = np.zeros((s.natm, 10))
    M[:, 0] = s.atom_Z * 0.1
    nmm_sub = max(1, min(s.nmm, 300))
    t0 = time.perf_counter()
    oracle.ewald_mm(s, M, mm_subset=sub[:nmm_sub])
    t_mm_s = time.perf_counter() - t0
    t_mm = t_mm_s * s.nmm / nmm_sub

    t_step = t_region1 + t_mult + t_pulay + t_tg + t_phi + t_mm
    sampled = t_pairs + t_mult_s + t_pul_s + t_tg + t_phi_s + t_mm_s
    return {"value": units / t_step, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"whole V+forces step estimated from bounded samples ({sampled:.1f} s of oracle time): "
                       f"V + adjoint on {n_pairs} random shell pairs x {nI} region-I charges ({t_region1:.0f} s "
                       f"scaled), moments/multipoles on {nsh} random shells ({t_mult:.1f} s scaled), region-II "
                       f"potential on {nsub} random MM charges ({t_phi:.1f} s scaled), MM-side Ewald derivatives "
                       f"on {nmm_sub} MM charges ({t_mm:.1f} s scaled), the Pulay term on the shell subset "
                       f"({t_pulay:.1f} s scaled) and the QM tensor gradient ({t_tg:.3f} s); FP64, OpenMP"),
            "step_s": t_step,
            "pieces_s": {"region1_v_adjoint": t_region1, "multipoles": t_mult, "pulay": t_pulay,
                         "qm_tensor_gradient": t_tg, "region2_potential": t_phi, "mm_ewald_derivatives": t_mm}}


def run_reference(args):
    """--impl reference: the oracle as the reference arm (host cores), bounded samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    s = make_system(args.config)
    per_step = max(2.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(s, seconds=per_step, seed=i, n_shell_pairs=SCREENED_SHELL_PAIRS.get(args.config))
        if i >= args.warmup:
            vals.append(cb)
    value = float(np.mean([v["value"] for v in vals]))
    import oracle  # noqa: F401
    nI = len(__import__("oracle").region1(s)[0])
    nsp = SCREENED_SHELL_PAIRS.get(args.config)
    # the same workload description and config keys as the GPU arm's line
    workload = (describe(s, {"n_shell_pairs": nsp, "n_region1": nI}) if nsp is not None else
                f"{s.name} ({s.natm} QM atoms, {s.nao} AOs, {s.nmm} MM charges, {nI} region-I)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload, "precision": "fp64",
                      "parallelism": "replicas" if args.gpus > 1 else "single GPU",
                      "units_per_step": (nsp * nI) if nsp is not None else None},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                            "sample": vals[0]["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_batched(args, q, torch, dev, emit=True):
    """Frames workload: 64 uneven frames (QM water clusters of 20-120 atoms, 20k-120k MM charges at
    water density), mixed-precision V + energy + gradient per frame through one recorded CUDA
    graph (qmmm_batch_run), against a loop of plain FP64 calls over the same frames.  Prints the
    JSON line (emit) or returns it (the default run adds it to its own line)."""
    import workloads
    frames = workloads.config5_frames(args.frames)
    n = len(frames)
    hs = [q.Handle(s, precision=q.QMMM_MIXED) for s in frames]
    # tune the largest frame; its measured class weights and block shapes serve every frame
    work = [h.info["n_prim_pairs"] * h.info["n_region1"] for h in hs]
    big = int(np.argmax(work))
    if not args.no_autotune:
        hs[big].autotune()
        for k in (1, 3):
            t = hs[big].tuning(k)
            for i, h in enumerate(hs):
                if i != big:
                    h.set_tuning(k, t["threads"], t["weight"])
    units = [h.info["n_shell_pairs"] * h.info["n_region1"] for h in hs]
    total_units = int(sum(units))
    dm = [torch.as_tensor(np.ascontiguousarray(s.dm), device=dev) for s in frames]
    z = lambda *shape: torch.zeros(shape, dtype=torch.float64, device=dev)  # noqa: E731
    V = [z(s.nao, s.nao) for s in frames]
    E = [z(4) for _ in frames]
    gq = [z(s.natm, 3) for s in frames]
    gm = [z(s.nmm, 3) for s in frames]
    gc = [z(s.nmm) for s in frames]
    stream = torch.cuda.Stream()
    b = q.Batch(hs, stream)
    for _ in range(args.warmup):
        b.run(dm, V, E, gq, gm, gc)
    runs, lat = [], []
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for k in range(args.steps):
            if k == args.steps - 1:  # the last timed batch as an NVTX range ("replay/")
                torch.cuda.nvtx.range_push("replay")
            b.run(dm, V, E, gq, gm, gc)
            if k == args.steps - 1:
                torch.cuda.nvtx.range_pop()
            tot, per = b.timing()
            runs.append(tot)
            lat += per
    ms = float(np.mean(runs))
    captures = b.captures()
    b.close()

    # the same frames through a loop of plain calls (one call at a time, synchronised per call)
    def plain_loop(prec, keep=False):
        out = []
        hh = [q.Handle(s, precision=prec) for s in frames] if prec != q.QMMM_MIXED else hs
        for h in hh:
            h.set_stream(torch.cuda.current_stream())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, h in enumerate(hh):
            Vp, _ = h.vpot(like=dm[i])
            Ep = h.energy(dm[i])
            g = h.forces(dm[i])
            if keep:
                out.append((Vp, Ep, g))
        torch.cuda.synchronize()
        t = (time.perf_counter() - t0) * 1e3
        if prec != q.QMMM_MIXED:
            for h in hh:
                h.close()
        return t, out

    ms_mixed_loop, _ = plain_loop(q.QMMM_MIXED)
    ms_f64_loop, ref = plain_loop(q.QMMM_FP64, keep=True)
    # errors of the batched mixed results against the FP64 loop
    fro = max(float(torch.linalg.norm(V[i] - ref[i][0]) / torch.linalg.norm(ref[i][0])) for i in range(n))
    gerr = 0.0
    for i in range(n):
        for a_, r_ in ((gq[i], ref[i][2][0]), (gm[i], ref[i][2][1]), (gc[i], ref[i][2][2])):
            gerr = max(gerr, float((a_ - r_).abs().max() / r_.abs().max()))
    eerr = max(float(abs(E[i][0] - ref[i][1][0]) / (ref[i][1][1].abs() + ref[i][1][2].abs() + ref[i][1][3].abs()))
               for i in range(n))
    for h in hs:
        h.close()
    lat = np.asarray(lat)
    value = total_units / (ms * 1e-3)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64", "data": "synthetic (seeded TIP3P water boxes + QM water clusters per frame)",
           "config": {"workload": f"frames_c5: {n} frames, QM {min(s.natm for s in frames)}-"
                                  f"{max(s.natm for s in frames)} atoms, {min(s.nmm for s in frames)}-"
                                  f"{max(s.nmm for s in frames)} MM charges, cutoff 12 A, alpha 0.3 A^-1",
                      "precision": "mixed", "units_per_step": total_units,
                      "l2": "inputs of all frames exceed L2 (129 MB)",
                      "graph": f"one CUDA graph per batch ({captures} recording(s))",
                      "sweep_schedule": "autotuned on the largest frame" if not args.no_autotune else "flop model"},
           "batched": {"ms_per_batch": ms, "frame_latency_ms_p50": float(np.percentile(lat, 50)),
                       "frame_latency_ms_p99": float(np.percentile(lat, 99)),
                       "fp64_loop_ms": ms_f64_loop, "fp64_loop_value": total_units / (ms_f64_loop * 1e-3),
                       "speedup_vs_fp64_loop": ms_f64_loop / ms, "mixed_loop_ms": ms_mixed_loop,
                       "rel_fro_err_V_max_frame": fro, "max_rel_err_forces": gerr, "max_rel_err_E": eerr},
           "clocks": clk.summary()}
    if not emit:
        return out
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c4", choices=["c1", "c2", "c4", "c5"])
    ap.add_argument("--frames", type=int, default=64, help="frames of the c5 (batched) workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the uneven-frames batch that the default run adds to its line")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-autotune", action="store_true", help="run the class sweeps with the flop-model schedule")
    ap.add_argument("--recip", default="auto", choices=["auto", "cuda", "tensor"],
                    help="reciprocal Ewald sums: auto (= tensor), CUDA cores, or tensor cores")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    import paper_2408_03273_gb300 as q

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    args.warmup = max(3, args.warmup)
    if args.config == "c5":
        return run_batched(args, q, torch, dev)

    s = make_system(args.config)
    prec = q.QMMM_MIXED if args.precision == "mixed" else q.QMMM_FP64
    h = q.Handle(s, precision=prec)
    stream = torch.cuda.current_stream()
    h.set_stream(stream)
    info = h.info
    tuning = {}

    RECIP = {"auto": q.QMMM_RECIP_AUTO, "cuda": q.QMMM_RECIP_CUDA_CORES, "tensor": q.QMMM_RECIP_TENSOR}[args.recip]
    RECIP_NAME = {q.QMMM_RECIP_CUDA_CORES: "CUDA cores (FP64; double-float on the mixed path)",
                  q.QMMM_RECIP_TENSOR: "tensor cores (BF16 products of exact 7-bit digit planes, FP64 class)"}

    def recip_in_effect(precision):
        if RECIP != q.QMMM_RECIP_AUTO:
            name = RECIP_NAME[RECIP]
        else:
            work = (s.kmax[0] + 1) * (2 * s.kmax[1] + 1) * (2 * s.kmax[2] + 1) * s.nmm
            name = RECIP_NAME[q.QMMM_RECIP_TENSOR if work >= 4e7 else q.QMMM_RECIP_CUDA_CORES]
        if precision == q.QMMM_MIXED and name == RECIP_NAME[q.QMMM_RECIP_TENSOR]:
            name = "tensor cores (BF16 products of exact 7-bit digit planes; structure factor FP64 class, MM side 34-bit)"
        return name

    def positions_ms(hh, n=10):
        # set_positions alone (region I and the region-II potential, i.e. the structure factor)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * n)]
        for k in range(n):
            ev[2 * k].record(stream)
            q.qmmm_set_positions(hh.h, qm_d, mm_d, q_d)
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        return float(np.median([ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(n)]))

    h.set_recip_method(RECIP)

    def tune(hh):
        # one-time plan step outside the timed region: block shape and SM split per angular class
        if args.no_autotune:
            return
        hh.autotune()
        for k in range(4):
            t = hh.tuning(k)
            if t["tuned"]:
                tuning[q.SWEEP_KINDS[k]] = {"threads": t["threads"], "share": t["share"]}

    tune(h)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa: E731
    qm_d, mm_d, q_d, dm_d = t(s.atom_xyz), t(s.mm_xyz), t(s.mm_q), t(s.dm)
    nao, natm, nmm = s.nao, s.natm, s.nmm
    V_d = torch.empty((nao, nao), dtype=torch.float64, device=dev)
    En_d, EII_d = torch.empty(1, dtype=torch.float64, device=dev), torch.empty(1, dtype=torch.float64, device=dev)
    M_d = torch.empty((natm, 10), dtype=torch.float64, device=dev)
    gq_d = torch.empty((natm, 3), dtype=torch.float64, device=dev)
    gm_d = torch.empty((nmm, 3), dtype=torch.float64, device=dev)
    gc_d = torch.empty((nmm,), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(hh, qm, mm, qq, dm, V, En, EII, M, gq, gm, gc, rec=None):
        q.qmmm_set_positions(hh.h, qm, mm, qq)
        q.qmmm_vpot(hh.h, V, En)
        if rec is not None:
            rec["vpot"].append(hh.last_timing()[0])
        q.qmmm_ewald(hh.h, dm, EII, M, None)
        q.qmmm_forces(hh.h, dm, gq, gm, gc)
        if rec is not None:
            rec["grad"].append(hh.last_timing()[0])

    def timed(hh, K, W):
        for _ in range(W):
            step(hh, qm_d, mm_d, q_d, dm_d, V_d, En_d, EII_d, M_d, gq_d, gm_d, gc_d)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        rec = {"vpot": [], "grad": []}
        total = 0.0
        for k in range(K):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if k == K - 1:  # the last timed step as an NVTX range (for ncu --nvtx-include "step/")
                torch.cuda.nvtx.range_push("step")
            e0.record(stream)
            step(hh, qm_d, mm_d, q_d, dm_d, V_d, En_d, EII_d, M_d, gq_d, gm_d, gc_d, rec)
            e1.record(stream)
            e1.synchronize()
            if k == K - 1:
                torch.cuda.nvtx.range_pop()
            total += e0.elapsed_time(e1)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return total / K, rec

    units_per_step = info["n_shell_pairs"] * info["n_region1"]
    with Clocks(local) as clk:
        ms, rec = timed(h, args.steps, args.warmup)
    ms = max_over_ranks(ms, dist, dev)
    value = job_rate(world, units_per_step, ms)

    # dominant kernel (region-I sweep) against the plain-ALU roofline
    t_v, t_g = float(np.mean(rec["vpot"])), float(np.mean(rec["grad"]))
    dom_adj = t_g >= t_v
    fl = sweep_flops(info, dom_adj)
    achieved = fl / ((t_g if dom_adj else t_v) * 1e-3) / 1e12
    peak = FP64_PEAK_TFLOPS if prec == q.QMMM_FP64 else FP32_PEAK_TFLOPS
    roof = {"kernel": "vgrad (region-I adjoint sweep)" if dom_adj else "vpot (region-I sweep)",
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": SWEEP_TRAFFIC.get((args.config, args.precision)) if dom_adj else None,
            "traffic_note": "DRAM bytes per adjoint sweep (all angular-class kernels), ncu capture",
            "kernel_ms": t_g if dom_adj else t_v, "other_sweep_ms": t_v if dom_adj else t_g,
            "peak_note": ("FP64 plain-ALU peak from the unit counts at 2070 MHz (152 SMs x 2 DFMA/clk)"
                          if prec == q.QMMM_FP64 else "FP32 plain-ALU peak at 2070 MHz (152 SMs x 128 FFMA/clk)"),
            "flops_per_launch": fl}

    # launches of our kernels per step (a claim; the ncu launch list of this command confirms the
    # composition).  Per call:
    #   set_positions: gather, region-I count/scan/fill, real-space pre-filter inputs, real-space,
    #     region-I tensors, background sum, QM-site reciprocal, final = 10 (mixed path: + the
    #     double-float g(G) S(G) table),
    #     plus the structure factor (tensor cores: max|q|, phases, B planes, MMA, reduction = 5;
    #     CUDA cores: kernel + slice sum = 2)
    #   vpot: one kernel per class and charge chunk + nuclear-MM term and its sum
    #   ewald: one moments kernel per class + the energy terms
    #   forces: two moments kernels per class (Pulay) + the adjoint sweep per class and chunk
    #     (mixed path: pair records, charge-lane sweep, pair gradients = 3 per class and chunk)
    #     + 8 fixed (nuclear-MM, sum, real space, region I, background, tensor
    #     gradient, scatter, unpermute) + the MM-side reciprocal sum (tensor cores: atom phases,
    #     multipole structure factor, phases, scales, B planes per N tile, MMA = 5 + tiles; CUDA
    #     cores: 3)
    # vpot adds one V slice-sum kernel when its classes split their charges (per-class slices:
    # 256 or more region-I charges and room for two partial matrices in 512 MB; or small systems
    # whose classes ask for less than half the SMs, which have fewer charges than that here).
    def launches_per_step(precision):
        ncls = sum(1 for n in info["n_prim_pairs_class"] if n > 0)
        nI = info["n_region1"]
        v_maxsl = min(8, min(nI, 4096) // 128, (512 << 20) // max(1, 8 * s.nao * s.nao))
        ch_f = math.ceil(nI / 4096) if nI else 0
        ch_g = math.ceil(nI / 2560) if nI else 0
        tensor = recip_in_effect(precision).startswith("tensor cores")
        # MM-side tiling as the library plans it (N rows per tile <= 96 with the FP64 path's five
        # accumulators, <= 160 with the mixed path's three); the sum stays on the CUDA cores if
        # 2 kz + 1 < 8
        kx, lim = s.kmax[0] + 1, (96 if precision == q.QMMM_FP64 else 160)
        cpt = next((c for c in (3, 2, 1) if 2 * c * kx <= lim), 1)
        mm_tc = tensor and (2 * cpt * kx + 15) // 16 * 16 <= lim and 2 * s.kmax[2] + 1 >= 8
        mm_tiles = -(-3 // cpt)
        sweep_g = ncls * ch_g * (3 if precision == q.QMMM_MIXED else 1)
        mixed = precision == q.QMMM_MIXED
        return (10 + (1 if mixed else 0) + (5 if tensor else 2)) + (ncls * ch_f + 2 + (1 if v_maxsl > 1 else 0)) + (ncls + 1) + \
            (2 * ncls + sweep_g + 8 + ((5 + mm_tiles) if mm_tc else 3))

    per_step = launches_per_step(prec)
    launches = per_step * args.steps

    # mixed precision beside FP64 (same GPU, same inputs), with its error against FP64
    mixed = None
    if not args.no_mixed and prec == q.QMMM_FP64:
        V64, gq64, gm64, gc64 = V_d.clone(), gq_d.clone(), gm_d.clone(), gc_d.clone()
        E64 = h.energy(dm_d).clone()
        hm = q.Handle(s, precision=q.QMMM_MIXED)
        hm.set_stream(stream)
        hm.set_recip_method(RECIP)
        tune(hm)
        ms_m, rec_m = timed(hm, args.steps, args.warmup)
        Em = hm.energy(dm_d)
        fro = float(torch.linalg.norm(V_d - V64) / torch.linalg.norm(V64))
        # raw max-relative error of each gradient: max |mixed - FP64| / max |FP64|
        raw = {"dE_dRqm": float((gq_d - gq64).abs().max() / gq64.abs().max()),
               "dE_dRmm": float((gm_d - gm64).abs().max() / gm64.abs().max()),
               "dE_dq": float((gc_d - gc64).abs().max() / gc64.abs().max())}
        gerr = max(raw.values())
        escale = float(E64[1].abs() + E64[2].abs() + E64[3].abs())
        t_vm, t_gm = float(np.mean(rec_m["vpot"])), float(np.mean(rec_m["grad"]))
        flm = sweep_flops(info, t_gm >= t_vm)
        ach_m = flm / (max(t_gm, t_vm) * 1e-3) / 1e12
        ms_m = max_over_ranks(ms_m, dist, dev)
        mixed = {"value": job_rate(world, units_per_step, ms_m), "ms_per_step": ms_m,
                 "speedup_vs_fp64": ms / ms_m, "vpot_sweep_ms": t_vm, "adjoint_sweep_ms": t_gm,
                 "rel_fro_err_V": fro, "max_rel_err_forces": gerr, "max_rel_err_forces_raw": raw,
                 "rel_err_E": float(abs(Em[0] - E64[0]) / escale),
                 "rel_err_E_raw": float(abs(Em[0] - E64[0]) / abs(E64[0])),
                 "gpu_launches_per_step": launches_per_step(q.QMMM_MIXED),
                 "roofline": {"bound": "alu", "achieved": ach_m, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                              "frac": ach_m / FP32_PEAK_TFLOPS,
                              "traffic": SWEEP_TRAFFIC.get((args.config, "mixed")) if t_gm >= t_vm else None}}
        # the region-II potential by each structure-factor method (set_positions alone)
        pos = {}
        for name, m in (("cuda_cores", q.QMMM_RECIP_CUDA_CORES), ("tensor_cores", q.QMMM_RECIP_TENSOR)):
            hm.set_recip_method(m)
            positions_ms(hm, 3)
            pos[name] = positions_ms(hm)
        hm.set_recip_method(RECIP)
        mixed["reciprocal_sums"] = recip_in_effect(q.QMMM_MIXED)
        mixed["set_positions_ms"] = pos
        hm.close()

    # end to end: host (pinned) inputs and outputs, copies inside the timed interval
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).pin_memory()  # noqa: E731
    qm_h, mm_h, q_h, dm_h = pin(s.atom_xyz), pin(s.mm_xyz), pin(s.mm_q), pin(s.dm)
    V_h = torch.empty((nao, nao), dtype=torch.float64).pin_memory()
    En_h, EII_h = torch.empty(1, dtype=torch.float64).pin_memory(), torch.empty(1, dtype=torch.float64).pin_memory()
    M_h = torch.empty((natm, 10), dtype=torch.float64).pin_memory()
    gq_h = torch.empty((natm, 3), dtype=torch.float64).pin_memory()
    gm_h = torch.empty((nmm, 3), dtype=torch.float64).pin_memory()
    gc_h = torch.empty((nmm,), dtype=torch.float64).pin_memory()
    for _ in range(2):
        step(h, qm_h, mm_h, q_h, dm_h, V_h, En_h, EII_h, M_h, gq_h, gm_h, gc_h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ne = max(3, args.steps // 2)
    for _ in range(ne):
        step(h, qm_h, mm_h, q_h, dm_h, V_h, En_h, EII_h, M_h, gq_h, gm_h, gc_h)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks((time.perf_counter() - t0) * 1e3 / ne, dist, dev)
    h2d = 8 * (3 * natm + 3 * nmm + nmm + 2 * nao * nao)  # positions, charges, density (ewald + forces)
    d2h = 8 * (nao * nao + 1 + 1 + 10 * natm + 3 * natm + 3 * nmm + nmm)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if prec == q.QMMM_FP64 else "f32+f64",
           "data": "synthetic (seeded TIP3P water box + random active-site QM region and basis)",
           "config": {"workload": describe(s, info), "precision": args.precision,
                      "reciprocal_sums": recip_in_effect(prec),
                      "l2": "flushed before every timed step (256 MiB write, outside the timed interval)",
                      "parallelism": "replicas" if world > 1 else "single GPU",
                      "units_per_step": units_per_step,
                      "prim_pairs_per_class": dict(zip(["ss", "ps", "pp", "ds", "dp", "dd", "fs", "fp", "fd", "ff"],
                                                       info["n_prim_pairs_class"])),
                      "sweep_schedule": ("flop-model SM split, 256-thread blocks" if args.no_autotune else
                                         {"autotuned": tuning})},
           "roofline": roof, "gpu_launches": launches, "clocks": clk.summary(),
           "e2e": {"value": job_rate(world, units_per_step, ms_e2e), "unit": UNIT, "ms_per_step": ms_e2e,
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}}
    if mixed:
        out["mixed"] = mixed
    if info["n_shell_pairs"] != SCREENED_SHELL_PAIRS.get(args.config, info["n_shell_pairs"]):
        out["config"]["note"] = "screened shell-pair count differs from the reference arm's table"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(s, seconds=16.0, n_shell_pairs=info["n_shell_pairs"])
    h.close()
    if args.config == "c4" and world == 1 and not args.no_batched and not args.no_mixed:
        # the batching pattern on its workload (64 uneven frames through one recorded graph, mixed
        # precision) beside the headline, so every default run measures it too
        import copy
        bargs = copy.copy(args)
        bargs.steps, bargs.warmup = 3, 3
        bt = run_batched(bargs, q, torch, dev, emit=False)
        out["batched"] = {"workload": bt["config"]["workload"], "value": bt["value"], "unit": UNIT,
                          "units_per_batch": bt["config"]["units_per_step"], "steps": 3, "warmup": 3,
                          **bt["batched"], "clocks": bt["clocks"]}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
