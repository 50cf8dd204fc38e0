#!/usr/bin/env python3
"""Benchmark of the DF J/K hot path on GB300.

One step = one SCF-like iteration of the paper's method on one synthetic
molecule: the FP64 Coulomb build (rho, J), the exchange build with both
contractions emulated over INT8 slices, and the energies.  Every timed step
runs a fixed slice count, by default 5, Table 1's level-2 count and the first
level whose emulation meets max|dK| <= 1e-10 max|K|; every run checks that
gate against the CPU oracle's K, J and energies (all auxiliary blocks) and
against the native-FP64 build of the same K on the same GPU.

metric: effective FP64 TFLOP/s of the exchange build, F_K = 4 nao^2 naux nocc
(the paper's FLOP model with dense B, Section 3.1) per step, divided by the
step time.  The default workload is the 240-atom molecule (nao 1200, naux
3600, nocc 250; B is 41.5 GB), far larger than L2, so no flush is needed
between steps.

Usage: python bench.py [--gpus N --steps K --warmup W --impl ours|reference
                        --workload large|medium|profile|small|batch|sequence|predictor|scf|crt
                        --nslices S --aux-blocks N --cluster-pairs 0|1|2]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "DF K-build effective FP64 TFLOP/s, INT8-adaptive vs native FP64, max|dK|<=1e-10"
UNIT = "TFLOP/s"
LAUNCHES_PER_STEP = 11     # rho, coulomb, 2 density-change kernels, split C, GEMM1, split X, GEMM2, reduce,
                           # 2 energy kernels
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["small", "profile", "medium", "large", "chain", "batch", "sequence",
                                           "predictor", "scf", "crt"],
                    default="large")
    ap.add_argument("--size", choices=["small", "profile", "medium", "large"], default=None,
                    help="molecule of the sequence / predictor evaluation (default: medium; predictor: large)")
    ap.add_argument("--train-molecules", type=int, default=200)
    ap.add_argument("--batch-size", type=int, default=48)
    ap.add_argument("--nslices", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-records", action="store_true",
                    help="skip the sequence, sweep and batch records that follow the timed steps")
    ap.add_argument("--aux-blocks", type=int, default=0,
                    help="keep only the first N 128-function auxiliary blocks of the workload (a smaller case of "
                         "the same kernels, for profiling); 0 keeps them all")
    ap.add_argument("--jk-overlap", type=int, choices=[0, 1, 2, 3, 4], default=4,
                    help="CTAs per SM of rho and J beside the X split in the J + K build (df_build_JK); "
                         "0 runs J, then K, in one stream")
    ap.add_argument("--cluster-pairs", type=int, choices=[0, 1, 2], default=1,
                    help="slice GEMMs on CTA pairs (cta_group::2): 0 never, 1 the first GEMM, 2 both GEMMs")
    return ap.parse_args()


def workload(name):
    from paper_2601_08077_gb300 import inputs
    return {"small": inputs.SMALL, "profile": inputs.PROFILE, "medium": inputs.MEDIUM,
            "large": inputs.LARGE, "chain": inputs.CHAIN}[name]


def flops_K(w):
    return 4.0 * w.nao ** 2 * w.naux * w.nocc


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return FALLBACK_PEAKS, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "df_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_reference(B, C, D, w):
    """The oracle as it stands, on the host cores, over every 128-function
    auxiliary block of the workload: the exchange build of the block's B_P
    (Eqs. df-k-1/2), its rho_P (Eq. df-j-1) and its share of J (Eq. df-j-2).
    K and J are the FP64 sums over blocks, the accuracy reference of the run.
    The exchange part is timed for cpu_baseline (about 8 s for the 240-atom
    molecule on 16 cores).  B may live on the device; each block is copied to
    the host first (not timed)."""
    from oracle import df_oracle as O
    cores = len(os.sched_getaffinity(0))
    nblk = (w.naux + 127) // 128
    K = np.zeros((w.nao, w.nao))
    J = np.zeros((w.nao, w.nao))
    rho = np.empty(w.naux)
    t_total, flops = 0.0, 0.0
    for b in range(nblk):
        p0, p1 = b * 128, min(w.naux, b * 128 + 128)
        Bb = B[p0:p1]
        Bb = Bb.cpu().numpy() if hasattr(Bb, "cpu") else Bb
        t0 = time.perf_counter()
        Kb = O.exchange(Bb, C)
        t_total += time.perf_counter() - t0
        flops += 4.0 * w.nao ** 2 * (p1 - p0) * w.nocc
        K += Kb
        rho[p0:p1] = O.rho(Bb, D)
        J += O.coulomb(Bb, rho[p0:p1])
    base = {"value": flops / t_total / 1e12, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "oracle FP64 exchange build (NumPy, Eqs. df-k-1/2) of all %d auxiliary blocks "
                      "(%d functions) of the %s workload, %.1f s" % (nblk, w.naux, w.name, t_total)}
    return base, K, J, rho


def oracle_gate(K_gpu, J_gpu, E_gpu, K_ref, J_ref, D):
    """Errors of the run's K (at the timed slice count), J and E_J + E_K against the
    oracle's, and the gate of the metric: max|dK| <= 1e-10 max|K| and |dE| <= 1e-9 Eh."""
    from oracle import df_oracle as O
    EJ, EK = O.energies(D, J_ref, K_ref)
    dK = float(np.max(np.abs(K_gpu - K_ref)) / np.max(np.abs(K_ref)))
    dJ = float(np.max(np.abs(J_gpu - J_ref)) / np.max(np.abs(J_ref)))
    dE = abs((E_gpu[0] + E_gpu[2]) - (EJ + EK))
    return {"max_dK_rel_vs_oracle": dK, "max_dJ_rel_vs_oracle": dJ, "dE_vs_oracle": dE,
            "dEJ_vs_oracle": abs(E_gpu[0] - EJ), "dEK_vs_oracle": abs(E_gpu[2] - EK),
            "E_oracle": EJ + EK, "gate_vs_oracle": bool(dK <= 1e-10 and dE <= 1e-9)}


def run_reference(args, w):
    """--impl reference: the CPU oracle, timed per step on a bounded sample."""
    from oracle import df_oracle as O
    from paper_2601_08077_gb300 import inputs
    nblk = max(1, min((w.naux + 127) // 128, 2))
    mol = inputs.molecule(w.n_atoms, w.seed)
    B = inputs.df_tensor_rows(mol, nblk * 128)       # only the sampled blocks are formed
    C = inputs.orbitals(mol.nao, w.nocc, w.seed + 1)
    cores = len(os.sched_getaffinity(0))

    def step():
        p1 = min(w.naux, nblk * 128)
        O.exchange(B[:p1], C)
        return 4.0 * w.nao ** 2 * p1 * w.nocc

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    fl = sum(step() for _ in range(args.steps))
    dt = time.perf_counter() - t0
    v = fl / dt / 1e12
    sample = "oracle FP64 exchange build of the first %d auxiliary blocks of %s per step" % (nblk, w.name)
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": w.name, "nao": w.nao, "naux": w.naux, "nocc": w.nocc, "parallelism": "replicas"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_batch(args):
    """Grouped batch: molecules of 30..120 atoms (nao 150..600, naux 3 nao, nocc nao/5), all
    exchange builds in grouped persistent launches captured as one CUDA graph, against one
    native-FP64 build per molecule on the same GPU."""
    import torch
    from paper_2601_08077_gb300 import build
    build.build_all()
    torch.cuda.set_device(0)
    return batch_record(args.batch_size, args.nslices, args.steps, args.warmup)


def batch_record(n_mol, s, steps, warmup):
    import types
    import torch
    from paper_2601_08077_gb300 import df, inputs
    args = types.SimpleNamespace(steps=steps, warmup=warmup)
    ws = inputs.batch_workloads(n_mol)
    t0 = time.perf_counter()
    ctxs, Bs, Cs, Ds = [], [], [], []
    for w in ws:
        mol = inputs.molecule(w.n_atoms, w.seed)
        B = inputs.df_tensor_device(mol)
        C = inputs.orbitals(mol.nao, w.nocc, w.seed + 1)
        ctx = df.Context(mol.nao, mol.naux, w.nocc, s_max=s)
        ctx.setup(B)
        ctxs.append(ctx)
        Bs.append(B)
        Cs.append(torch.from_numpy(C).cuda())
        Ds.append(torch.from_numpy(inputs.density(C)).cuda())
    gen_s = time.perf_counter() - t0
    Ks = [torch.empty((c.nao, c.nao), dtype=torch.float64, device="cuda") for c in ctxs]
    Js = [torch.empty_like(k) for k in Ks]
    batch = df.Batch(ctxs)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        choice = batch.autotune(Cs, s, Ks)
        for _ in range(args.warmup):
            batch.build_J(Ds, Js)
            batch.build_K(Cs, s, Ks)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        with Clocks(0) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                batch.build_J(Ds, Js)
                batch.build_K(Cs, s, Ks)
            e1.record(stream)
            stream.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    FK = sum(4.0 * w.nao ** 2 * w.naux * w.nocc for w in ws)
    # accuracy of the batch against the FP64 build, and the FP64 builds' time (one per molecule)
    worst = 0.0
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    K64 = [torch.empty_like(k) for k in Ks]
    f0.record()
    for ctx, C, K in zip(ctxs, Cs, K64):
        ctx.build_K(C, 0, K)
    f1.record()
    torch.cuda.synchronize()
    ms64 = f0.elapsed_time(f1)
    for K, K0 in zip(Ks, K64):
        worst = max(worst, float((K - K0).abs().max() / K0.abs().max()))
    return {"metric": "batched DF J/K builds, molecules/s and effective FP64 TFLOP/s", "value": FK / (ms * 1e-3) / 1e12,
            "unit": UNIT, "molecules_per_s": len(ws) / (ms * 1e-3), "n_molecules": len(ws), "ms_per_batch": ms,
            "steps": args.steps, "warmup": args.warmup, "nslices": s, "autotune": {"ksplit_cap": choice[0],
                                                                                 "order": choice[1],
                                                                                 "gemm1_tile": "256x128 CTA pair"
                                                                                 if choice[2] else "128x128"},
            "fp64_per_molecule": {"ms_per_batch": ms64, "tflops": FK / (ms64 * 1e-3) / 1e12,
                                  "molecules_per_s": len(ws) / (ms64 * 1e-3)},
            "max_dK_rel_vs_fp64": worst, "generation_s": gen_s,
            "config": {"workload": "batch-%d-molecules-30to120-atoms" % len(ws), "nao": [w.nao for w in ws],
                       "naux_per_nao": 3, "nocc": "nao/5"},
            "clocks": clk.summary()}


def sweep_record(reps=10):
    """The fixed-slice sweep on the 120-atom molecule (nao 600, naux 1800, nocc 120): K at 3..8
    slices per operand, throughput per count, max|dK| against the native FP64 build, |dE|
    against FP64, and J against the CPU oracle (J does not depend on the count)."""
    import torch
    from oracle import df_oracle as O
    from paper_2601_08077_gb300 import df, inputs
    w = inputs.MEDIUM
    mol = inputs.molecule(w.n_atoms, w.seed)
    ctx = df.Context(w.nao, w.naux, w.nocc)
    Bg = ctx.setup_integrals(torch.from_numpy(inputs.int3c(mol)).cuda(), torch.from_numpy(inputs.metric(mol)).cuda())
    C = inputs.orbitals(mol.nao, w.nocc, w.seed + 1)
    D = inputs.density(C)
    Cg, Dg = torch.from_numpy(C).cuda(), torch.from_numpy(D).cuda()
    J, rho = ctx.build_J(Dg)
    K64 = ctx.build_K(Cg, 0)[0].clone()
    E64 = ctx.energy(Dg, J, K64, rho)
    kmax = float(K64.abs().max())
    Jh = J.cpu().numpy()
    J_ref = np.zeros_like(Jh)
    for p0 in range(0, w.naux, 128):
        Bb = Bg[p0:p0 + 128].cpu().numpy()
        J_ref += O.coulomb(Bb, O.rho(Bb, D))
    rows = []
    for s in range(3, 9):
        K = ctx.build_K(Cg, s)[0]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            ctx.build_K(Cg, s, K)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        E = ctx.energy(Dg, J, K, rho)
        rows.append({"slices": s, "k_build_ms": ms, "tflops": flops_K(w) / (ms * 1e-3) / 1e12,
                     "max_dK_rel_vs_fp64": float((K - K64).abs().max()) / kmax,
                     "dE_vs_fp64": abs((E[0] + E[2]) - (E64[0] + E64[2]))})
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    ctx.build_K(Cg, 0, K64)
    f1.record()
    torch.cuda.synchronize()
    ms64 = f0.elapsed_time(f1)
    return {"workload": w.name, "per_slice_count": rows,
            "max_dJ_rel_vs_oracle": float(np.max(np.abs(Jh - J_ref)) / np.max(np.abs(J_ref))),
            "fp64_native": {"k_build_ms": ms64, "tflops": flops_K(w) / (ms64 * 1e-3) / 1e12}}


def _molecule_on_device(w, order=False):
    import torch
    from paper_2601_08077_gb300 import df, inputs, predictor
    mol = inputs.molecule(w.n_atoms, w.seed)
    B = inputs.df_tensor_device(mol)
    C = inputs.orbitals(mol.nao, w.nocc, w.seed + 1)
    ctx = df.Context(mol.nao, mol.naux, w.nocc)
    ctx.setup(B, perm=predictor.magnitude_order(B) if order else None)
    return ctx, B, C


def run_sequence(args):
    """The 15-iteration SCF-like sequence under the Table 1 rule, against an all-FP64 sequence."""
    import torch
    from paper_2601_08077_gb300 import build, sequence
    build.build_all()
    torch.cuda.set_device(0)
    w = workload(args.size or "medium")
    ctx, B, C = _molecule_on_device(w)
    orbs = sequence.orbital_sequence(C, 15, w.seed)
    return sequence_record(ctx, w, orbs, full_fp64=True)


def sequence_record(ctx, w, orbs, full_fp64=True):
    """Rule (level 0 in FP64), rule with level 0 as 8 slices, and all-FP64 along the sequence.
    full_fp64 False compares with FP64 at the last iteration only and times the FP64
    sequence as one native iteration times the iteration count."""
    from paper_2601_08077_gb300 import sequence
    cache = {}
    cmp = True if full_fp64 else "last"
    sequence.run(ctx, orbs[:2], compare_fp64=False)     # warm-up
    rule = sequence.run(ctx, orbs, fp64_cache=cache, compare_fp64=cmp)
    rule8 = sequence.run(ctx, orbs, level0_slices=8, fp64_cache=cache, compare_fp64=cmp)
    if full_fp64:
        fp64 = sequence.run(ctx, orbs, mode="fp64", compare_fp64=False)
        t_fp64 = sum(r["ms"] for r in fp64)
        fp64_how = "measured, every iteration"
    else:
        one = sequence.run(ctx, orbs[:1], mode="fp64", compare_fp64=False)
        t_fp64 = one[0]["ms"] * len(orbs)
        fp64_how = "one native-FP64 iteration (J + K + energies) measured, times %d" % len(orbs)
    t_rule = sum(r["ms"] for r in rule)
    t_rule8 = sum(r["ms"] for r in rule8)
    FK = flops_K(w) * len(orbs)
    return {"metric": "adaptive-precision DF sequence (15 iterations, J + K + energies per iteration)",
            "workload": w.name, "ms_total_rule": t_rule, "ms_total_fp64": t_fp64, "fp64_timing": fp64_how,
            "speedup": t_fp64 / t_rule, "effective_tflops_rule": FK / (t_rule * 1e-3) / 1e12,
            "level0_as_8_slices": {"ms_total": t_rule8, "speedup": t_fp64 / t_rule8,
                                   "effective_tflops": FK / (t_rule8 * 1e-3) / 1e12,
                                   "levels": [r["level"] for r in rule8],
                                   "slices": [r["slices"][0] for r in rule8],
                                   "dE_vs_fp64_final": rule8[-1]["dE_vs_fp64"],
                                   "max_dK_rel_final": rule8[-1]["max_dK_rel"]},
            "levels": [r["level"] for r in rule], "slices": [r["slices"][0] for r in rule],
            "ms_per_iteration": [round(r["ms"], 3) for r in rule],
            "max_dK_rel": [r.get("max_dK_rel") for r in rule], "dE_vs_fp64": [r.get("dE_vs_fp64") for r in rule],
            "density_change": [r["dnorm"] for r in rule], "E_final": rule[-1]["E"],
            "E_fp64_final": rule[-1]["E_fp64"]}


def run_predictor(args):
    """The learned part as specified: a network trained on generated molecules of nao 100-600
    (labels from the method against FP64: per level, the per-block counts with the fewest
    slice pairs whose summed block errors stay within the rule's), then the 240-atom
    sequence run by the library's learned mode (prediction, low-confidence fallback,
    FP64-free bound check and recompute) against the same sequence under the rule."""
    import torch
    from paper_2601_08077_gb300 import build, inputs, predictor, sequence
    build.build_all()
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    Fs, ys = [], []
    opt_pairs, rule_pairs = 0, 0
    ws = inputs.training_workloads(args.train_molecules)
    for w in ws:
        ctx, B, C = _molecule_on_device(w, order=True)
        F, y, err, kmax = predictor.molecule_dataset(ctx, torch.from_numpy(C).cuda(), seed=w.seed)
        Fs.append(F)
        ys.append(y)
        nb = err.shape[0]
        for lv, (tau, s_rule) in predictor.LEVELS.items():
            rule_pairs += nb * predictor.pairs(s_rule)
            opt_pairs += sum(predictor.pairs(int(s)) for s in predictor.labels_at_rule_accuracy(err, s_rule))
        del ctx, B
        torch.cuda.empty_cache()
    F = torch.cat(Fs)
    y = torch.cat(ys)
    t_data = time.perf_counter() - t0
    p = predictor.SlicePredictor(seed=0)
    t0 = time.perf_counter()
    hist = p.fit(F, y, steps=3000, lr=3e-3, batch=512)
    t_train = time.perf_counter() - t0
    acc = float((p.mlp.forward(F).argmax(1).to(torch.int32) == y).float().mean())
    w = workload(args.size or "large")
    ctx, B, C = _molecule_on_device(w, order=True)
    orbs = sequence.orbital_sequence(C, 15, w.seed)
    cache = {}
    sequence.run(ctx, orbs[:2], compare_fp64=False)     # warm-up
    rule = sequence.run(ctx, orbs, fp64_cache=cache)
    p.attach(ctx)
    sequence.run(ctx, orbs[:2], mode="learned", compare_fp64=False)
    learned = sequence.run(ctx, orbs, mode="learned", fp64_cache=cache)
    per_it = [{"level": a["level"], "pairs_rule": a["slice_pairs"], "pairs_learned": b["slice_pairs"],
               "slices_learned": b["slices"], "recomputed": b["recomputed"], "low_confidence": b["low_confidence"],
               "bound_ratio": b["bound_ratio"], "ms_rule": a["ms"], "ms_learned": b["ms"],
               "max_dK_rel_rule": a.get("max_dK_rel"), "max_dK_rel_learned": b.get("max_dK_rel")}
              for a, b in zip(rule, learned)]
    return {"metric": "learned per-block slice counts vs the Table 1 rule (240-atom sequence)",
            "train_molecules": len(ws), "train_nao": [min(x.nao for x in ws), max(x.nao for x in ws)],
            "train_samples": int(F.shape[0]), "train_seconds": t_train, "data_seconds": t_data,
            "loss_first_last": [hist[0], hist[-1]], "train_accuracy": acc,
            "train_label_pairs_vs_rule": [opt_pairs, rule_pairs],
            "eval_workload": w.name,
            "slice_pairs": {"learned": sum(r["slice_pairs"] for r in learned),
                            "rule": sum(r["slice_pairs"] for r in rule)},
            "recomputed_blocks": sum(r["recomputed"] for r in learned),
            "low_confidence_blocks": sum(r["low_confidence"] for r in learned),
            "ms_learned": sum(r["ms"] for r in learned), "ms_rule": sum(r["ms"] for r in rule),
            "dE_vs_fp64_final": {"learned": learned[-1]["dE_vs_fp64"], "rule": rule[-1]["dE_vs_fp64"]},
            "max_dK_rel_worst": {"learned": max(r["max_dK_rel"] for r in learned if r["slices"][0]),
                                 "rule": max(r["max_dK_rel"] for r in rule if r["slices"][0])},
            "iterations": per_it}


def run_scf(args):
    """RHF to convergence on the neutral He cluster of the chosen size, the
    exchange precision chosen by the Table 1 rule (level 0 in FP64, and level 0
    as 8 slices), against the same SCF with every K in native FP64, and with
    every K at level 4's 3 slices (whose energy error floor the rule avoids)."""
    import torch
    from paper_2601_08077_gb300 import build, df, inputs, scf
    build.build_all()
    torch.cuda.set_device(0)
    w = workload(args.size or "medium")
    mol = inputs.molecule(w.n_atoms, w.seed)
    Z = inputs.nuclear_charges(mol)
    S, T, V, En = inputs.one_electron(mol, Z)
    h = T + V
    nocc = mol.n_atoms
    ctx = df.Context(mol.nao, mol.naux, nocc)
    if mol.n_atoms >= 120:
        # the library forms B from the integrals on the device (Cholesky + triangular solve)
        Tg = torch.from_numpy(inputs.int3c(mol)).cuda()
        Vg = torch.from_numpy(inputs.metric(mol)).cuda()
        Bg = ctx.setup_integrals(Tg, Vg)
        del Vg
    else:
        Bg = inputs.df_tensor_device(mol)
        ctx.setup(Bg)
    runs = {}
    for name, kw in (("fp64", {"mode": "fp64"}), ("rule", {"mode": "rule"}),
                     ("rule_level0_8_slices", {"mode": "rule", "level0_slices": 8}),
                     ("fixed_3_slices", {"mode": "fixed", "fixed_slices": 3})):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = scf.run(ctx, h, S, nocc, En, **kw)
        wall = time.perf_counter() - t0
        its = res["iterations"]
        runs[name] = {"E": res["E"], "converged": res["converged"], "iterations": len(its),
                      "ms_jk_total": sum(r["ms"] for r in its), "s_wall": wall,
                      "levels": [r["level"] for r in its], "slices": [r["slices"] for r in its]}
    ref = runs["fp64"]
    for name in ("rule", "rule_level0_8_slices", "fixed_3_slices"):
        r = runs[name]
        r["dE_vs_fp64_scf"] = r["E"] - ref["E"]
        r["jk_speedup_vs_fp64"] = ref["ms_jk_total"] / r["ms_jk_total"]
    return {"metric": "RHF to convergence with DF J/K, exchange precision by the Table 1 rule vs native FP64",
            "workload": "scf-" + w.name, "nuclear_charge": 2.0, "nocc": nocc, "E_nuc": En, **runs}


def run_crt(args):
    """The two exchange contractions of the chosen molecule (X = B C over rows
    (P, mu), and one block's K_b = X_b X_b^T) emulated by INT8 slices and by
    the CRT variant (Ozaki scheme II) at each Table 1 level (the CRT modulus
    count resolving rows like the level's slices), against cuBLAS DGEMM:
    per-call time (split, tensor-core GEMMs, recombination or reconstruction;
    scratch from a warm pool) and error relative to max|DGEMM|."""
    import torch
    from paper_2601_08077_gb300 import build, df, inputs
    build.build_all()
    torch.cuda.set_device(0)
    w = workload(args.size or "medium")
    mol = inputs.molecule(w.n_atoms, w.seed)
    Bt = inputs.df_tensor_device(mol)
    nao, nocc = mol.nao, w.nocc
    C = torch.from_numpy(inputs.orbitals(nao, nocc, w.seed + 1)).cuda()
    A1 = Bt.reshape(-1, nao)
    B1 = C.T.contiguous()
    Xb = (A1[:128 * nao] @ C).reshape(128, nao, nocc)
    A2 = Xb.permute(1, 0, 2).reshape(nao, -1).contiguous()

    def timed(fn, reps=5, warm=2):
        for _ in range(warm):
            out = fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), out

    shapes = {}
    for name, A, B in (("X=BC", A1, B1), ("K_b=X_bX_b^T", A2, A2)):
        M, K = A.shape
        N = B.shape[0]
        flops = 2.0 * M * N * K
        t64, ref = timed(lambda: A @ B.T)
        scale = float(ref.abs().max())
        rows = []
        for s in (3, 4, 5, 6, 7):
            n = df.crt_moduli_for_bits(K, 8 * s - 1)
            ts, o_s = timed(lambda: df.emulated_gemm(A, B, s))
            tc, o_c = timed(lambda: df.emulated_gemm_crt(A, B, n))
            rows.append({"slices": s, "slice_products": s * (s + 1) // 2, "ms_slices": ts,
                         "err_slices": float((o_s - ref).abs().max()) / scale,
                         "moduli": n, "q": df.crt_operand_bits(K, n), "ms_crt": tc,
                         "err_crt": float((o_c - ref).abs().max()) / scale,
                         "tflops_slices": flops / ts / 1e9, "tflops_crt": flops / tc / 1e9})
            del o_s, o_c
        shapes[name] = {"M": M, "N": N, "K": K, "ms_dgemm": t64, "tflops_dgemm": flops / t64 / 1e9,
                        "levels": rows}
    return {"metric": "emulated FP64 GEMM, INT8 slices vs CRT (Ozaki scheme II), per Table 1 level",
            "workload": w.name, "shapes": shapes}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload in ("batch", "sequence", "predictor", "scf", "crt"):
        if rank == 0:
            fn = {"batch": run_batch, "sequence": run_sequence, "predictor": run_predictor,
                  "scf": run_scf, "crt": run_crt}[args.workload]
            print(json.dumps(fn(args)), flush=True)
        return
    w = workload(args.workload)
    if args.aux_blocks > 0 and args.aux_blocks * 128 < w.naux:
        import types
        naux = args.aux_blocks * 128
        w = types.SimpleNamespace(name="%s-aux%d" % (w.name, naux), n_atoms=w.n_atoms, nocc=w.nocc, seed=w.seed,
                                  nao=w.nao, naux=naux, shape=w.shape, tau=w.tau)

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, w)), flush=True)
        return

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2601_08077_gb300 import build, df, inputs, shard
    if rank == 0 or world == 1:
        build.build_all()
    if world > 1:
        dist.barrier()

    dev = torch.device("cuda", local)
    mol = inputs.workload_molecule(w)
    ctx = df.Context(w.nao, w.naux, w.nocc)
    if w.n_atoms >= 120:
        # the library forms B from the integrals on the device (Cholesky + triangular solve);
        # a screened workload zeroes its Schwarz-screened pairs first (Section 2.1)
        sub = inputs.leading_aux(mol, w.naux)
        Tg = torch.from_numpy(inputs.screened_int3c(sub, w.tau)).to(dev)
        Vg = torch.from_numpy(inputs.metric(sub)).to(dev)
        Bg = ctx.setup_integrals(Tg, Vg)
        del Vg
    else:
        Bh = inputs.df_tensor_rows(mol, w.naux) if w.naux < mol.naux else inputs.df_tensor(mol)
        Bg = torch.from_numpy(Bh).to(dev)
        ctx.setup(Bg)
    sparsity = ctx.sparsity()
    C = inputs.orbitals(mol.nao, w.nocc, w.seed + 1)
    D = inputs.density(C)
    Cg = torch.from_numpy(C).to(dev)
    Dg = torch.from_numpy(D).to(dev)
    B_bytes = Bg.numel() * 8
    ctx.set_cluster_pairs(args.cluster_pairs)
    ctx.set_jk_overlap(args.jk_overlap)
    J = torch.empty((w.nao, w.nao), dtype=torch.float64, device=dev)
    K = torch.empty_like(J)
    rho = torch.empty(w.naux, dtype=torch.float64, device=dev)
    s = args.nslices

    # accuracy gate against the native FP64 build on the same GPU
    K64 = ctx.build_K(Cg, 0)[0].clone()
    Ks = ctx.build_K(Cg, s)[0]
    scale = float(K64.abs().max())
    dK = float((Ks - K64).abs().max()) / scale
    ctx.build_J(Dg, J, rho)
    E_fp64 = ctx.energy(Dg, J, K64, rho)
    E_s = ctx.energy(Dg, J, Ks, rho)
    dE = abs((E_s[0] + E_s[2]) - (E_fp64[0] + E_fp64[2]))
    ctx.sync_status()
    K_gate, J_gate = Ks.cpu().numpy(), J.cpu().numpy()
    del Ks, K64

    def step():
        ctx.build_JK(Dg, Cg, s, J, rho, K)
        ctx.energy(Dg, J, K, rho)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.phase_times()
    ctx.set_profiling(True)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ctx.set_profiling(False)
    phases = ctx.phase_times()
    # the one-call build returns the separate builds' J and K bit for bit
    jk_same = bool(np.array_equal(J.cpu().numpy(), J_gate) and np.array_equal(K.cpu().numpy(), K_gate))
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = shard.max_over_ranks(ms, dev)
    ctx.sync_status()

    # the exchange build alone (INT8 slices): in the timed step the X split shares
    # the SMs with rho and J, so its phase time there is not the K build's
    nk = max(1, min(10, args.steps))
    torch.cuda.synchronize()
    ctx.phase_times()
    ctx.set_profiling(True)
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(nk):
        ctx.build_K(Cg, s, K)
    k1.record(stream)
    torch.cuda.synchronize()
    ctx.set_profiling(False)
    k_phases = ctx.phase_times()
    ms_k = k0.elapsed_time(k1) / nk

    # native FP64 exchange build, same GPU, same B (the comparison build)
    nfp = max(1, min(3, args.steps))
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(nfp):
        ctx.build_K(Cg, 0, K)
    f1.record(stream)
    torch.cuda.synchronize()
    ms_fp64 = f0.elapsed_time(f1) / nfp

    # end to end through the public API with host buffers (pinned), copies timed
    Ch = torch.from_numpy(C).pin_memory()
    Dh = torch.from_numpy(D).pin_memory()
    Jh = torch.empty((w.nao, w.nao), dtype=torch.float64).pin_memory()
    Kh = torch.empty_like(Jh).pin_memory()
    Cd = torch.empty_like(Cg)
    Dd = torch.empty_like(Dg)

    def step_e2e():
        Cd.copy_(Ch, non_blocking=True)
        Dd.copy_(Dh, non_blocking=True)
        ctx.build_JK(Dd, Cd, s, J, rho, K)
        ctx.energy(Dd, J, K, rho)
        Jh.copy_(J, non_blocking=True)
        Kh.copy_(K, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    step_e2e()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    torch.cuda.synchronize()
    ms_e2e = (time.perf_counter() - t0) / args.steps * 1e3
    h2d = C.nbytes + D.nbytes
    d2h = 2 * w.nao * w.nao * 8 + 3 * 8

    FK = flops_K(w)
    value = FK * world / (ms * 1e-3) / 1e12
    # roofline of the dominant kernel (the slice GEMM launch with the largest share)
    pk, src = peaks()
    g1_ms = phases["gemm1"][0] / max(1, phases["gemm1"][1])
    g2_ms = phases["gemm2"][0] / max(1, phases["gemm2"][1])
    pairs = s * (s + 1) // 2
    g1_flops = pairs * 2.0 * w.nocc * w.naux * w.nao * w.nao
    g2_flops = pairs * 2.0 * (w.nao * (w.nao + 1) / 2) * w.naux * w.nocc
    if g1_ms >= g2_ms:
        kname, kms, kfl = "slice_gemm (X = B C)", g1_ms, g1_flops
    else:
        kname, kms, kfl = "slice_gemm (K_b = X_b X_b^T)", g2_ms, g2_flops
    peak = float(pk.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"]))
    achieved = kfl / (kms * 1e-3) / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (INT8 slices as BF16 on tcgen05, exact INT accumulation)",
        "data": "synthetic (seeded s-type Gaussian molecule, integrals and DF tensor generated)",
        "config": {"workload": w.name, "nao": w.nao, "naux": w.naux, "nocc": w.nocc, "nslices": s,
                   "slice_count": "fixed for every step (5 = Table 1 level 2's count, the first level meeting "
                                  "max|dK| <= 1e-10 max|K|)" if s == 5 else "fixed for every step", "l2": "inputs larger than L2 (B %.1f GB)" % (B_bytes / 1e9),
                   "cluster_pairs": args.cluster_pairs,
                   "jk_overlap": ("J, then K, in one stream (df_build_JK; a block-sparse B runs its masked "
                                  "kernels in order)" if sparsity[1] < 1.0 else
                                  "rho and J on %d CTAs per SM beside the X split (df_build_JK)" % args.jk_overlap)
                                 if args.jk_overlap else "J, then K, in one stream",
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": FK / (ms_e2e * 1e-3) / 1e12 * world, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e},
        "gpu_launches": LAUNCHES_PER_STEP * args.steps,
        "roofline": {"bound": "tensor", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": recorded_traffic(kname, w.name, s, args.cluster_pairs),
                     "peak_source": "bf16_tflops_sustained (%s)" % src,
                     "algorithmic": "s(s+1)/2 slice-pair products x 2 flops per multiply-add, no padding"},
        "accuracy": {"max_dK_rel_vs_fp64": dK, "dE_vs_fp64": dE, "gate_1e-10": dK <= 1e-10,
                     "jk_bit_identical_to_separate_builds": jk_same},
        "fp64_native": {"k_build_ms": ms_fp64, "tflops": FK / (ms_fp64 * 1e-3) / 1e12,
                        "speedup_of_int8": ms_fp64 / ms_k},
        "phases_ms_per_step": {k: v[0] / args.steps for k, v in phases.items()},
        "phases_note": "CUDA-event intervals per phase; rho and J run beside the X split (df_build_JK), "
                       "so those three intervals overlap" if args.jk_overlap else "phases in one stream, in order",
        "k_build_tflops": FK / (ms_k * 1e-3) / 1e12,
        "k_build_alone": {"ms": ms_k, "builds": nk,
                          "phases_ms": {k: v[0] / nk for k, v in k_phases.items() if v[1]}},
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"], K_ref, J_ref, _ = oracle_reference(Bg, C, D, w)
        out["accuracy"].update(oracle_gate(K_gate, J_gate, E_s, K_ref, J_ref, D))
        if not out["accuracy"]["gate_vs_oracle"]:
            print("bench: the run misses the accuracy gate against the oracle", file=sys.stderr)
    if rank == 0 and not args.no_records and args.aux_blocks == 0 and w.name == workload("large").name:
        # the other workloads of the metric, outside the timed region: the adaptive
        # sequence on this molecule, then (memory freed) the fixed-slice sweep and the batch
        from paper_2601_08077_gb300 import sequence
        t0 = time.perf_counter()
        orbs = sequence.orbital_sequence(C, 15, w.seed)
        out["records"] = {"sequence": sequence_record(ctx, w, orbs, full_fp64=False)}
        del ctx, Bg, K, J
        if "Tg" in locals():
            del Tg      # the same storage as Bg (B formed in place from the integrals)
        torch.cuda.empty_cache()
        out["records"]["sweep"] = sweep_record()
        torch.cuda.empty_cache()
        out["records"]["batch"] = batch_record(48, 5, 5, 2)
        out["records"]["seconds"] = time.perf_counter() - t0
    if w.tau > 0:
        n_scr = int(inputs.schwarz_pairs(mol, w.tau).sum())
        fk, fc = sparsity
        out["screening"] = {"tau": w.tau, "pairs_kept": n_scr / w.nao ** 2,
                            "gemm1_ktiles_kept": fk, "rho_J_chunks_kept": fc,
                            "flop_model_screened": 2.0 * (n_scr + w.nao ** 2) * w.naux * w.nocc,
                            "tflops_screened_model": 2.0 * (n_scr + w.nao ** 2) * w.naux * w.nocc * world
                            / (ms * 1e-3) / 1e12}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# Source files whose change invalidates a recorded DRAM-traffic figure of the
# slice GEMM (the kernel, its launch parameters and the device helpers).
TRAFFIC_SOURCES = ("paper_2601_08077_gb300/csrc/slicegemm.cu", "paper_2601_08077_gb300/csrc/df_internal.h",
                   "paper_2601_08077_gb300/csrc/df_device.cuh", "paper_2601_08077_gb300/csrc/df_api.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")


def kernel_source_sha():
    import hashlib
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(kernel, workload_name, nslices, cluster_pairs):
    """DRAM bytes per launch of `kernel` (dram__bytes_read.sum + write.sum from
    one ncu capture of this bench command), if the capture in
    profiles/dram_traffic.txt (JSON records) matches the workload, the slice
    count, the pair mode and the current kernel sources; else None."""
    try:
        with open(TRAFFIC_FILE) as f:
            recs = json.load(f)
    except (OSError, ValueError):
        return None
    sha = kernel_source_sha()
    for r in recs:
        if (r.get("kernel") == kernel and r.get("workload") == workload_name and r.get("nslices") == nslices
                and r.get("cluster_pairs") == cluster_pairs and r.get("source_sha256") == sha):
            return float(r["dram_bytes_per_launch"])
    return None


if __name__ == "__main__":
    main()
