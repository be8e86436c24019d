#!/usr/bin/env python
"""Throughput of the GAP hot path on the fitting workload.

Workload: 200 seeded diamond-Si cells of 64-216 atoms (2x2x2 to 3x3x3
conventional cells, displacements sigma uniform in [0.05, 0.2] A, symmetric
lattice strain within +-3%), SOAP n_max = 8, l_max = 6, cutoff 5 A,
atom_sigma 0.5 A (D = 252), M = 2000 sparse points, zeta = 4, delta = 1 eV,
targets from a teacher model.  One step is one pass of the whole hot path
over the batch, every array resident in HBM:
  1. gap_assemble_knm: neighbours, descriptors, energy rows and 3N force
     rows of K_NM (tensor-core split-BF16 contraction, FP32 accumulate);
  2. gap_solve: FP64-accurate regularised least squares (shifted
     CholeskyQR with exact modular Gram matrices on the tensor cores);
  3. gap_predict: energies, forces and virials of the batch with the new
     coefficients.
Metric: K_NM rows/s over the step (rows = cells + 3 atoms; higher is
better); the assembly-only row rate and the E+F atoms/s of step 3 are
reported beside it.  After the timed region the line also carries the
error of every result (eps, E, F, V, K_NM) against the FP64 oracle on a
sample of the batch (`parity`), the achieved rate of the CUDA-core kernels
against an FMA probe run in the same process (`alu_rooflines`), and the
tensor-core rooflines against the measured BF16 burst peak.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload (see cpu_baseline).  Multi-GPU runs are
replicas: each rank runs the whole workload on its own GPU (the path needs no
exchange), and value is the total over ranks.
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

from paper_2310_03921_gb300 import synth  # noqa: E402

METRIC = "K_NM rows/s"
UNIT = "rows/s"
WORKLOAD = dict(workload="200 strained diamond-Si cells, 64-216 atoms (K_NM fit)", n_configs=200, n_max=8, l_max=6,
                cutoff=5.0, atom_sigma=0.5, D=252, M=2000, zeta=4, delta=1.0, jitter=1e-8,
                sigma_energy_per_atom=0.001, sigma_force=0.1, precision="bf16x3")
SIG_E, SIG_F, JITTER = 0.001, 0.1, 1e-8
L2_BYTES = 129 * 2 ** 20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("bf16_tflops_sustained", 1700.0), d.get("bf16_tflops", 1900.0), d.get("hbm_gbs", 6800.0), \
            "measured"
    return 1700.0, 1900.0, 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- our arm
def targets(model, batch, cells, torch, device):
    """Teacher energies and forces in K_NM row order, and the per-row sigma."""
    w = synth.workload(1)
    alpha0 = np.concatenate(model._al)
    model.set_alpha(synth.SplitMix64(synth.seed_for(1, 0, "teacher")).normal(alpha0.size, 0.1))
    out = model.predict(batch, precision="fp64", local=False, virial=False)
    E, F = out["energy"].cpu().numpy(), out["forces"].cpu().numpy()
    model.set_alpha(alpha0)
    y, sig, a = [], [], 0
    for k, c in enumerate(cells):
        y.append([E[k]])
        y.append(F[a:a + c.n].reshape(-1))
        sig.append([SIG_E * np.sqrt(c.n)])
        sig.append(np.full(3 * c.n, SIG_F))
        a += c.n
    y, sig = np.concatenate(y), np.concatenate(sig)
    return torch.as_tensor(y, device=device), torch.as_tensor(sig, device=device), y, sig


# Moduli of the modular products (the library's table: 16 byte moduli, then
# primes below 512) and the counts it takes for a Gram matrix of m rows and a
# congruence of n_ext columns.
CRT_MODULI = [256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193, 509, 503, 499, 491,
              487, 479, 467, 463, 461, 457, 449, 443, 439, 433, 431, 421, 419, 409, 401, 397, 389, 383, 379, 373]


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one K_NM
# force-row GEMM launch (k_tc_gemm, TMEM-resident K_NM epilogue), from one ncu
# capture on the first 20 cells of the fit workload (194,934 Jacobian rows):
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none \
#       --kernel-name-base demangled -k "regex:\(int\)192" -s 1 -c 1 \
#       python -m paper_2310_03921_gb300.profile_run --fit 20 --steps 1
# (the 128 x 192 tile with twelve epilogue warps that the autotuner picks)
# The operand rows, the W' rows and the K_NM rows all grow with the Jacobian
# rows, so a full launch is scaled by 3 (N + P).
KNM_TRAFFIC_READ, KNM_TRAFFIC_WRITE, KNM_TRAFFIC_JROWS = 223092736, 82601984, 194934


def crt_moduli_counts(m: int, n_ext: int):
    def count(need, limit):
        have = 0.0
        for t, p in enumerate(CRT_MODULI[:limit]):
            have += np.log2(p)
            if have > need:
                return t + 1
        return 0
    T1 = count(107.0 + np.log2(max(m, 1)) + 1e-9, 16)
    T2 = count(2 * np.log2(n_ext) + 212.0 + np.log2(max(m, 1) + 2.0) + 1.0 + 1e-9, 40)
    return T1, T2


def chol_blocks(n: int, block: int = 64, split: int = 32) -> list:
    """Orders of the diagonal blocks the recursive factorisation of an n x n
    Gram matrix hands to its block kernel (halves rounded up to a multiple
    of `split` until a block is at most `block`)."""
    if n <= block:
        return [n]
    n1 = (n // 2 + split - 1) // split * split
    return chol_blocks(n1, block, split) + chol_blocks(n - n1, block, split)


def block_flops(m: int) -> float:
    """FP64 flops of the block kernel on an m x m block: elimination on
    [A | I], step k updating rows i > k on their live columns (A: j >= i,
    B: j <= k), two flops per multiply-add."""
    f = 0
    for k in range(m - 1):
        for i in range(k + 1, m):
            f += (m - i) + (k + 1)
    return 2.0 * f


def alu_rooflines(per_launch, n_atoms, n_pairs, n_max, l_max, D, M, fp32_peak, fp64_peak, hbm, n_sm, n_fact):
    """Achieved rate of the kernels bound by CUDA-core arithmetic, against the
    FMA probe measured in the same process, with their algorithmic HBM bytes
    against the measured copy bandwidth.  Per launch (one stage interval);
    single species, so one accumulation channel group.
      expansion  per pair: radial lookups (cubic, n (l+1)), Y_lm recurrence
                 (~3 (l+1)^2), c accumulation 2 n (l+1)^2; per atom: power
                 spectrum 2 npair (l+1)^2 and normalisation 3 D.  Bytes:
                 24 per pair read (FP32 vector, neighbour index, species),
                 coefficients 4 n (l+1)^2 and p_hat 4 D written per atom.
      pairforce  per pair: A_lm, B_lm = 4 n (l+1)^2, the radial lookups with
                 derivatives 12 n (l+1), the force sum 8 (l+1)^2.  Bytes: 24
                 read and 12 written per pair, 4 n (l+1)^2 read per atom.
      knm_jacobian per pair, with the separable pair derivative
                 dc/dr = w (dR u Y + R grad Y): A = sum_m Y c and
                 B = sum_m grad Y c per channel and l, 8 n (l+1)^2; per
                 descriptor entry and direction the derivative (5 multiply-
                 adds) and the projection (2), 42 D.  Bytes: the Jacobian
                 rows written, 3 (N + P) rows x 2 BF16 planes x D16 x 2 B.
      solve_block the elimination on [A | I] of one diagonal block of the
                 factorisation (mean over the blocks of an M x M Gram
                 matrix), on ONE SM: the peak is the chip's FP64 rate / SMs."""
    L1 = l_max + 1
    lam = L1 * L1
    npair = n_max * (n_max + 1) // 2
    D16 = (D + 15) // 16 * 16
    P, N = n_pairs, n_atoms
    kern = {
        "expansion": ("k_expand", P * (6 * n_max * L1 + 3 * lam + 2 * n_max * lam) + N * (2 * npair * lam + 3 * D),
                      24 * P + N * (4 * n_max * lam + 4 * D + 4), fp32_peak, "FP32"),
        "pairforce": ("k_pairforce", P * (4 * n_max * lam + 12 * n_max * L1 + 8 * lam),
                      36 * P + N * 4 * n_max * lam, fp32_peak, "FP32"),
        "knm_jacobian": ("k_jacobian_rows", P * (8 * n_max * lam + 42 * D),
                         3 * (N + P) * 2 * D16 * 2, fp32_peak, "FP32"),
    }
    out = {}
    for st, (name, flops, nbytes, peak, kind) in kern.items():
        if st not in per_launch:
            continue
        t = per_launch[st] / 1e3
        a = flops / t / 1e12
        out[st] = {"kernel": name, "bound": "alu", "ms_per_launch": per_launch[st], "flops": float(flops),
                   "achieved_tflops": a, "peak_tflops": peak, "peak_source": f"{kind} FMA probe, same process",
                   "frac": a / peak, "hbm_bytes": float(nbytes), "hbm_gbs": nbytes / t / 1e9,
                   "hbm_frac": nbytes / t / 1e9 / hbm}
    if "solve_block" in per_launch:
        blocks = chol_blocks(M)
        fl = sum(block_flops(b) for b in blocks) / len(blocks)
        t = per_launch["solve_block"] / 1e3
        a = fl / t / 1e12
        sm_peak = fp64_peak / n_sm
        out["solve_block"] = {"kernel": "k_chol_inv_block", "bound": "alu", "ms_per_launch": per_launch["solve_block"],
                              "flops": fl, "blocks_per_factorisation": len(blocks), "factorisations": n_fact,
                              "achieved_tflops": a, "peak_tflops": sm_peak,
                              "peak_source": f"FP64 FMA probe / {n_sm} SMs (one CTA)", "frac": a / sm_peak,
                              "frac_of_chip": a / fp64_peak}
    return out



def max_over_ranks(t_ms: float, dist, device) -> float:
    """The job's step time: the slowest rank's (every rank calls this; a
    barrier follows so that no rank starts the next phase early)."""
    if dist is None:
        return t_ms
    import torch
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def replica_throughput(units_per_rank: float, world: int, t_ms: float) -> float:
    """Whole-job throughput of `world` replicas that each process
    `units_per_rank` units in `t_ms` (the max over ranks)."""
    return world * units_per_rank / (t_ms / 1e3)


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2310_03921_gb300 import build as B
    from paper_2310_03921_gb300 import gap, workloads

    B.build()
    torch.cuda.set_device(local_rank)
    device = f"cuda:{local_rank}"
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(device))

    w, soap, model = workloads.model_for(1, gap, device)
    cells = synth.structures(1)
    hb = synth.make_batch(cells)
    batch = gap.Batch.from_synth(hb, device=device)
    n_atoms, n_cfg = hb.n_atoms, hb.n_configs
    rows = n_cfg + 3 * n_atoms
    y_d, sig_d, y_h, sig_h = targets(model, batch, cells, torch, device)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream()

    def step(prec="bf16x3", marks=None, method="cholqr_tc"):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if marks is not None else None
        if ev: ev[0].record(stream)
        K = model.assemble_knm(batch, precision=prec)
        if ev: ev[1].record(stream)
        a = model.solve(K, y_d, sig_d, jitter=JITTER, method=method)
        model.set_alpha(a)
        if ev: ev[2].record(stream)
        out = model.predict(batch, precision=prec, local=False)
        if ev:
            ev[3].record(stream)
            marks.append(ev)
        return out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank) if rank == 0 else None
    launches0 = gap.launch_count()
    times, marks = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(marks=marks)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    launches = gap.launch_count() - launches0
    clk = clocks.stop() if clocks else None
    t_mean = sum(times) / len(times)
    phase = {k: statistics.mean(m[i].elapsed_time(m[i + 1]) for m in marks)
             for i, k in enumerate(("assemble_ms", "solve_ms", "predict_ms"))}
    t_mean = max_over_ranks(t_mean, dist, device)

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    pos_h = torch.from_numpy(hb.pos).pin_memory().numpy()
    spec_h = torch.from_numpy(hb.species).pin_memory().numpy()
    hbatch = gap.Batch(pos_h, spec_h, hb.cell, hb.pbc, hb.config_offsets)
    yp = torch.from_numpy(np.ascontiguousarray(y_h)).pin_memory().numpy()
    sp = torch.from_numpy(np.ascontiguousarray(sig_h)).pin_memory().numpy()
    e2e_t = []
    for _ in range(max(2, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # gap_fit: K_NM assembled, solved and installed without leaving the
        # device; then predict with the new coefficients
        a = model.fit(hbatch, yp, sp, jitter=JITTER, method="cholqr_tc", precision="bf16x3")
        out = model.predict(hbatch, precision="bf16x3", local=False)
        e2e_t.append(time.perf_counter() - t0)
    h2d = 2 * (hb.pos.nbytes + hb.species.nbytes + hb.cell.nbytes) + yp.nbytes + sp.nbytes
    d2h = a.nbytes + out["forces"].nbytes + out["energy"].nbytes + out["virial"].nbytes

    # per-stage durations (CUDA events recorded inside the calls, on their stream)
    gap.profile_enable(True)
    gap.profile_reset()
    for _ in range(3):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    stages = gap.profile_read()
    gap.profile_enable(False)

    # plain FP64 GPU path, same step (the comparator), after one untimed step
    # (first use of its library kernels and workspace)
    step("fp64", method="householder")
    torch.cuda.synchronize()
    fp64_marks = []
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step("fp64", marks=fp64_marks, method="householder")
    e1.record(stream)
    e1.synchronize()
    fp64_ms = e0.elapsed_time(e1)
    fm = fp64_marks[0]
    fp64_phase = {k: fm[i].elapsed_time(fm[i + 1]) for i, k in enumerate(("assemble_ms", "solve_ms", "predict_ms"))}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return None

    sus, burst, hbm, src = peaks()
    D, M = soap.dim, w.M
    n_pairs = soap.descriptor_sizes(batch)[1]
    per_launch = {k: v[0] / max(v[1], 1) for k, v in stages.items() if v[1] > 0}
    per_step = {k: v[0] / 3 for k, v in stages.items() if v[1] > 0}
    # Tensor-core kernels with their algorithmic flops per step:
    #  knm_gemm   the K_NM contraction, 2 (3 (N + P) + N) D M (the split-precision
    #             scheme issues 3x that);
    #  solve_gemm the modular products of the CholeskyQR solve: the Gram
    #             matrix of the m data rows with the right-hand side appended
    #             (n = M + 1 columns, upper triangle: T1 m n (n + 1) flops), and
    #             two congruences W^T G W (triangular W: T2 n^2 (n + 1) for
    #             H = G W, T2 n (n + 1) (n + 2) / 3 for the symmetric W^T H),
    #             T1 and T2 the moduli counts the library chooses.
    m_ls, n_ext = rows, M + 1
    T1, T2 = crt_moduli_counts(m_ls, n_ext)
    solve_flops = (T1 * m_ls * n_ext * (n_ext + 1)
                   + 2 * T2 * (n_ext ** 2 * (n_ext + 1) + n_ext * (n_ext + 1) * (n_ext + 2) / 3.0))
    tensor = {
        "knm_gemm": ("k_tc_gemm (K_NM force rows, split BF16x3)",
                     2.0 * 3.0 * (n_atoms + n_pairs) * D * M,
                     "2 * 3 (N + P) * D * M: one D x M sweep per Jacobian row (3 own rows per atom, 3 per pair); "
                     "the energy rows are a separate launch; the split scheme issues 3x this on the tensor cores"),
        "solve_gemm": ("k_crt_gemm (modular FP64 products of CholeskyQR3)", float(solve_flops),
                       f"Gram T1 m n (n + 1) + 2 congruences T2 (n^2 (n + 1) + n (n + 1) (n + 2) / 3), "
                       f"n = M + 1, T1 = {T1}, T2 = {T2}"),
    }
    dom = max(tensor, key=lambda k: per_step.get(k, 0.0))
    rooflines = {}
    for k, (kern, flops, note) in tensor.items():
        if k in per_step:
            a = flops / (per_step[k] / 1e3) / 1e12
            rooflines[k] = {"kernel": kern, "achieved_tflops": a, "frac": a / burst, "ms": per_step[k],
                            "flops": flops, "note": note}
    achieved = rooflines[dom]["achieved_tflops"]
    fp32_peak, fp64_peak = gap.fma_peak_tflops(False), gap.fma_peak_tflops(True)
    n_sm = torch.cuda.get_device_properties(device).multi_processor_count
    n_fact = stages.get("solve_potrf", (0.0, 0))[1] / 3
    alu = alu_rooflines(per_launch, n_atoms, n_pairs, soap.n_max, soap.l_max, D, M, fp32_peak, fp64_peak, hbm, n_sm,
                        n_fact)
    knm_traffic = (KNM_TRAFFIC_READ + KNM_TRAFFIC_WRITE) * (3.0 * (n_atoms + n_pairs)) / KNM_TRAFFIC_JROWS
    nested = ("knm_jacobian", "solve_block")  # intervals inside other stages
    step_total = sum(v for k, v in per_step.items() if k not in nested)
    value = replica_throughput(rows, world, t_mean)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_mean, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16",
        "dtype_detail": "bf16x3 tensor-core contraction (f32 accumulate), f32 descriptors, f64 solve and sums",
        "data": "synthetic: seeded strained/displaced diamond Si, random-selected sparse points, teacher targets",
        "config": dict(WORKLOAD, n_atoms=n_atoms, rows=rows, n_pairs=n_pairs,
                       parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                       l2="flushed between timed steps (256 MiB write)"),
        "phases_ms": {k: round(v, 4) for k, v in phase.items()},
        "knm_assembly_rows_per_s": rows / (phase["assemble_ms"] / 1e3),
        "ef_atoms_per_s": n_atoms / (phase["predict_ms"] / 1e3),
        "e2e": {"value": world * rows / statistics.mean(e2e_t), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": {"bound": "tensor", "kernel": rooflines[dom]["kernel"], "stage": dom, "achieved": achieved,
                     "peak": burst, "peak_source": f"bf16_tflops burst ({src}): each launch is a few ms, "
                     "far shorter than the seconds-long loop of the sustained figure", "unit": "TFLOP/s",
                     "frac": achieved / burst, "traffic": knm_traffic if dom == "knm_gemm" else None,
                     "traffic_unit": "bytes per K_NM GEMM launch (ncu capture, scaled by Jacobian rows)",
                     "note": rooflines[dom]["note"]},
        "tensor_rooflines": rooflines,
        "stages_ms_per_step": {k: round(v, 4) for k, v in per_step.items()},
        "stage_share": {k: round(v / step_total, 4) for k, v in per_step.items()},
        "alu_rooflines": alu,
        "probe_peaks_tflops": {"fp32": fp32_peak, "fp64": fp64_peak},
        "fp64_path": {"value": rows / (fp64_ms / 1e3), "unit": UNIT, "ms_per_step": fp64_ms,
                      "phases_ms": {k: round(v, 3) for k, v in fp64_phase.items()},
                      "knm_assembly_rows_per_s": rows / (fp64_phase["assemble_ms"] / 1e3),
                      "ef_atoms_per_s": n_atoms / (fp64_phase["predict_ms"] / 1e3)},
    }
    if not args.no_md:
        line["md_predict"] = md_predict(gap, workloads, torch, device, flush, args, 2)
        line["md_predict"]["parity_bf16x3"] = md_parity(gap, device, 2)
        line["predict_workloads"] = {str(k): md_predict(gap, workloads, torch, device, flush, args, k)
                                     for k in (0, 3, 4)}
    line["tile_tuning"] = gap.tile_tuning()
    sample = oracle_sample()
    ref = []
    base = cpu_baseline(sample, 1, keep=ref)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = base
    line["parity"] = parity(gap, device, sample, ref)
    if dist:
        dist.destroy_process_group()
    return line


PREDICT_WORKLOADS = {
    0: "64-atom diamond-Si cell (2x2x2, sigma 0.1 A), n_max 6, l_max 4, D 105, M 100",
    2: "32768-atom diamond-Si supercell (16^3 cells, sigma 0.1 A), n_max 8, l_max 8, cutoff 5 A, D 324, M 4000",
    3: "512 random-packed 4-species boxes of 8-256 atoms at 0.05 A^-3, compressed SOAP n_max 8, l_max 6, "
       "K 4 (D 1008), M 3000 per species",
    4: "110592-atom random network at 0.1 A^-3, SOAP n_max 10, l_max 8, cutoff 4.5 A (D 495), M 9000, "
       "plus 2-body (M 50)",
}


def md_predict(gap, workloads, torch, device, flush, args, index=2):
    """E+F atoms/s of a predict workload: one step (neighbour rebuild,
    descriptors, energies, forces, virial) as a captured CUDA graph, the same
    call eagerly, and the plain FP64 GPU path; L2 flushed between steps."""
    w, soap, model = workloads.model_for(index, gap, device)
    hb = synth.make_batch(synth.structures(index))
    batch = gap.Batch.from_synth(hb, device=device)
    stream = torch.cuda.current_stream()
    graph = gap.StepGraph(model, batch, precision="bf16x3", pair_capacity=1.2)

    def timed(fn, steps, warm=3):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    k0 = gap.launch_count()
    t_graph = timed(graph.launch, max(args.steps, 10))
    graph.status()
    t_eager = timed(lambda: model.predict(batch, precision="bf16x3", local=False), max(args.steps, 10))
    t_fp64 = timed(lambda: model.predict(batch, precision="fp64", local=False), 1)
    n = hb.n_atoms
    return {"workload": PREDICT_WORKLOADS[index] + ", zeta 4: energy, forces, virial per step", "n_atoms": n,
            "n_configs": hb.n_configs,
            "graph_ms_per_step": t_graph, "ef_atoms_per_s_graph": n / (t_graph / 1e3),
            "eager_ms_per_step": t_eager, "ef_atoms_per_s_eager": n / (t_eager / 1e3),
            "fp64_ms_per_step": t_fp64, "fp64_atoms_per_s": n / (t_fp64 / 1e3),
            "kernels_per_step": graph.kernels, "l2": "flushed between steps",
            "launches_counted": gap.launch_count() - k0}


# ---------------------------------------------------------- oracle (CPU) arm
SAMPLE_CELLS = 8


def oracle_sample(n_cells=SAMPLE_CELLS):
    """The bounded CPU sample: the first `n_cells` cells of the batch with the
    workload's SOAP parameters and M = 2000 sparse points drawn ('random'
    selection, the workload's seeds) from the oracle's own descriptors of the
    candidate cells, alpha the workload's seeded draw; one sample step = the
    K_NM rows and the energies, forces and virials of those cells."""
    import oracle as O
    w = synth.workload(1)
    sp = w.soap
    soap = O.Soap(sp.n_max, sp.l_max, sp.rc, sp.sigma, sp.d)
    pool = np.concatenate([O.descriptor(soap, c)[0] for c in synth.sparse_candidate_structures(1)])
    idx = synth.sparse_indices(1, 0, pool.shape[0], w.M)
    model = O.Model([pool[idx]], [synth.alpha_draw(1, 0, w.M)], w.delta, w.zeta)
    cells = synth.structures(1, n_cells)
    return O, soap, model, cells


def sample_desc(cells):
    n = sum(c.n for c in cells)
    return (f"K_NM rows (energy + force rows, M = 2000) and E+F+virial of the first {len(cells)} cells of the batch "
            f"({n} atoms, {len(cells) + 3 * n} rows) with the FP64 oracle; the least-squares solve is not part of "
            f"the sample")


def oracle_step(O, soap, model, cells, keep=None):
    t0 = time.perf_counter()
    rows = 0
    for c in cells:
        K = O.knm(soap, model, c)
        res = O.predict(soap, model, c)
        rows += 1 + 3 * c.n
        if keep is not None:
            keep.append((K,) + tuple(res))
    return rows, time.perf_counter() - t0


def cpu_baseline(sample, steps=1, keep=None):
    O, soap, model, cells = sample
    rs, ts = [], []
    for k in range(steps):
        r, t = oracle_step(O, soap, model, cells, keep if k == 0 else None)
        rs.append(r)
        ts.append(t)
    return {"value": rs[0] / statistics.mean(ts), "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": sample_desc(cells)}


def _err(a, b):
    d = np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)).ravel()
    return {"max": float(d.max()) if d.size else 0.0, "rms": float(np.sqrt(np.mean(d ** 2))) if d.size else 0.0}


def parity(gap, device, sample, ref):
    """Error of every result against the FP64 oracle on the sample cells, for
    the headline precision (split BF16x3) and the plain FP64 GPU path: the
    GPU model is built from the oracle's own sparse points and the seeded
    alpha (no input comes from the CUDA path), the oracle's results `ref` are
    those of the cpu_baseline step.  eps in eV per atom, E in eV per
    configuration, F in eV/A per component, V in eV per component, K_NM
    absolute and relative to max |K_NM|."""
    O, soap_o, model_o, cells = sample
    w = synth.workload(1)
    soap = gap.Soap.from_spec(w.soap)
    model = gap.Model(soap, [model_o.sparse], [model_o.alpha], w.delta, w.zeta)
    batch = gap.Batch.from_synth(synth.make_batch(cells), device=device)
    K_ref = np.concatenate([r[0] for r in ref])
    E_ref = np.array([r[1] for r in ref])
    le_ref = np.concatenate([r[2] for r in ref])
    F_ref = np.concatenate([r[3] for r in ref])
    V_ref = np.stack([r[4] for r in ref])
    kmax = float(np.abs(K_ref).max())
    out = {"sample": f"first {len(cells)} cells of the batch ({sum(c.n for c in cells)} atoms), oracle sparse points "
                     f"(M = {model_o.alpha.size}) and seeded alpha", "units": "eps eV/atom, E eV/config, F eV/A, "
                     "V eV, K_NM absolute (rel = max / max|K_NM|)"}
    for prec in ("bf16x3", "fp64"):
        p = model.predict(batch, precision=prec)
        K = model.assemble_knm(batch, precision=prec).cpu().numpy()
        r = {"eps": _err(p["local_e"].cpu().numpy(), le_ref), "E": _err(p["energy"].cpu().numpy(), E_ref),
             "F": _err(p["forces"].cpu().numpy(), F_ref), "V": _err(p["virial"].cpu().numpy().reshape(-1, 3, 3), V_ref),
             "K_NM": _err(K, K_ref)}
        r["K_NM"]["rel"] = r["K_NM"]["max"] / kmax
        out[prec] = r
    out["force_err_max"] = out["bf16x3"]["F"]["max"]
    out["force_tolerance"] = 1e-4
    out["within_tolerance"] = bool(out["bf16x3"]["F"]["max"] <= 1e-4 and out["fp64"]["eps"]["max"] <= 1e-6)
    return out


def md_parity(gap, device, index=2, n_sample=64):
    """Error of the split-BF16x3 predict against the FP64 oracle on n_sample
    seeded random atoms of a large single-species cell (the oracle's sampled
    predict evaluates each through its local cluster of radius 2 r_c).  The
    GPU model is built from the oracle's own sparse points ('random'
    selection among the oracle descriptors of the candidate cells) and the
    seeded alpha."""
    import oracle as O
    w = synth.workload(index)
    sp = w.soap
    soap_o = O.Soap(sp.n_max, sp.l_max, sp.rc, sp.sigma, sp.d)
    pool = np.concatenate([O.descriptor(soap_o, c)[0] for c in synth.sparse_candidate_structures(index)])
    idx = synth.sparse_indices(index, 0, pool.shape[0], w.M)
    X, a = pool[idx], synth.alpha_draw(index, 0, w.M)
    model_o = O.Model([X], [a], w.delta, w.zeta)
    s = synth.structures(index)[0]
    sel = synth.SplitMix64(synth.seed_for(index, 0, "count")).choice(s.n, n_sample)
    le_o, F_o = O.predict_sampled(soap_o, model_o, s, sel)
    soap = gap.Soap.from_spec(sp)
    model = gap.Model(soap, [X], [a], w.delta, w.zeta)
    batch = gap.Batch.from_synth(synth.make_batch([s]), device=device)
    p = model.predict(batch, precision="bf16x3", virial=False)
    le, F = p["local_e"].cpu().numpy()[sel], p["forces"].cpu().numpy()[sel]
    return {"sample": f"{n_sample} seeded random atoms of the {s.n}-atom cell, oracle sparse points (M = {w.M})",
            "eps": _err(le, le_o), "F": _err(F, F_o), "force_err_max": _err(F, F_o)["max"]}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    O, soap, model, cells = oracle_sample()
    for _ in range(args.warmup):
        oracle_step(O, soap, model, cells)
    rs, ts = [], []
    for _ in range(args.steps):
        r, t = oracle_step(O, soap, model, cells)
        rs.append(r)
        ts.append(t)
    v = rs[0] / statistics.mean(ts)
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(ts), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(WORKLOAD, precision="fp64 (CPU oracle)"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": sample_desc(cells)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-md", action="store_true", help="skip the 32768-atom MD-step measurement")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_ours(args, rank, world, local_rank)
    if rank == 0 and line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
