"""Runs a few steps of a workload on cuda:0 (for profilers such as ncu).

  python -m paper_2310_03921_gb300.profile_run [--workload 2] [--steps 3] [--precision bf16x3]
  python -m paper_2310_03921_gb300.profile_run --fit 20 [--steps 1]
  python -m paper_2310_03921_gb300.profile_run --chol 2000 [--steps 2]

--tile-variant v (0..3) fixes the tensor-core contractions' tile instead of
timing the candidates (under a profiler the timings carry its overhead):
0 = 128 x 256, 1 = 128 x 128 with two TMA stages, 2 = with three, 3 = 128 x
192 with twelve epilogue warps, where that variant applies.

Without --fit: predict steps (energies, forces, virials) of the workload.
With --fit C: fit steps of the 200-cell K_NM workload restricted to its
first C cells: K_NM assembly, the CholeskyQR least-squares solve with
tensor-core FP64 products, and predict with the new coefficients.
With --chol n: the solve's recursive Cholesky factor and inverse of a seeded
n x n SPD matrix (the Gram matrix of Gaussian (n + 100) x n data), once per
step.
"""
from __future__ import annotations

import argparse

import numpy as np

from . import build, gap, synth, workloads


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--precision", default="bf16x3")
    ap.add_argument("--fit", type=int, default=0, help="cells of the K_NM fit workload (0: predict steps)")
    ap.add_argument("--chol", type=int, default=0, help="order of a recursive Cholesky factorisation to run")
    ap.add_argument("--tile-variant", type=int, default=-1, help="fixed contraction tile (-1: autotuned)")
    args = ap.parse_args()
    import torch
    build.build()
    torch.cuda.set_device(0)
    gap.test_tc_force_variant(args.tile_variant)
    if args.chol:
        rng = np.random.default_rng(0)
        A = rng.normal(size=(args.chol + 100, args.chol))
        Gm = A.T @ A
        for _ in range(args.steps):
            R, X = gap.test_chol_inv(Gm)
        print(f"Cholesky factor and inverse of order {args.chol}: max |R X - I| = {np.abs(R @ X - np.eye(args.chol)).max():.2e}")
        return
    if args.fit:
        w, soap, model = workloads.model_for(1, gap, "cuda:0")
        cells = synth.structures(1)[:args.fit]
        batch = gap.Batch.from_synth(synth.make_batch(cells), device="cuda:0")
        rows = batch.n_configs + 3 * batch.n_atoms
        rng = np.random.default_rng(0)
        y = torch.as_tensor(rng.normal(size=rows), device="cuda:0")
        sig = torch.full((rows,), 0.1, dtype=torch.float64, device="cuda:0")
        for _ in range(args.steps):
            K = model.assemble_knm(batch, precision=args.precision)
            a = model.solve(K, y, sig, jitter=1e-8, method="cholqr_tc")
            model.set_alpha(a)
            out = model.predict(batch, precision=args.precision, local=False)
        torch.cuda.synchronize()
        n_pairs = soap.descriptor_sizes(batch)[1]
        print(f"fit of {len(cells)} cells: {rows} rows x {model.columns} columns, "
              f"{3 * (batch.n_atoms + n_pairs)} Jacobian rows, E[0] = {float(out['energy'][0]):.6f} eV")
        return
    w, soap, model = workloads.model_for(args.workload, gap, "cuda:0")
    batch = gap.Batch.from_synth(synth.make_batch(synth.structures(args.workload)), device="cuda:0")
    for _ in range(args.steps):
        out = model.predict(batch, precision=args.precision, local=False)
    torch.cuda.synchronize()
    print(f"{w.name}: {batch.n_atoms} atoms, E[0] = {float(out['energy'][0]):.6f} eV")


if __name__ == "__main__":
    main()
