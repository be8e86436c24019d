"""Runs a few predict steps of a workload on cuda:0 (for profilers such as ncu).

  python -m paper_2310_03921_gb300.profile_run [--workload 2] [--steps 3] [--precision bf16x3]
"""
from __future__ import annotations

import argparse

from . import build, gap, synth, workloads


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--precision", default="bf16x3")
    args = ap.parse_args()
    import torch
    build.build()
    torch.cuda.set_device(0)
    w, soap, model = workloads.model_for(args.workload, gap, "cuda:0")
    batch = gap.Batch.from_synth(synth.make_batch(synth.structures(args.workload)), device="cuda:0")
    for _ in range(args.steps):
        out = model.predict(batch, precision=args.precision, local=False)
    torch.cuda.synchronize()
    print(f"{w.name}: {batch.n_atoms} atoms, E[0] = {float(out['energy'][0]):.6f} eV")


if __name__ == "__main__":
    main()
