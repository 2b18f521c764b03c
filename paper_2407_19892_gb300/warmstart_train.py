"""Train the warm-start network on the GPU and save its parameters.

    python -m paper_2407_19892_gb300.warmstart_train [--problems 800] [--steps 6000]

Training pairs are generated by the method itself: seeded scRNA-like count
matrices (log-uniform 1k-200k cells x 500-5000 genes by default, random
cluster counts and cell ranks) go through the GPU preprocessing, Gram, FP64
spectra and the cold-start eigenvalue solve; the network learns solved
eigenvalues from spectra.  Forward, backward and Adam run in the library's kernels.  Writes
``warmstart_mlp.npz`` next to this file.
"""

import argparse
import json
import time

import torch

from . import build, warmstart


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=5000)
    ap.add_argument("--cells", type=int, nargs=2, default=(1000, 200000), help="log-uniform range of cells")
    ap.add_argument("--genes", type=int, nargs=2, default=(500, 5000), help="log-uniform range of genes")
    ap.add_argument("--max-minutes", type=float, default=None, help="stop generating problems after this long")
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=20240731)
    ap.add_argument("--out", default=warmstart.WEIGHTS)
    a = ap.parse_args()
    build.build()
    dev = torch.device("cuda:0")
    t0 = time.time()
    deadline = t0 + 60.0 * a.max_minutes if a.max_minutes else None
    F, T = warmstart.method_pairs(a.problems, seed=a.seed, device=dev, cell_range=tuple(a.cells),
                                  gene_range=tuple(a.genes), deadline=deadline)
    t1 = time.time()
    p = warmstart.init_params(a.seed, dev)
    loss0, _ = warmstart.loss_grad(p, F, T)
    lr = a.lr
    adam = None
    for phase in range(3):  # step the learning rate down
        _, adam = warmstart.train(p, F, T, steps=a.steps // 3, batch=a.batch, lr=lr, seed=a.seed + phase, adam=adam)
        lr *= 0.3
    loss1, _ = warmstart.loss_grad(p, F, T)
    torch.cuda.synchronize()
    warmstart.save(p, a.out)
    print(json.dumps({"pairs": int(F.shape[0]), "cells": list(a.cells), "genes": list(a.genes),
                      "gen_s": round(t1 - t0, 1), "train_s": round(time.time() - t1, 1),
                      "loss_initial": loss0, "loss_final": loss1, "out": a.out}))


if __name__ == "__main__":
    main()
