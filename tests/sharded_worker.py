"""One process of the cell-sharded fit, for the multi-process tests.

Run with RANK / WORLD_SIZE / MASTER_ADDR / MASTER_PORT set (gloo): takes its
block of rows of a seeded count matrix, runs
``paper_2407_19892_gb300.sharded.fit_two_axis_sharded`` with the oracle
test double (``oracle``) or the library's GPU backend on cuda:0 (``gpu``),
and writes its result and the communicator's exchange log to a file."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main(out_pattern, mode, cells, genes, r, k, splits):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2407_19892_gb300 import sharded
    from synth import scrna_counts
    world, rank = int(os.environ["WORLD_SIZE"]), int(os.environ["RANK"])
    dist.init_process_group("gloo", init_method="env://", world_size=world, rank=rank)
    counts = scrna_counts(cells, genes, 4, seed=20240801)
    cuts = [0] + [int(c) for c in splits.split(",") if c] + [cells]
    block = counts[cuts[rank]:cuts[rank + 1]].contiguous()
    if mode == "gpu":
        backend = sharded.GpuBackend(tol=1e-12)
        block = block.to("cuda:0")
    else:
        from sharded_backends import OracleBackend
        backend = OracleBackend()
    comm = sharded.TorchComm()
    res = sharded.fit_two_axis_sharded(block, r, k, k, backend, comm)
    rec = {"rank": rank, "row0": res.row0, "n_total": res.n_total, "log": comm.log,
           "e": res.e_cols.cpu().numpy(), "lr": res.lam_rows.cpu().numpy(), "lc": res.lam_cols.cpu().numpy(),
           "idx": res.idx_rows.cpu().numpy(), "val": res.val_rows.cpu().numpy(),
           "idx_c": None if res.idx_cols is None else res.idx_cols.cpu().numpy()}
    np.save(out_pattern % rank, rec, allow_pickle=True)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    a = sys.argv
    main(a[1], a[2], int(a[3]), int(a[4]), int(a[5]), int(a[6]), a[7])
