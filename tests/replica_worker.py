"""One rank of the replica layout, for the world-size-2 gloo test.

Run as a child process with RANK / WORLD_SIZE / MASTER_ADDR / MASTER_PORT
set: fits its own small dataset with the FP64 oracle (the replica's work),
then takes part in the barrier and the max-over-ranks timing reduction that
the benchmark uses, and writes what it saw to a JSON file.
"""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

CELLS, GENES, CLUSTERS, R_CELLS, K = 120, 24, 4, 6, 3


def replica_fit(seed):
    import numpy as np
    from oracle.fit import fit_two_axis
    from oracle.gram import log1p_centre
    from synth import scrna_counts
    counts = scrna_counts(CELLS, GENES, CLUSTERS, seed=seed).numpy().astype(np.float64)
    fit = fit_two_axis(log1p_centre(counts), R_CELLS, GENES, K, K)
    return {"lam_rows": fit.lam_rows.tolist(), "lam_cols": fit.lam_cols.tolist(),
            "topk_rows": np.asarray(fit.topk_rows[0]).tolist()}


def main(out_pattern, seed, delay_ms):
    import torch.distributed as dist
    from paper_2407_19892_gb300 import replicas
    world, rank, _ = replicas.rank_env()
    dist.init_process_group("gloo", init_method="env://", world_size=world, rank=rank)
    my_seed = replicas.replica_seed(seed, rank)
    fit = replica_fit(my_seed)
    replicas.barrier()
    t0 = time.perf_counter()
    time.sleep(delay_ms * (rank + 1) / 1e3)  # rank 1 is the slow one
    my_ms = (time.perf_counter() - t0) * 1e3
    ms = replicas.max_over_ranks(my_ms)
    replicas.barrier()
    rec = {"rank": rank, "world": world, "seed": my_seed, "my_ms": my_ms, "max_ms": ms,
           "value": replicas.job_throughput(CELLS, world, ms), **fit}
    with open(out_pattern % rank, "w") as f:
        json.dump(rec, f)
    dist.destroy_process_group()


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]), float(sys.argv[3]))
