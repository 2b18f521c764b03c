"""The cell-sharded fit (paper_2407_19892_gb300.sharded) run as two gloo
processes against the same fit in one process: the exchange pattern and
sizes, and equal results (spectrum, eigenvalue sums, every row's top-k
list).  The CPU test runs the per-process arithmetic through the FP64
oracle (a test double); the GPU test runs the library's kernels in two
processes sharing cuda:0, their exchanges staged through host memory (the
processes' kernels never wait on one another)."""

import os
import socket
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(tmp_path, mode, world, cells, genes, r, k, splits):
    port = _free_port()
    out = str(tmp_path / f"{mode}_w{world}_%d.npy")
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        if mode != "gpu":
            env["CUDA_VISIBLE_DEVICES"] = ""
        procs.append(subprocess.Popen([sys.executable, os.path.join(HERE, "sharded_worker.py"), out, mode,
                                       str(cells), str(genes), str(r), str(k), splits],
                                      env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
    for p in procs:
        try:
            log, _ = p.communicate(timeout=600)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            pytest.fail("sharded ranks did not finish")
        assert p.returncode == 0, log.decode()[-3000:]
    return [np.load(out % r_, allow_pickle=True).item() for r_ in range(world)]


def _expected_log(p, r, nb):
    return [("all_reduce", (p,), "torch.float64"), ("all_reduce", (1,), "torch.float64"),
            ("all_reduce", (p, p), "torch.float64"), ("broadcast", (p,), "torch.float64"),
            ("broadcast", (p, r), "torch.float64"), ("broadcast", (r + p,), "torch.float64"),
            ("all_reduce", (2,), "torch.float64"), ("all_gather", (nb, r), None)]


def _check_log(log, p, r, nb):
    exp = _expected_log(p, r, nb)
    assert len(log) == len(exp)
    for got, want in zip(log, exp):
        assert got[0] == want[0] and tuple(got[1]) == want[1]
        if want[2]:
            assert got[2] == want[2]


CELLS, GENES, R, K = 300, 40, 6, 5


@pytest.fixture(scope="module")
def oracle_runs(tmp_path_factory):
    tmp = tmp_path_factory.mktemp("sharded")
    one = _run(tmp, "oracle", 1, CELLS, GENES, R, K, ",")
    two = _run(tmp, "oracle", 2, CELLS, GENES, R, K, "170")
    return one, two


def test_exchanges_are_the_five_of_the_design(oracle_runs):
    _, two = oracle_runs
    for rec, nb in zip(two, (170, 130)):
        _check_log(rec["log"], GENES, R, nb)


def test_two_processes_equal_one(oracle_runs):
    from oracle.recon import topk_gap
    one, two = oracle_runs
    a = one[0]
    assert [r["row0"] for r in two] == [0, 170] and all(r["n_total"] == CELLS for r in two)
    for rec in two:
        np.testing.assert_allclose(rec["e"], a["e"], rtol=1e-12)
        s1 = a["lr"][:, None] + a["lc"][None, :]
        s2 = rec["lr"][:, None] + rec["lc"][None, :]
        assert np.max(np.abs(s2 - s1) / s1) <= 1e-10
    idx2 = np.concatenate([two[0]["idx"], two[1]["idx"]])
    assert idx2.shape == a["idx"].shape
    assert np.array_equal(idx2, a["idx"])  # FP64 on both sides, same rounding of each row
    assert np.array_equal(two[0]["idx_c"], a["idx_c"]) and two[1]["idx_c"] is None


@pytest.mark.gpu
def test_two_gpu_processes_equal_one(tmp_path, cuda_dev):
    cells, genes, r, k = 20_000, 300, 20, 10
    one = _run(tmp_path, "gpu", 1, cells, genes, r, k, ",")[0]
    two = _run(tmp_path, "gpu", 2, cells, genes, r, k, "11111")
    for rec, nb in zip(two, (11111, cells - 11111)):
        _check_log(rec["log"], genes, r, nb)
    for rec in two:
        # the two processes' Gram partials drain the FP32 accumulation at
        # other cells than one process does: sums agree to that rounding
        s1 = one["lr"][:, None] + one["lc"][None, :]
        s2 = rec["lr"][:, None] + rec["lc"][None, :]
        assert np.max(np.abs(s2 - s1) / s1) <= 1e-5
    idx2 = np.concatenate([two[0]["idx"], two[1]["idx"]])
    assert idx2.shape == one["idx"].shape
    same = np.mean(np.all(np.sort(idx2, 1) == np.sort(one["idx"], 1), axis=1))
    assert same > 0.98
