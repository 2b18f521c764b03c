"""World-size-2 runs of the replica layout on CPU (gloo): each rank fits its
own dataset, ranks meet only at the barrier and the max-over-ranks step time,
and the job rate is the units of all ranks over the slowest rank's time."""

import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

import replica_worker as rw  # noqa: E402
from paper_2407_19892_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_world(tmp_path, world, seed=7, delay_ms=60.0):
    port = _free_port()
    out = str(tmp_path / "rank%d.json")
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, os.path.join(HERE, "replica_worker.py"), out, str(seed),
                                       str(delay_ms)], env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
    for p in procs:
        try:
            log, _ = p.communicate(timeout=240)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            pytest.fail("replica ranks did not finish")
        assert p.returncode == 0, log.decode()[-2000:]
    return [json.load(open(out % r)) for r in range(world)]


@pytest.fixture(scope="module")
def world2(tmp_path_factory):
    return _run_world(tmp_path_factory.mktemp("w2"), 2)


def test_every_rank_sees_the_slowest_rank_time(world2):
    own = [r["my_ms"] for r in world2]
    assert own[1] > own[0]
    for r in world2:
        assert r["max_ms"] == pytest.approx(max(own), rel=0, abs=0)


def test_job_rate_counts_every_rank_over_the_slowest_time(world2):
    for r in world2:
        assert r["value"] == pytest.approx(2 * rw.CELLS / (max(x["my_ms"] for x in world2) / 1e3), rel=1e-12)
    assert replicas.job_throughput(1000, 4, 500.0) == pytest.approx(8000.0)


def test_ranks_fit_different_datasets(world2):
    assert world2[0]["seed"] != world2[1]["seed"]
    assert not np.allclose(world2[0]["lam_rows"], world2[1]["lam_rows"])


def test_a_rank_result_does_not_depend_on_the_world_size(world2):
    # rank r of a 2-rank job computes exactly what one process computes on
    # the same replica seed: no data-path exchange
    for r in world2:
        solo = rw.replica_fit(r["seed"])
        np.testing.assert_array_equal(np.asarray(r["lam_rows"]), np.asarray(solo["lam_rows"]))
        np.testing.assert_array_equal(np.asarray(r["lam_cols"]), np.asarray(solo["lam_cols"]))
        np.testing.assert_array_equal(np.asarray(r["topk_rows"]), np.asarray(solo["topk_rows"]))


def test_single_process_helpers_need_no_process_group(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("LOCAL_RANK", raising=False)
    assert replicas.rank_env() == (1, 0, 0)
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.replica_seed(10, 0) == 10 and replicas.replica_seed(10, 3) == 13
    replicas.barrier()
