"""Host-side logic without a GPU: the bench's cross-rank timing over gloo
(world size 2), its launch count, the reference arm's rank handling, and the
determinism of the seeded scene generators."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

import bench  # noqa: E402
from paper_2503_05046_gb300 import scenes  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_max_over_ranks_and_whole_job_value_gloo_two_ranks():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, os.path.join(ROOT, "tests", "dist_worker.py")],
                                      env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["ws"] == 2
        assert o["max"] == pytest.approx(2.5)          # the slowest rank's time
        assert o["value"] == pytest.approx(2 * 1000.0 / 2.5)  # all ranks' units / that time


def test_single_rank_helpers_are_identities():
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.whole_job_value(10.0, 1, 2.0) == 5.0


@pytest.mark.parametrize("res,n_sub,expected", [
    ((128, 128, 128), 10, 1 + 5 * 3 + 1 + 50),  # 32 blocks per axis: 15 + 6 key bits, 3 passes
    ((40, 16, 24), 1, 1 + 5 * 3 + 1 + 5),       # 10 blocks: 12 + 6 key bits, 3 passes
    ((8, 8, 8), 2, 1 + 5 * 2 + 1 + 10),         # 2 blocks: 3 + 6 key bits, 2 passes
])
def test_kernel_launch_count(res, n_sub, expected):
    assert bench.kernel_launches_per_step(res, n_sub) == expected


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 3
    called = []
    monkeypatch.setattr(bench, "make_scene", lambda *a, **k: called.append(1))
    assert bench.run_reference(Args()) is None
    assert called == []
    assert capsys.readouterr().out == ""


def test_scene_generators_are_seeded():
    a = scenes.granular_scoop(n_particles=20_000)
    b = scenes.granular_scoop(n_particles=20_000)
    np.testing.assert_array_equal(a["groups"][0]["x"], b["groups"][0]["x"])
    np.testing.assert_array_equal(a["groups"][0]["v"], b["groups"][0]["v"])
    assert len(a["groups"][0]["x"]) == 20_000
    c = scenes.cube_contact(n_side=6, v0=(0.0, 0.0, -0.05))
    d = scenes.cube_contact(n_side=6, v0=(0.0, 0.0, -0.05))
    for ga, gb in zip(c["groups"], d["groups"]):
        np.testing.assert_array_equal(ga["x"], gb["x"])


def test_bench_config_names_the_workload():
    sc = scenes.granular_scoop(n_particles=10_000)
    cfg = bench.bench_config(sc, 10_000, 1)
    assert cfg["workload"] == bench.WORKLOAD
    assert cfg["particles"] == 10_000
    assert cfg["substeps_per_step"] == sc["substeps"]
    assert "model" not in cfg
