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
        assert o["shard_total"] == 10                   # scenes counted over the ranks
    # the batched scenes split over the ranks: disjoint, together all of them
    a, b = (set(o["shard"]) for o in sorted(outs, key=lambda o: o["rank"]))
    assert not (a & b) and a | b == set(range(10))


def test_single_rank_helpers_are_identities():
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.whole_job_value(10.0, 1, 2.0) == 5.0


@pytest.mark.parametrize("res,n_sub,nb,expected", [
    ((128, 128, 128), 10, 7, 1 + 5 * 3 + 1 + 60 + 1),  # 32 blocks per axis: 15 + 6 key bits, 3 passes
    ((320, 184, 64), 10, 12, 1 + 5 * 4 + 1 + 60 + 1),  # 80 blocks: 21 + 6 key bits, 4 passes
    ((40, 16, 24), 1, 0, 1 + 5 * 3 + 1 + 6),           # 10 blocks: 12 + 6 key bits, 3 passes; no bodies
    ((8, 8, 8), 2, 1, 1 + 5 * 2 + 1 + 12 + 1),         # 2 blocks: 3 + 6 key bits, 2 passes
])
def test_kernel_launch_count(res, n_sub, nb, expected):
    assert bench.kernel_launches_per_step(res, n_sub, nb) == expected


def test_kernel_launch_count_small_scene():
    # up to 8,192 particles the sort is one block and the permutation
    assert bench.kernel_launches_per_step((64, 64, 64), 10, 2, n_particles=8000) == 2 + 60 + 1
    assert bench.kernel_launches_per_step((64, 64, 64), 10, 2, n_particles=8193) == \
        bench.kernel_launches_per_step((64, 64, 64), 10, 2)


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
    assert cfg["workload"] == "granular_scoop_10000"
    assert cfg["particles"] == 10_000
    assert cfg["substeps_per_step"] == sc["substeps"]
    assert "model" not in cfg
    big = bench.make_scene(bench.SECONDARY)
    assert bench.workload_name(big) == bench.SECONDARY == "granular_scoop_1M"
    head = bench.make_scene(bench.WORKLOAD)
    assert bench.workload_name(head) == bench.WORKLOAD == "mixed_manipulation_4M"
    cfg = bench.bench_config(head, scenes.n_particles(head), 1)
    assert cfg["objects"] == 32 and cfg["bodies"] == 12
    assert cfg["materials"] == ["corotated_elastic", "drucker_prager_sand"]


class _FakeSim:
    """Stands in for native.Sim: records the calls the autograd binding makes
    and keeps native.Sim's rule that replacing the bodies clears their
    dynamics."""

    def __init__(self, n, bodies):
        self.n, self.ctx, self.calls = n, None, []
        self.scene = {"groups": [{"material": {"model": 0, "E": 1e4, "nu": 0.3, "rho": 1e3}}]}
        self._bodies = [dict(b) for b in bodies]
        self.dynamics = {}

    def bodies(self):
        return [dict(b) for b in self._bodies]

    def set_bodies(self, bodies):
        self.calls.append(("set_bodies", [dict(b) for b in bodies]))
        self._bodies = [dict(b) for b in bodies]
        self.dynamics = {}

    def set_dynamics(self, i, d):
        self.calls.append(("set_dynamics", i))
        self.dynamics[i] = d

    def set_particles(self, *a):
        pass

    def tape_begin(self):
        self.calls.append(("tape_begin", dict(self.dynamics)))

    def step(self, solver=None):
        for b in self._bodies:  # bodies move over a step
            b["p"] = np.asarray(b["p"]) + 1.0

    def tape_end(self):
        pass

    device = None  # torch.device("cpu") once torch is imported (see below)

    def get_particles(self):
        return {"x": np.zeros((self.n, 3), np.float32), "v": np.zeros((self.n, 3), np.float32)}

    def read_particles(self, x=None, v=None, Cm=None, F=None):
        for a in (x, v, Cm, F):
            if a is not None:
                a.zero_()

    def backward(self, x_bar=None, v_bar=None, eps_r=None):
        import torch
        return {"x": torch.ones((self.n, 3)), "v": torch.ones((self.n, 3)), "E": [2.0], "nu": [3.0],
                "mu": [4.0], "body_v": [[5.0, 6.0, 7.0]]}


def test_autograd_rollout_keeps_dynamics_and_start_bodies(monkeypatch):
    """The rollout replaces the bodies (to apply mu and body_v), which clears
    dynamics; it sets them again before recording. An explicit `bodies`
    repeats a rollout from the same start; the gradients come back in the
    inputs' dtypes."""
    import torch
    from paper_2503_05046_gb300 import autograd, native
    monkeypatch.setattr(native, "mpm_set_material", lambda ctx, gi, m: None)
    b0 = {"p": np.zeros(3), "v": np.array([0.1, 0.0, 0.0]), "mu": 0.5}
    sim = _FakeSim(4, [b0])
    sim.device = torch.device("cpu")
    sim.set_dynamics(0, {"mass": 1.0, "inertia": [1.0, 1.0, 1.0]})
    x0 = torch.zeros(4, 3)
    v0 = torch.zeros(4, 3, requires_grad=True)
    E = torch.tensor([1e4], dtype=torch.float64, requires_grad=True)
    nu = torch.tensor([0.3], dtype=torch.float64)
    mu = torch.tensor([0.7], dtype=torch.float64, requires_grad=True)
    for start, p_start in ((None, 0.0), (None, 2.0), ([b0], 0.0)):
        sim.calls.clear()
        xf, vf = autograd.rollout(sim, 2, x0, v0, E, nu, mu, bodies=start)
        kinds = [c[0] for c in sim.calls]
        assert kinds.index("set_dynamics") > kinds.index("set_bodies")
        assert sim.calls[kinds.index("tape_begin")][1] == {0: {"mass": 1.0, "inertia": [1.0, 1.0, 1.0]}}
        set_to = sim.calls[kinds.index("set_bodies")][1][0]
        assert set_to["mu"] == 0.7 and np.allclose(set_to["v"], [0.1, 0.0, 0.0])
        assert np.allclose(set_to["p"], p_start)  # the default follows the moved bodies
    (xf.sum() + vf.sum()).backward()
    assert v0.grad.dtype == torch.float32 and torch.all(v0.grad == 1.0)
    assert E.grad.item() == 2.0 and mu.grad.item() == 4.0


def test_traffic_table_covers_every_kernel_the_bench_reports():
    """Every (kernel, workload) key bench.py may ask `profiles/traffic.txt` for
    has a line: each P2G form and block size the tuner can choose, and G2P,
    on both bench workloads; the scaled value is proportional to n."""
    import inspect
    from paper_2503_05046_gb300 import tune
    cands = inspect.signature(tune.tune_p2g_form).parameters["candidates"].default
    keys = ["p2g_%s_%d" % (("gather", "scatter")[f], c) for f, c in cands]
    keys.append("g2p")
    for wl, n in (("mixed_manipulation_4M", 3997168), ("granular_scoop_1M", 1000000)):
        for k in keys:
            t = bench.profiled_traffic(k, wl, n)
            assert t is not None, (k, wl)
            # within [0.5, 1.5] of the algorithmic bytes: a capture of this kernel
            alg = (bench.G2P_BYTES_PER_PARTICLE * n if k == "g2p" else
                   bench.P2G_BYTES_PER_PARTICLE * n)
            assert 0.5 * alg < t < 1.5 * alg + 16 * 2e6, (k, wl, t, alg)
            assert bench.profiled_traffic(k, wl, 2 * n) == pytest.approx(2 * t)
    assert bench.profiled_traffic("p2g_gather_512", "mixed_manipulation_4M", 1) is None


def test_clock_sampler_parses_clocks_and_throttle_reasons(tmp_path):
    """The nvidia-smi samples of the timed region: median SM clock, the
    highest maximum clock, and every throttle reason seen Active (a run with
    hw_slowdown or a thermal reason is rejected; sw_power_cap is kept)."""
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 2055, 2070, 1010.0, 0x8, Active, Not Active, Not Active, Not Active\n")
        f.write("0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("a short line\n")

    class FakeSmi:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s.proc = FakeSmi()
    s.out = open(os.devnull, "w")
    r = s.stop()
    assert r == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0,
                 "reasons": ["hw_slowdown", "sw_power_cap"], "samples": 3}
    assert not os.path.exists(s.path)
    assert bench.ClockSampler(0).stop() is None  # never started: no clock record
