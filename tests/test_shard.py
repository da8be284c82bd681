"""Sharding of independent scenes across ranks: the greedy assignment, and a two-rank
gloo run (CPU, oracle arithmetic) whose gathered per-scene results equal a single
process's."""
import os
import socket

import numpy as np
import pytest

from paper_2311_04648_gb300 import shard


def test_assignment_covers_every_scene_once_and_balances():
    rng = np.random.default_rng(4)
    costs = np.round(np.exp(rng.uniform(np.log(1e3), np.log(5e4), size=512)))
    for n_ranks in (1, 2, 3, 8):
        parts = shard.assign(costs, n_ranks)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(costs)))
        ld = shard.loads(costs, parts)
        assert max(ld) - sum(ld) / n_ranks <= costs.max() + 1e-9
        assert parts == shard.assign(costs, n_ranks)      # deterministic
    assert shard.assign([5.0, 5.0, 1.0], 2) == [[0, 2], [1]]
    with pytest.raises(ValueError):
        shard.assign([1.0], 0)


def _scenes():
    from paper_2311_04648_gb300 import workloads as W
    return [W.free_spheres(n=40 + 15 * k, seed=50 + k, vel_sigma=0.4) for k in range(5)]


def _run(scene):
    import oracle
    o = oracle.OracleWorld(scene)
    assert o.step(30) == 0
    ke = o.diagnostics()["ke"]
    return [float(ke), o.x.tobytes().hex()]


def _rank(rank, world, port, out_path):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        scenes = _scenes()
        parts = shard.assign([s.n_sphere * 30 for s in scenes], world)
        local = {k: _run(scenes[k]) for k in parts[rank]}
        res = shard.gather_results(local, len(scenes))
        if rank == 0:
            import json
            with open(out_path, "w") as f:
                json.dump(res, f)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_gather_the_single_process_results(tmp_path):
    import json
    import torch.multiprocessing as mp

    out = os.path.join(str(tmp_path), "res.json")
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = json.load(open(out))
    want = [_run(s) for s in _scenes()]
    assert got == want
