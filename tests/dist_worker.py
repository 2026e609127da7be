"""One rank of the two-process gloo test of the bench's cross-rank timing
(run by tests/test_host_logic.py with RANK / WORLD_SIZE / MASTER_* set)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main():
    dist.init_process_group("gloo")
    ws, rank, _ = bench.dist_env()
    seconds = 1.5 + rank  # rank r took 1.5 + r seconds
    worst = bench.max_over_ranks(seconds, ws)
    value = bench.whole_job_value(1000.0, ws, worst)
    mine = bench.shard(10, rank, ws)
    total = bench.sum_over_ranks(float(len(mine)), ws)
    dist.barrier()
    dist.destroy_process_group()
    print(json.dumps({"rank": rank, "ws": ws, "max": worst, "value": value, "shard": mine,
                      "shard_total": total}))


if __name__ == "__main__":
    main()
