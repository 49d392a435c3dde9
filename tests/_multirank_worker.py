"""One rank of the two-rank CPU check of bench.py's multi-rank logic (gloo on
127.0.0.1): prints the reduced step time and a digest of its inputs as JSON."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main():
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 3.0 * rank, dist, "cpu")
    p = bench.rank_problem(2, 1, 3, 3, 16, 8, rank)
    again = bench.rank_problem(2, 1, 3, 3, 16, 8, rank)
    dist.barrier()
    print(json.dumps(dict(rank=rank, ms=ms, digest=float(p.orb.xyz.sum() + p.orb.exps.sum() + p.aux.exps.sum()),
                          deterministic=bool((p.orb.exps == again.orb.exps).all()), npair=int(p.npair),
                          naux=int(p.naux))), flush=True)
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
