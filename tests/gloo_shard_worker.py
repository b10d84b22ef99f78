"""One rank of the 2-process CPU (gloo) sharding test, launched by
torch.distributed.run from tests/test_sharding.py.  Each rank evaluates the
oracle's lightcone terms for its own edge range, then the library's
reduce_partials sums E and a per-rank gradient stand-in over the ranks."""
import json
import os
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent
sys.path.insert(0, str(ROOT))

import numpy as np  # noqa: E402
import torch  # noqa: E402
import torch.distributed as dist  # noqa: E402

from oracle import lightcone as lc  # noqa: E402
from paper_2106_15740_gb300.sharding import edge_costs, partition, reduce_partials  # noqa: E402
from workloads import random_angles, random_regular_graph  # noqa: E402


def main():
    out = Path(sys.argv[1])
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    n, p, B = 12, 2, 2
    edges = random_regular_graph(n, 3, 21)
    g, b = random_angles(B, p, 77)
    ranges = partition(edge_costs(n, edges, p, batch=B), world)
    a, e1 = ranges[rank]
    part = np.zeros(B)
    for k in range(B):
        for e in range(a, e1):
            part[k] += 0.5 * (1.0 - lc.lightcone_zz(n, edges, p, g[k], b[k], e)[0].real)
    grad = torch.full((B, 2 * p), float(rank + 1), dtype=torch.float64)
    e_tot, g_tot = reduce_partials(torch.tensor(part), grad)
    res = dict(rank=rank, world=world, range=[a, e1], ranges=ranges, partial=part.tolist(),
               energy=e_tot.tolist(), grad=g_tot.tolist())
    (out / f"rank{rank}.json").write_text(json.dumps(res))
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    main()
