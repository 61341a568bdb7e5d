"""Write the golden files of this directory from the CPU oracle alone.

Each file records one oracle result on a seeded synthetic input:
  solve_12x5_seed0.json   exact solve, 12 jobs x 5 machines, p uniform [1,99]
                          from seed 0, depth-first, UB = +inf, pool 1024
                          (Sec. II-A operators, Sec. III pool selection)
  bound_20x20_seed1.json  bounds of the first 64 nodes of the 20 x 20 seed-1
                          bounding workload (prefixes of random permutations)
Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1206_4973_gb300 import inputs  # noqa: E402


def main():
    n, m, seed, pool = 12, 5, 0, 1024
    p = inputs.instance(n, m, seed)
    r = oracle.solve(p, pool=pool)
    g = {"kind": "solve", "n": n, "m": m, "seed": seed, "pool": pool, "ub0": oracle.INF,
         "cmax": r["cmax"], "perm": [int(x) for x in r["perm"]]}
    g.update({k: r[k] for k in oracle.STATS})
    with open(os.path.join(HERE, "solve_12x5_seed0.json"), "w") as f:
        json.dump(g, f, indent=1)
    n, m, seed, count = 20, 20, 1, 64
    p, _, nodes = inputs.pool_workload(n, m, seed, count)
    g = {"kind": "bound_pool", "n": n, "m": m, "seed": seed, "count": count,
         "lb": oracle.bound_pool(p, nodes).tolist()}
    with open(os.path.join(HERE, "bound_20x20_seed1.json"), "w") as f:
        json.dump(g, f)


if __name__ == "__main__":
    main()
