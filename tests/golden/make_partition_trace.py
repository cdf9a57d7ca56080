"""Writes tests/golden/partition_trace.json: full traces of small multilevel partitions (every level's
size, cluster bound U and seed, every initial-partitioning try's seed, cut and balance, the try kept,
the cut after each projection and refinement, the final partition), computed by the step-by-step
restatement of the multilevel scheme in tests/test_oracle_driver.py, which calls only the oracle's
separately pinned primitives. tests/test_oracle_driver.py checks the oracle's driver against it.

    python tests/golden/make_partition_trace.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import graphgen as gg  # noqa: E402
import oracle as O  # noqa: E402
from test_oracle_driver import EPS, _params, _path, restated_partition  # noqa: E402

CASES = [
    # 4x6 grid, k=2: U = max(1, floor(12 / 2)) = 6, T = 4, so that exactly two contractions happen
    {"grid": [4, 6], "k": 2, "seed": 1, "params": {"coarse_min": 4, "coarse_per_k": 1, "cluster_div": 2}},
    # path of 30 vertices, k=3, seven tries
    {"path_n": 30, "k": 3, "seed": 7, "params": {"coarse_min": 6, "coarse_per_k": 1, "cluster_div": 2,
                                                  "ip_tries": 7}},
]


def main():
    out = []
    for c in CASES:
        g = _path(c["path_n"]) if "path_n" in c else gg.grid(*c["grid"])
        part, tr = restated_partition(g, c["k"], EPS, c["seed"], _params(**c["params"]))
        tr["levels"] = [{k: (str(v) if k == "seed" else v) for k, v in x.items()} for x in tr["levels"]]
        for x in tr.get("tries", []):
            x["s_try"] = str(x["s_try"])
        out.append({**c, "trace": tr, "part": [int(x) for x in part]})
    with open(os.path.join(HERE, "partition_trace.json"), "w") as f:
        json.dump({"eps": EPS, "cases": out}, f, indent=1)
    for c in out:
        print(c.get("grid", c.get("path_n")), "levels", len(c["trace"]["levels"]), "level_n", c["trace"]["level_n"])


if __name__ == "__main__":
    main()
