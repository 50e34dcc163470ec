"""Write useful_counts.json: per-ray interaction counts of the paper's tree
(Sec. 3.2 algorithm as the oracle implements it: leaf < 5 particles, per-ray
MAC, big-particle lists) on a 4,096-ray sample of each benchmark workload.

These counts, times the per-interaction flop table, are the "useful" work the
roofline fraction divides by: work the GPU does beyond them (a group MAC
opens more boxes than any one ray needs) is not counted.  Calls only the
input generators and oracle/.  Run:  python tests/golden/make_useful_counts.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import lensgen  # noqa: E402
import oracle  # noqa: E402


def counts_for(comps, rx, ry, theta, leaf_max=5):
    t = oracle.PaperTree(comps, leaf_max, theta)
    _, cnt = t.eval(rx, ry)
    keys = ["far_cells", "near_point", "near_full", "big_corrections", "boxes_visited"]
    return {k: float(v) for k, v in zip(keys, cnt.mean(axis=0))}


def main():
    out = {}
    # smoothed NFW particles, 2048^2 grid over [-1, 1]^2 (the headline workload)
    w = lensgen.workload_nfw_sph()
    p = w["gauss"].astype(np.float64)
    comps = oracle.make_components(oracle.GAUSS, p[:, 0], p[:, 1], p[:, 2], p[:, 3], w["q"])
    g = lensgen.rng(4242)
    idx = lensgen.sample_indices(g, w["rx"].size, 4096)
    rx, ry = w["rx"][idx].astype(np.float64), w["ry"][idx].astype(np.float64)
    out["nfw_sph_1e6_2048sq"] = {th: counts_for(comps, rx, ry, float(th)) for th in ["0.3", "0.1"]}
    out["nfw_sph_1e6_2048sq"]["sample"] = "4096 grid rays drawn with PCG64 seed 4242"
    with open(os.path.join(HERE, "useful_counts.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
