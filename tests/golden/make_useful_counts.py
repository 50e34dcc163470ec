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

    # NFW halos + stars, uneven refinement batches
    w = lensgen.workload_mixed_batches()
    s, h = w["points"].astype(np.float64), w["nfw"].astype(np.float64)
    comps = oracle.concat(oracle.make_components(oracle.POINT, s[:, 0], s[:, 1], s[:, 2]),
                          oracle.make_components(oracle.NFW, h[:, 0], h[:, 1], h[:, 2], h[:, 3],
                                                 w["conc"] * h[:, 3]))
    g = lensgen.rng(4243)
    idx = lensgen.sample_indices(g, w["dx"].size, 4096)
    b = np.searchsorted(w["offsets"], idx, side="right") - 1
    rx = w["origins"][b, 0] + w["dx"][idx].astype(np.float64)
    ry = w["origins"][b, 1] + w["dy"][idx].astype(np.float64)
    out["mixed_batches_256"] = {th: counts_for(comps, rx, ry, float(th)) for th in ["0.3", "0.1"]}
    out["mixed_batches_256"]["sample"] = "4096 batch rays drawn with PCG64 seed 4243"

    # microlensing: 1e7 stars (the SIS is evaluated once per ray, outside the tree)
    w = lensgen.workload_microlensing()
    s = w["points"].astype(np.float64)
    comps = oracle.make_components(oracle.POINT, s[:, 0], s[:, 1], s[:, 2])
    g = lensgen.rng(4244)
    idx = lensgen.sample_indices(g, w["dx"].size, 4096)
    rx = w["origin"][0] + w["dx"][idx].astype(np.float64)
    ry = w["origin"][1] + w["dy"][idx].astype(np.float64)
    out["microlensing_1e7_4096sq"] = {"0.1": counts_for(comps, rx, ry, 0.1)}
    out["microlensing_1e7_4096sq"]["sample"] = "4096 patch rays drawn with PCG64 seed 4244"

    # lens fit: 1e5 fixed-width Gaussians, 1000^2 grid
    w = lensgen.workload_fit()
    p = w["gauss"].astype(np.float64)
    comps = oracle.make_components(oracle.GAUSS, p[:, 0], p[:, 1], p[:, 2], p[:, 3], w["q"])
    g = lensgen.rng(4245)
    idx = lensgen.sample_indices(g, w["rx"].size, 4096)
    rx, ry = w["rx"][idx].astype(np.float64), w["ry"][idx].astype(np.float64)
    out["fit_1e5_1000sq"] = {th: counts_for(comps, rx, ry, float(th)) for th in ["0.3", "0.1"]}
    out["fit_1e5_1000sq"]["sample"] = "4096 grid rays drawn with PCG64 seed 4245"

    # equal point masses in the unit disk, FP64 64^2 grid over [-1.2, 1.2]^2
    # (the FP64 workload): every ray of the grid
    w = lensgen.workload_point_disk()
    p = w["points"]
    comps = oracle.make_components(oracle.POINT, p[:, 0], p[:, 1], p[:, 2])
    out["point_disk_2000_64sq"] = {"0.1": counts_for(comps, w["rx"], w["ry"], 0.1)}
    out["point_disk_2000_64sq"]["sample"] = "all 4096 grid rays"
    with open(os.path.join(HERE, "useful_counts.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
