"""Write tests/golden/flop_model.json: the algorithmic flop model of the
classification for the benchmark workloads, counted by the oracle.

Run: python -m oracle.flop_model   (calls only the oracle and the input generator)
"""
import json
import os

import oracle
from paper_1809_04352_gb300 import inputs

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                   "flop_model.json")


def main():
    res = {"_unit_costs": {"per_reach_atom": 8, "per_face_candidate": 12, "per_face_freeness_test": 8,
                           "per_saddle_candidate": 30, "per_concave_candidate": 8,
                           "per_edge_sphere_candidate": 20, "per_edge_torus_candidate": 150},
           "_written_by": "python -m oracle.flop_model"}
    for cfg in (1, 2):
        wl = inputs.WORKLOADS[cfg]
        xyz, rad = inputs.workload_atoms(cfg)
        c = oracle.flop_counts(xyz, rad, wl.r_p, wl.h, wl.margin)
        c["flops_per_point"] = c["model_flops"] / c["points"]
        # edge terms: the oracle's own crossing edges (Algorithm 1 over 64-point blocks)
        r = oracle.run(xyz, rad, wl.r_p, wl.h, wl.margin, block_pts=64)
        ec = oracle.edge_flop_counts(xyz, rad, wl.r_p, wl.h, wl.margin, r.idx)
        c["edge_counts"] = ec
        c["edge_flops_per_edge"] = ec["model_flops"] / max(ec["edges"], 1)
        c.update(workload=wl.name, n_atoms=int(xyz.shape[0]), r_p=wl.r_p, h=wl.h, margin=wl.margin)
        res[wl.name] = c
        print(wl.name, c)
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
