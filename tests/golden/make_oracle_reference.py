"""Write tests/golden/oracle_full_size.json: the FP64 CPU oracle's results on
the full-size workloads (2048^2 correlated networks, 256^3 percolation).

Calls only the oracle and the seeded input generators.  Each entry records the
effective conductance (Eq. 4 flow / pressure drop), the CG iteration count of
the oracle's Jacobi-PCG, its final relative residual and the wall time, so
that the full-size parity tests and the CPU-baseline scaling can use them
without re-running a solve of many minutes.  For the 2048^2 networks it also
stores the pressures of a strided sample of nodes (every 32nd row from row 7,
every 32nd column from column 3: 64 x 64 nodes) for an element-by-element
comparison.

    python tests/golden/make_oracle_reference.py [case ...]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1908_03301_gb300 import netgen  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_full_size.json")

CASES = {
    "fbm2048_iso_x": lambda: (netgen.workload_fbm2d(variant="isotropic"), 0),
    "fbm2048_strat_x": lambda: (netgen.workload_fbm2d(variant="stratified"), 0),
    "fbm2048_strat_y": lambda: (netgen.workload_fbm2d(variant="stratified"), 1),
    "perc256_x": lambda: (netgen.workload_perc3d(), 0),
}


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        (dims, planes), f = CASES[name]()
        t = time.time()
        r = oracle.solve(dims, planes, flow_axis=f, tol=1e-13)
        dt = time.time() - t
        data[name] = {"dims": list(dims), "flow_axis": f, "g_eff": r.g_eff, "q_out": r.q_out,
                      "energy_g": r.energy_g, "iters": r.iters, "rel_residual": r.rel_residual,
                      "max_imbalance": r.max_imbalance, "n_active": r.n_active,
                      "status": r.status, "seconds": dt, "threads": oracle.max_threads(),
                      "tol": 1e-13}
        if len(dims) == 2:
            rows = list(range(7, dims[1], 32))
            cols = list(range(3, dims[0], 32))
            data[name]["P_sample"] = {"rows": rows, "cols": cols,
                                      "values": [[float(v) for v in r.P[y, cols]] for y in rows]}
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        print(name, data[name], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
