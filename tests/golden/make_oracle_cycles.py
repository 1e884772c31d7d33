"""Writes oracle_cycles_sphere256.json: the number of V-cycles the FP64 oracle
needs to reach a relative residual of 1e-8 on the 256^3 uniform-sphere
workload with the benchmark's solver settings (RKL2 smoother, s = 3,
tau = 0.9 tau_max, N_pre = 5, N_post = 3 on the finest level and 3, 2 on the
levels below it, five levels, coarse tolerance 1e-2).
The CPU reference arm of bench.py times one oracle V-cycle and multiplies by
this count.  Calls only oracle/ and workloads/ (a few minutes of CPU time).

    python tests/golden/make_oracle_cycles.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def main():
    p = W.sphere(256)
    opts = O.Options(rkl_order=2, s_smooth=3, tau_frac=0.9, n_pre=5, n_post=3, inner_n_pre=3, inner_n_post=2,
                     coarse_tol=1e-2, coarse_max_ss=64)
    _, info = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, 1.0, tol=1e-8, levels=5, opts=opts)
    out = {"workload": "sphere256", "tol": 1e-8, "levels": 5,
           "solver": "RKL2 s=3 tau_frac=0.9 n_pre=5 n_post=3 inner_n_pre=3 inner_n_post=2 coarse_tol=1e-2 "
                     "coarse_max_ss=64",
           "cycles": int(info.cycles), "final_rel_residual": float(info.history[-1])}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_cycles_sphere256.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
