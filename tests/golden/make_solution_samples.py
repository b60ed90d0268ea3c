"""Write the oracle's converged solution of the n = 255, N = 64 workload
(16 field modes, amplitude 1.0, nu = 1e-6, y_d = sin(pi x) sin(pi y),
seed 2) at a seeded sample of nodes, for checks that cannot afford the
oracle's minute-long solve (the benchmark's error report).

Calls only the oracle and the seeded input module.  The solution is the
oracle's stationary V(2,2) red-black iteration (Algorithm 1, Eq. (13) per
node) run to the paper's relative residual 1e-10 (Sec. 3.2).  Stored per
sampled node i: y[i][0..N), u[i], p[i][0..N), plus each block's largest
magnitude over the whole grid (the scale of the relative errors).

    python tests/golden/make_solution_samples.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import inputs  # noqa: E402
import oracle.cmg_oracle as O  # noqa: E402

CONFIG = "n255_N64"
NODES = 48
NODE_SEED = 20260


def main():
    cfg = inputs.CONFIGS[CONFIG]
    pr = inputs.make_problem(**cfg)
    levels = O.make_hierarchy(pr.n, pr.N, pr.nu, O.sine_mode_field(pr.xi, pr.amp))
    f = O.fine_rhs(levels[0], pr.yd)
    sol = O.solve_stationary(levels, f, O.CycleOptions(), tol=1e-10, maxit=40)
    n, N = pr.n, pr.N
    y = sol.x[0].reshape(n * n, N)
    u = sol.x[1].reshape(n * n)
    p = sol.x[2].reshape(n * n, N)
    idx = np.sort(np.random.default_rng(NODE_SEED).choice(n * n, size=NODES, replace=False))
    out = {
        "source": "oracle/cmg_oracle.py solve_stationary (V(2,2) red-black, Algorithm 1, Eq. (13)) to the paper's "
                  "relative residual 1e-10 (Sec. 3.2); written by tests/golden/make_solution_samples.py",
        "config": CONFIG, "workload": cfg, "cycles": sol.iters, "relres": sol.relres,
        "nodes": [int(i) for i in idx],
        "max_abs": {"y": float(np.abs(y).max()), "u": float(np.abs(u).max()), "p": float(np.abs(p).max())},
        "y": [[float(v) for v in y[i]] for i in idx],
        "u": [float(u[i]) for i in idx],
        "p": [[float(v) for v in p[i]] for i in idx],
    }
    path = os.path.join(HERE, f"{CONFIG}_solution_samples.json")
    with open(path, "w") as fh:
        json.dump(out, fh)
    print(path, sol.iters, sol.relres)


if __name__ == "__main__":
    main()
