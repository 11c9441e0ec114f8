"""Writes the regression fixtures of this directory from the FP64 oracle
(and the seeded input module) only:

    python tests/golden/make_golden.py

The paper prints no worked example to copy here (its figures carry the only
results, and Sec. IV gives the setup's ranges, not trajectories), so every
fixture is an oracle output; each records how it was made.  Tests compare
the oracle (not gpu) and the GPU path (gpu) with them.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def single_update():
    """The single robust update (Alg. 1 joint bisection on the FC3 stand-in):
    x_t at the 100 A equilibrium, r = 250 A, 32 Philox scenarios (seed 0,
    update 0), horizon 500, N_kappa = 12."""
    from oracle import oracle as O
    from paper_2510_08288_gb300 import inputs
    w = inputs.WORKLOADS["single"]
    p = inputs.fc3_params()
    x_t = O.equilibrium(p, w["v_prev"])
    d = O.sample_disturbances(w["seed"], w["update"], w["N"], w["H"], inputs.DIST_AMP)
    c = O.cfg(H=w["H"], N=w["N"])
    k, f = O.bisect_joint(p, c, x_t, w["v_prev"], w["r"], w["n_bisect"], d)
    k3, f3 = O.alg3(p, c, x_t, w["v_prev"], w["r"], 2 ** (w["n_bisect"] - 1) + 1, d)
    return {"source": "oracle (FP64): bisect_joint and alg3, written by tests/golden/make_golden.py",
            "cite": "Alg. 1 (joint predicate over the scenarios), Alg. 3, Eq. 2, Eq. 4",
            "workload": dict(w, dist_amp=list(inputs.DIST_AMP)),
            "x_t": [float(v) for v in x_t],
            "kappa": float(k), "flags": int(f),
            "kappa_alg3_dyadic_grid": float(k3), "flags_alg3": int(f3),
            "v_t": float(w["v_prev"] + k * (w["r"] - w["v_prev"]))}


def closed_loop_prefix():
    """The first 10 updates of the closed-loop workload (1,024 scenarios,
    horizon 2,000, staircase r, seed 1, plant disturbances from stream 1)."""
    from oracle import oracle as O
    from paper_2510_08288_gb300 import inputs
    w = inputs.WORKLOADS["closed_loop"]
    p = inputs.fc3_params()
    T = 10
    r = inputs.staircase(w["T"], w["levels"], w["hold"], w["seed"])[:T]
    x0 = O.equilibrium(p, w["v0"])
    v, k, f, xs = O.closed_loop(p, O.cfg(H=w["H"], N=w["N"]), x0, w["v0"], r, w["seed"], 0,
                                inputs.DIST_AMP, inputs.DIST_AMP, search=0, n_kappa=w["n_bisect"],
                                nthreads=os.cpu_count() or 1)
    return {"source": "oracle (FP64): closed_loop with plain joint bisection, written by tests/golden/make_golden.py",
            "cite": "Fig. 1 loop; Alg. 1; Eq. 2; Eq. 4",
            "workload": {"N": w["N"], "H": w["H"], "n_bisect": w["n_bisect"], "seed": w["seed"], "t0": 0,
                         "updates": T, "v0": w["v0"], "staircase": [w["T"], w["levels"], w["hold"], w["seed"]]},
            "r": [float(x) for x in r],
            "kappa": [float(x) for x in k], "flags": [int(x) for x in f], "v": [float(x) for x in v],
            "x": [[float(c) for c in row] for row in xs]}


def main():
    for name, fn in (("single_update.json", single_update), ("closed_loop_prefix.json", closed_loop_prefix)):
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(fn(), f, indent=1)
            f.write("\n")
        print("wrote", name)


if __name__ == "__main__":
    main()
