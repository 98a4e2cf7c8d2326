"""Writes tests/golden/adjoint_n256.json: the FP64 oracle's discrete-adjoint gradient of the
log-power-spectrum loss (Sec. 2's RK4IP integration of Eq. 1, the four-wave-mixing sum taken as
the direct triple sum of Eq. 2 / Eq. 3) for two seeded N = 256 instances over 200 steps.

The oracle's adjoint costs about 2 s per step at N = 256 (direct O(N^3) sums), too long to run
inside a GPU test, so its result is stored here.  Only `oracle/` and the seeded input
generators of `workloads.py` are called; the GPU path plays no part.

    python tests/golden/make_adjoint_n256.py          # about 7 minutes, two processes
"""
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "adjoint_n256.json")

# Recipe shared with tests/test_gpu_adjoint.py (which rebuilds the same inputs).
RECIPE = {
    "N": 256, "h": 2e-3, "nsteps": 200, "D2": 0.01, "D3": 1e-4, "noise": 1e-3,
    "instances": [{"sigma": 3.0, "A_in": [2.0, 0.0], "seed": 4600},
                  {"sigma": 1.0, "A_in": [2.5, 0.5], "seed": 4601}],
    "target": "workloads.sech2_target(256, 2)",
}


def inputs():
    from paper_1307_3428_gb300 import workloads as wl
    r = RECIPE
    insts = [wl.make_instance(r["N"], r["D2"], r["D3"], s["sigma"], complex(*s["A_in"]),
                              r["noise"], seed=s["seed"]) for s in r["instances"]]
    return insts, wl.sech2_target(r["N"], len(insts))


def _one(k):
    import oracle
    insts, T = inputs()
    g = oracle.log_spectrum_grad(insts[k], RECIPE["h"], RECIPE["nsteps"], T[k])
    return {"loss": g["loss"], "sigma": g["sigma"], "D2": g["D2"], "D3": g["D3"],
            "A_in": [g["A_in"].real, g["A_in"].imag],
            "D0": [[z.real, z.imag] for z in g["D0"]],
            "omega": [float(x) for x in g["omega"]], "kappa": [float(x) for x in g["kappa"]]}


def main():
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(len(RECIPE["instances"])) as pool:
        res = pool.map(_one, range(len(RECIPE["instances"])))
    doc = {"what": "FP64 oracle discrete adjoint (direct-sum RK4IP) of the log-power-spectrum "
                   "misfit; per instance: loss and dL/d(sigma, D2, D3, A_in, D0, omega, kappa), "
                   "centred order, complex values as [re, im]",
           "cite": "Sec. 2 (RK4 integration of Eq. 1 with the FWM term of Eq. 2 / Eq. 3)",
           "writer": "tests/golden/make_adjoint_n256.py (calls oracle/ only)",
           "recipe": RECIPE, "instances": res}
    with open(OUT, "w") as fh:
        json.dump(doc, fh, indent=0)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
