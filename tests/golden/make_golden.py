"""Writes oracle_dcpfphd_small.json: a small DCPFPHD run of the FP64 oracle
(Algorithm 1, Steps 1-6) on seeded inputs, as a regression record of the
oracle's own outputs.  Calls only `oracle` (and the seeded input generators
of `scenario`); run it from the repository root:

    python tests/golden/make_golden.py

A change to the oracle's arithmetic that moves these numbers has to be
justified by the passage of the paper (or the reading of it) it follows."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle     # noqa: E402
import scenario   # noqa: E402

SEED, STEPS = 17, 6


def workload():
    """4 PEs, 3 targets present from scan 1, linear sensor, 10 % ring exchange."""
    return scenario.workload("dist16_10t", num_pe=4, n_targets=3, clutter_rate=8.0, particles_per_target=200,
                             birth_count=120, birth_steps=(1, 1, 1), exchange_frac=0.1, steps=STEPS)


def run():
    w = workload()
    sc = scenario.simulate(w, SEED)
    # each PE starts with a seeded cloud around the scan-1 truth (mass 3 / K)
    rng = np.random.default_rng(SEED)
    centres = sc.truth[0][:, [0, 2]]
    init = [scenario.random_particles(rng, w, 40 + 5 * j, centres=centres, spread=20.0, mass=3.0 / w.num_pe)
            for j in range(w.num_pe)]
    f = oracle.OracleFilter(w, [a for a, _ in init], [b for _, b in init])
    out = []
    for k in range(STEPS):
        noise = scenario.step_noise(SEED, k, w.num_pe, w.pe_cap)
        U = scenario.resample_u32(SEED, k, w.num_pe)
        xu = scenario.exchange_u32(SEED, k, w.num_pe, w.pe_cap)
        lab, zet = f.step(sc.meas[k], noise, U, xu)
        L = f.last
        out.append({
            "scan": k,
            "M": int(len(sc.meas[k])),
            "C_local": [np.asarray(c).tolist() for c in L["C_local"]],
            "N": [float(v) for v in L["Nk"]],
            "local_labels": [np.asarray(e.labels).tolist() for e in L["extract"]],
            "fused_labels": np.asarray(lab).tolist(),
            "fused_states": np.asarray(zet).tolist(),
            "resample_counts": [int(len(p)) for p in L["parents"]],
            "parents_head": [np.asarray(p[:16]).tolist() for p in L["parents"]],
        })
    return out


if __name__ == "__main__":
    path = os.path.join(HERE, "oracle_dcpfphd_small.json")
    with open(path, "w") as fh:
        json.dump({"seed": SEED, "steps": STEPS, "cite": "Algorithm 1, Steps 1-6; Eq. 5-8, 10-18",
                   "record": run()}, fh, indent=1)
    print("wrote", path)
