"""Write the FP64 oracle's per-scan OSPA record of whole runs of a workload.

Calls only the oracle and the scenario generator: for each seed, the oracle
filter (Algorithm 1 with K = 1 for the global workloads) runs every scan of
`scenario.simulate(w, seed)` with the scenario's injected random numbers,
rounded to FP32 exactly as the GPU path receives them (`step_noise(...,
float32)`, `resample_u32`), and the record keeps per scan the OSPA of its
estimates against the truth (c = 100 m, p = 2 and p = 1), its mass N_k, the
number of estimates and of truth targets.  The benchmark compares the GPU
filter's OSPA on the same seeds and scans with it (matched OSPA).

    python tests/golden/make_oracle_ospa.py dense_rb_100t 0 1 2

runs the oracle on all host cores (its OpenMP build, bit-identical to the
single-threaded one) and writes tests/golden/oracle_ospa_<workload>.json.
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import scenario  # noqa: E402


def run(wname: str, seed: int) -> dict:
    w = scenario.workload(wname)
    sc = scenario.simulate(w, seed)
    f = oracle.OracleFilter(w)
    K = w.num_pe
    rows = []
    t0 = time.time()
    for k, Z in enumerate(sc.meas):
        noise = scenario.step_noise(seed, k, K, w.pe_cap, np.float32)
        xu = scenario.exchange_u32(seed, k, K, w.pe_cap) if K > 1 else None
        lab, zet = f.step(Z, noise, scenario.resample_u32(seed, k, K), xu)
        X = zet[:, [0, 2]] if len(zet) else np.zeros((0, 2))
        tr = sc.truth[k]
        Y = tr[:, [0, 2]] if len(tr) else np.zeros((0, 2))
        rows.append({"scan": k, "ospa2": oracle.ospa(X, Y, 100.0, 2.0), "ospa1": oracle.ospa(X, Y, 100.0, 1.0),
                     "mass": float(np.sum(f.last["Nk"])), "estimates": int(len(lab)), "truth": int(len(tr))})
    return {"seed": seed, "seconds": round(time.time() - t0, 1), "scans": rows}


def main(argv):
    wname = argv[1]
    seeds = [int(s) for s in argv[2:]] or [0]
    oracle.set_threads(os.cpu_count() or 1)
    out = {"workload": wname, "generator": "tests/golden/make_oracle_ospa.py", "ospa": {"c": 100.0, "p": [2, 1]},
           "noise": "scenario.step_noise(seed, scan, K, pe_cap, float32), resample_u32, exchange_u32",
           "host": platform.machine(), "oracle_threads": oracle.threads(), "runs": []}
    for s in seeds:
        r = run(wname, s)
        print(f"seed {s}: {r['seconds']} s, mean OSPA (p=2) scans 50+: "
              f"{np.mean([x['ospa2'] for x in r['scans'][50:]]):.2f}", flush=True)
        out["runs"].append(r)
    path = os.path.join(HERE, f"oracle_ospa_{wname}.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=0)
    print(path)


if __name__ == "__main__":
    main(sys.argv)
