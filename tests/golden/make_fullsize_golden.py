"""Write the FP64 oracle's whole-registration results for the full-size
single-pair workloads 1 and 3 (tests/golden/fullsize_*.json), which the GPU
parity test `test_gpu_fullsize_parity.py` reads as expected values.

Calls only the oracle (oracle/) on inputs from the seeded generator module
(paper_2007_07627_gb300.synth, which holds none of the method's arithmetic).
The correspondence step is the oracle's k-d tree query, pinned to equal its
exhaustive search bit for bit (tests/test_oracle_pins.py), so the results are
those of the exhaustive oracle.

    python tests/golden/make_fullsize_golden.py [1] [3]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2007_07627_gb300 import synth  # noqa: E402

# workload -> (variant, parameter overrides): workload 1 is Fast ICP capped at
# 100 iterations; workload 3 is Welsch point-to-plane with the paper's defaults.
WORKLOADS = {1: ("p2p", dict(max_iters=100)), 3: ("p2pl_welsch", {})}


def path(cfg):
    v, _ = WORKLOADS[cfg]
    return os.path.join(HERE, f"fullsize_config{cfg}_{v}.json")


def main(cfgs):
    for cfg in cfgs:
        variant, over = WORKLOADS[cfg]
        pair = synth.config_pair(cfg)
        t0 = time.time()
        r = oracle.register(pair.P, pair.Q, oracle.Params(variant=variant, nn="kdtree", **over),
                            normals=pair.normals)
        out = {
            "workload": cfg, "variant": variant, "overrides": over, "M": pair.M, "N": pair.N,
            "seed": synth.CONFIG_SEEDS[cfg], "status": r["status"],
            "R": r["R"].tolist(), "t": r["t"].tolist(),
            "iterations": r["iterations"], "corr_passes": r["corr_passes"], "reverts": r["reverts"],
            "aa_accepted": r["aa_accepted"], "line_search_trials": r["line_search_trials"],
            "stages": r["stages"], "nu_max": r["nu_max"], "nu_min": r["nu_min"],
            "final_energy": r["final_energy"], "trace": np.asarray(r["trace"]).tolist(),
            "oracle_seconds": round(time.time() - t0, 1),
        }
        with open(path(cfg), "w") as f:
            json.dump(out, f, indent=1)
        print(cfg, variant, "iterations", r["iterations"], "passes", r["corr_passes"],
              "seconds", out["oracle_seconds"], flush=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [1, 3])
