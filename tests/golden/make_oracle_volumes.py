"""Writes oracle_volumes.json: exact degrees of the seeded benchmark systems, computed by the
oracle only (Python big-int Smith form + placing-triangulation volume).  No value here comes
from the CUDA path.  Run: python tests/golden/make_oracle_volumes.py"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.degree import degree  # noqa: E402
from workloads import CONFIGS, batch_systems, config_system  # noqa: E402


def main():
    out = {"source": "oracle/degree.py (placing triangulation), systems from workloads/", "configs": {},
           "batch_first_256": []}
    for name in CONFIGS:
        s = config_system(name)
        t = time.time()
        r = degree(s.A.tolist())
        out["configs"][name] = dict(degree=r.degree, nvol=r.nvol, torsion=r.torsion, rank=r.rank, dim=r.dim,
                                    oracle_seconds=round(time.time() - t, 3))
        print(name, out["configs"][name], flush=True)
    for s in batch_systems(256):
        r = degree(s.A.tolist())
        out["batch_first_256"].append(dict(seed=s.meta["batch_seed"], degree=r.degree, nvol=r.nvol,
                                           torsion=r.torsion, dim=r.dim))
    with open(os.path.join(HERE, "oracle_volumes.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
