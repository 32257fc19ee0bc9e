"""Write large_m900_oracle.json: double-double oracle Hafnians and probabilities
of all 80 patterns of the large workload (M = 900, r = 1, 64 at n = 28 and 16
at n = 30). Calls only the oracle and the seeded input generators.

    python tests/golden/make_large_golden.py [--out DIR]

The Haar draw comes from a LAPACK QR whose last bits differ between
platforms; the file records a SHA-256 of U's bytes, and must be written on
the platform whose GPU tests read it.

Takes tens of minutes on a few cores (the oracle is the plain subset sum with
repeated products in double-double arithmetic)."""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def main():
    U, r, pats = W.workload("large_m900")
    Bdd = oracle.build_B_dd(U, np.tanh(r))
    B = (Bdd[..., 0] + Bdd[..., 1]) + 1j * (Bdd[..., 2] + Bdd[..., 3])
    out = {"workload": "large_m900", "m": 900, "r": 1.0,
           "U_sha256": hashlib.sha256(np.ascontiguousarray(U, dtype=np.complex128).tobytes()).hexdigest(),
           "B_checksum": [float(np.abs(B).sum()), float(B.real.sum()), float(B.imag.sum())],
           "patterns": []}
    t0 = time.time()
    for i, x in enumerate(pats):
        res = oracle.prob(U, r, [x], Bdd=Bdd)
        hd = res["haf_dd"][0]
        out["patterns"].append({"i": i, "n": len(x), "x": [int(v) for v in x],
                                "haf_dd": [float(v) for v in hd], "p": float(res["p"][0]),
                                "logp": float(res["logp"][0]), "kappa": float(res["kappa"][0])})
        print("%d/%d n=%d %.0fs" % (i + 1, len(pats), len(x), time.time() - t0), flush=True)
    out_dir = os.path.abspath(sys.argv[2]) if sys.argv[1:2] == ["--out"] else HERE
    os.makedirs(out_dir, exist_ok=True)
    with open(os.path.join(out_dir, "large_m900_oracle.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
