"""Write double-double oracle values for the parity tests at full workload size.

    python tests/golden/make_golden.py [--out DIR] [name ...]

Calls only the oracle and the seeded input generators. Each file holds, per
pattern (or request), the oracle's Hafnian of B_x rounded to complex128, log p,
and the cancellation ratio kappa = sum_S |f(X A_S)| / |Haf| of the subset sum
taken the way the library takes it by default: positions t and t + n/2 form
pair t (the list x read in the order x[0], x[h], x[1], x[h+1], ...) and the
diagonal of B_x set to 0 (no perfect matching uses it, Eq. HafMatch; neither
choice changes Haf or p, only the individual subset terms).

Files (tests/golden/):
  batched_m64_n16_oracle.json   all 4096 patterns of the n = 16, M = 64 batch
  mixed_m144_oracle.json        all 2048 patterns of the mixed-n, M = 144 batch
  serving_m256_oracle.json      requests with even n >= 22 among the first 400
                                of the M = 256 serving stream
  large_m900_default_order.json patterns 0-3 (n = 28) and 64-65 (n = 30) of the
                                M = 900 batch: kappa in the default order

Each file records a SHA-256 of the Haar draw U's bytes: the draw comes from a
LAPACK QR, whose last bits differ between platforms, so the values must be
written on the platform whose GPU tests read them (the tests check the hash).

Takes about ten minutes on eight cores.
"""
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


def default_order(x):
    """x read so that consecutive positions (2t, 2t+1) are x[t], x[t + n/2]."""
    x = np.asarray(x, dtype=np.int32)
    h = len(x) // 2
    return np.array([x[(p >> 1) + (h if p & 1 else 0)] for p in range(len(x))], dtype=np.int32)


def table(U, r, pats, name, extra=None):
    Bdd = oracle.build_B_dd(U, np.tanh(r))
    B = (Bdd[..., 0] + Bdd[..., 1]) + 1j * (Bdd[..., 2] + Bdd[..., 3])
    t0 = time.time()
    ordered = [default_order(x) for x in pats]
    res = oracle.prob(U, r, ordered, Bdd=Bdd, zero_diag=True)
    haf = res["haf"]
    mod = np.abs(haf)
    kappa = np.where(mod > 0, res["kappa"] / np.where(mod > 0, mod, 1.0), 0.0)
    out = {"workload": name, "m": int(U.shape[0]),
           "U_sha256": u_hash(U),
           "B_checksum": [float(np.abs(B).sum()), float(B.real.sum()), float(B.imag.sum())],
           "order": "pair t = positions (t, t + n/2); zero diagonal",
           "x": [[int(v) for v in p] for p in pats],
           "haf_re": [float(v) for v in haf.real], "haf_im": [float(v) for v in haf.imag],
           "logp": [float(v) for v in res["logp"]], "kappa": [float(v) for v in kappa]}
    if extra:
        out.update(extra)
    print("%s: %d patterns, %.0f s" % (name, len(pats), time.time() - t0), flush=True)
    return out


def u_hash(U):
    """SHA-256 of the Haar draw's bytes (complex128, row-major)."""
    return hashlib.sha256(np.ascontiguousarray(U, dtype=np.complex128).tobytes()).hexdigest()


OUT = HERE


def write(fname, obj):
    os.makedirs(OUT, exist_ok=True)
    with open(os.path.join(OUT, fname), "w") as f:
        json.dump(obj, f, separators=(",", ":"))


def main(names):
    if not names or "batched_m64_n16" in names:
        U, r, pats = W.workload("batched_m64_n16")
        write("batched_m64_n16_oracle.json", table(U, r, pats, "batched_m64_n16"))
    if not names or "mixed_m144" in names:
        U, r, pats = W.workload("mixed_m144")
        write("mixed_m144_oracle.json", table(U, r, pats, "mixed_m144"))
    if not names or "serving_m256" in names:
        U, r, _ = W.workload("serving_m256")
        reqs = W.serving_requests(400)
        sel = [i for i, (_, x) in enumerate(reqs) if len(x) >= 22 and len(x) % 2 == 0]
        write("serving_m256_oracle.json",
              table(U, r, [reqs[i][1] for i in sel], "serving_m256", {"request_index": sel}))
    if not names or "large_m900" in names:
        U, r, pats = W.workload("large_m900")
        sel = [0, 1, 2, 3, 64, 65]
        write("large_m900_default_order.json",
              table(U, r, [pats[i] for i in sel], "large_m900", {"pattern_index": sel}))


if __name__ == "__main__":
    args = sys.argv[1:]
    if args[:1] == ["--out"]:
        OUT = os.path.abspath(args[1])
        args = args[2:]
    main(args)
