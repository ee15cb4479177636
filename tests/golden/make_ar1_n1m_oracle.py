"""Write tests/golden/ar1_n1m_oracle.json: the FP64 oracle's complete result
for the 1,048,576-point AR(1) workload (phi = 0.95, seed 1003, z-scored;
m = 3, tau = 1, L2, eps = 0.5, Theiler 1, minimum lines 2), computed in the
oracle's streaming mode on all host cores (about 15 minutes on 16 cores).

The three histograms (1,048,575 entries each) are stored as SHA-256 digests
of their little-endian uint64 bytes plus their non-zero entries up to length
64 and their totals; the measures are stored in full.  Only oracle/ and the
seeded input recipe are used.

    python tests/golden/make_ar1_n1m_oracle.py [out.json]
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def digest(h):
    return hashlib.sha256(np.ascontiguousarray(h, dtype="<u8").tobytes()).hexdigest()


def main():
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(HERE, "ar1_n1m_oracle.json")
    s, p = synth.workload("ar1_n1m")
    t0 = time.time()
    r = oracle.rqa(s, oracle.Settings(**p), mode="streaming")
    sec = time.time() - t0
    rec = {
        "workload": "ar1_n1m", "N": len(s), "params": p, "n_vec": r["n"], "rp": r["rp"],
        "oracle_seconds": sec, "oracle_threads": os.cpu_count(),
        "measures": r["measures"],
    }
    for k in ("hd", "hv", "hw"):
        h = r[k]
        rec[k] = {"sha256": digest(h), "sum": int(h.sum()),
                  "weighted_sum": int((np.arange(len(h), dtype=np.uint64) * h).sum()),
                  "max_len": int(np.nonzero(h)[0].max()) if h.any() else 0,
                  "head": {str(l): int(h[l]) for l in range(1, 65) if h[l]}}
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    print(out, sec)


if __name__ == "__main__":
    main()
