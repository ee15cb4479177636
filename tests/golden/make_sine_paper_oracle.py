"""Write tests/golden/sine_paper_oracle.json: the FP64 oracle's complete
result for the paper's runtime workload (Sect. 8.2): sin over 1,000,001
evenly spaced points of [0, 1000 pi], m = 2, tau = 2, L2, eps = 1.0, no
Theiler window, minimum lines 2 -- n = 999,999 vectors, about 1.0e12 cells,
computed in the oracle's streaming mode on all host cores (about half an
hour on 8 cores).

The three histograms (1,000,000 entries each) are stored as SHA-256 digests
of their little-endian uint64 bytes, their totals and weighted totals, the
longest length present and the non-zero entries up to length 64; the
measures are stored in full.  Only oracle/ and the input recipe are used.

    python tests/golden/make_sine_paper_oracle.py [out.json]
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
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(HERE, "sine_paper_oracle.json")
    s, p = synth.workload("sine_paper")
    t0 = time.time()
    r = oracle.rqa(s, oracle.Settings(**p), mode="streaming")
    sec = time.time() - t0
    rec = {
        "workload": "sine_paper", "N": len(s), "params": p, "n_vec": r["n"], "rp": r["rp"],
        "oracle_seconds": sec, "oracle_threads": os.cpu_count(),
        "measures": r["measures"],
    }
    for k in ("hd", "hv", "hw"):
        h = r[k]
        nz = np.nonzero(h)[0]
        rec[k] = {"sha256": digest(h), "sum": int(h.sum()),
                  "weighted_sum": int((np.arange(len(h), dtype=np.uint64) * h).sum()),
                  "max_len": int(nz.max()) if len(nz) else 0,
                  "nonzero_bins": int(len(nz)),
                  "head": {str(l): int(h[l]) for l in range(1, 65) if h[l]}}
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    print(out, sec)


if __name__ == "__main__":
    main()
