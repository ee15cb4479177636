"""Tune tile shapes on this GPU for the classes the batched and served
workloads use, and write them to tuning_b300.txt beside this file, which the
package loads with the library (set RQA_NO_TUNING_TABLE to skip it).

Classes: RQA with FP32 distances, m = 2..8, each norm, and every
ceil(log2 n) bucket from 9 to 18 (series of 500 to 200,000 points).  Each
class is tuned on the library's built-in z-scored AR(1) series (rqa_autotune
with no series) of 3/4 of the bucket's top size, with tau = 2 and eps = 0.3
(the middle of the 0.05 .. 0.5 std range of those workloads); rqa_autotune
times every strip width at four and two columns per lane, and the band
height where the winner runs in row bands.

    python -m paper_2402_16853_b300.make_tuning_table [--out PATH] [--m 2-8]
"""
from __future__ import annotations

import argparse
import os
import time

from . import rqa as R


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=R.TUNING_TABLE)
    ap.add_argument("--mmin", type=int, default=2)
    ap.add_argument("--mmax", type=int, default=8)
    ap.add_argument("--bmin", type=int, default=9)
    ap.add_argument("--bmax", type=int, default=18)
    a = ap.parse_args()
    os.environ["RQA_NO_TUNING_TABLE"] = "1"   # start from the size rule
    R.load()
    R.autotune_clear()
    t0 = time.time()
    rows = []
    for m in range(a.mmin, a.mmax + 1):
        for norm in (0, 1, 2):
            for b in range(a.bmin, a.bmax + 1):
                n = (3 << b) // 4
                tau = 2
                st = R.Settings(m=m, tau=tau, eps=0.3, norm=norm, theiler=1)
                t = R.autotune_shape(st, n_points=n + (m - 1) * tau)
                rows.append((m, norm, b, t))
                print(f"m={m} norm={norm} log2n={b}: warps {t['warps']} cols {t['cols']} "
                      f"band {t['band_scale']:+d}  {t['ms']:.3f} ms", flush=True)
    R.save_tuning_table(a.out)
    print(f"{len(rows)} classes in {time.time() - t0:.0f} s -> {a.out}")


if __name__ == "__main__":
    main()
