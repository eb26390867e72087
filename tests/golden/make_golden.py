"""Write the stored expected values under tests/golden/ from the oracle only.

The paper prints no worked example (no numeric output of any pass), so every
stored value here is the oracle's: a fixed snapshot that later changes to the
oracle are checked against, and that the CUDA library is compared with.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import py_oracle as orc  # noqa: E402

# Small correctness workload: n=4, N=256, seed 1, every returnable value of
# each pass returned (frac=1), mu=0, sigma=1, 1000 passes.
CASES = [
    dict(name="n4_N256_seed1_frac1", n=4, N=256, seed=1, frac=1.0, passes=[1, 2, 10, 100, 1000]),
    dict(name="n8_N128_seed3_frac05", n=8, N=128, seed=3, frac=0.5, passes=[1, 5, 50]),
    dict(name="n4_N1000_seed9_frac033", n=4, N=1000, seed=9, frac=1 / 3, passes=[1, 7, 40]),
]


def snapshot(case):
    g = orc.Generator(case["n"], case["N"], case["seed"], case["frac"])
    rows = []
    st = g.stats()
    rows.append(dict(passes=0, Q=str(st.Q), c32=int(np.float32(st.c32).view(np.uint32)),
                     pool_head=[int(v) for v in g.pool32()[:16].view(np.uint32)],
                     pool_last=int(g.pool32()[-1:].view(np.uint32)[0])))
    done = 0
    for p in case["passes"]:
        while done < p:
            g.pass_()
            done += 1
        st = g.stats()
        pool = g.pool32()
        rows.append(dict(passes=p, Q=str(st.Q), c32=int(np.float32(st.c32).view(np.uint32)),
                         alpha=[int(a) for a in st.alpha[:case["n"]]],
                         gamma=[int(x) for x in st.gamma[:case["n"]]],
                         pool_head=[int(v) for v in pool[:16].view(np.uint32)],
                         pool_last=int(pool[-1:].view(np.uint32)[0]),
                         pool_sum_bits=int(np.float64(pool.astype(np.float64).sum()).view(np.uint64)),
                         status=int(st.status)))
    return rows


def main():
    for case in CASES:
        data = dict(case=case, source="oracle/wallace_oracle.c via tests/golden/make_golden.py",
                    snapshots=snapshot(case))
        with open(os.path.join(HERE, case["name"] + ".json"), "w") as f:
            json.dump(data, f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main()
