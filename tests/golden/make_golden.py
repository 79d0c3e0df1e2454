"""Writes tests/golden/oracle_er64.json from the oracle alone.

The paper prints no worked example with values (its example graph and the
execution trace of an RR set are figures), so the stored values here come
from the oracle: a directed Erdos-Renyi graph with n = 64, m = 256 (seed 9),
weighted-cascade weights 1/indeg(v) in fp32 (Sec. IV-B), Philox seed 5.
For IC and LT: RR sets 0..99 as sorted vertex lists (the RR-set definition
of Sec. II-E under each model), the greedy seeds, marginal gains and covered
count for k = 5 over those 100 sets (Alg. 1's maximum-coverage step), and
IMM (Alg. 2 then Alg. 1) with k = 3, eps = 0.5, l = 1.

Run from the repository root: python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2009_07325_gb300 import inputs as I  # noqa: E402

SEED = 5


def main():
    O.build()
    I.build()
    g = I.wc_weights(I.er(64, 256, 9))
    out = {"graph": "directed Erdos-Renyi n=64 m=256 seed 9, weighted cascade 1/indeg(v) fp32",
           "philox_seed": SEED, "models": {}}
    for name, model in (("IC", O.IC), ("LT", O.LT)):
        o = O.Oracle(g)
        o.sample(model, SEED, 100, 1)
        off, mem = o.export()
        sets = [sorted(mem[off[j]:off[j + 1]].tolist()) for j in range(100)]
        seeds, gains, cov = o.greedy(5)
        imm = O.Oracle(g).imm(model, 3, 0.5, 1.0, SEED)
        out["models"][name] = {
            "rr_sets": sets,
            "greedy_k5": {"seeds": seeds.tolist(), "gains": gains.tolist(), "covered": cov},
            "imm_k3_eps05": {"seeds": imm["seeds"].tolist(), "theta": imm["theta"], "lb": imm["lb"],
                             "rr_count": imm["rr_count"]},
        }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_er64.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(path)


if __name__ == "__main__":
    main()
