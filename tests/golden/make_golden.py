"""Write the stored C1 equilibrium (tests/golden/c1_equilibrium.txt).

The paper prints no worked example, so the stored values come from the FP64
oracle: the C1 market (n = 200 buyers, m = 100 goods, each pair kept with
probability 0.2, u ~ U(0,1), w ~ U(0.5,1.5), seeded), solved by the oracle's
PDHCG (Alg. 2) to relative KKT 1e-12.  Prices and utilities of a linear Fisher
market are unique (Fact 1), so they are the reference any solver must reach;
the allocation x is one equilibrium allocation (x is not unique), stored so
that the equilibrium conditions can be checked on the stored point itself.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import certify, fisher as F  # noqa: E402
from paper_2506_06258_gb300 import synth as S  # noqa: E402

OUT = os.path.join(HERE, "c1_equilibrium.txt")


def main():
    mk = S.config1()
    r = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-12, max_iter=2_000_000))
    if not r.converged:
        raise SystemExit("oracle did not reach KKT 1e-12")
    cert = certify.certificate(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, r.x, r.p)
    with open(OUT, "w") as f:
        f.write("# C1 Fisher market equilibrium, FP64 oracle PDHCG (Alg. 2) to relative KKT 1e-12\n")
        f.write("# market: synth.config1() (n=200, m=100, q=0.2, u~U(0,1), w~U(0.5,1.5), seeded)\n")
        f.write("# written by tests/golden/make_golden.py; p and t are unique (Fact 1), x is one equilibrium allocation\n")
        f.write(f"# n {mk.n} m {mk.m} nnz {mk.nnz} kkt {r.kkt.kkt:.3e} iters {r.iters}\n")
        f.write("# certificate " + " ".join(f"{k} {v:.3e}" for k, v in sorted(cert.items()) if k != "t") + "\n")
        for name, arr in (("p", r.p), ("t", r.t), ("x", r.x)):
            f.write(f"{name} {len(arr)}\n")
            for v in arr:
                f.write(f"{v:.17g}\n")
    print(f"wrote {OUT}: kkt {r.kkt.kkt:.3e}")


if __name__ == "__main__":
    main()
