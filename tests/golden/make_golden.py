"""Write the stored equilibria under tests/golden/.

c1_equilibrium.txt  (python tests/golden/make_golden.py)

The paper prints no worked example, so the stored values come from the FP64
oracle: the C1 market (n = 200 buyers, m = 100 goods, each pair kept with
probability 0.2, u ~ U(0,1), w ~ U(0.5,1.5), seeded), solved by the oracle's
PDHCG (Alg. 2) to relative KKT 1e-12.  Prices and utilities of a linear Fisher
market are unique (Fact 1), so they are the reference any solver must reach;
the allocation x is one equilibrium allocation (x is not unique), stored so
that the equilibrium conditions can be checked on the stored point itself.

c3law_equilibrium.txt  (python tests/golden/make_golden.py c3law)
The skewed law of the nnz = 1e9 benchmark market (Zipf(2) buyer degrees on
[10, 2000] rescaled, popularity rank^-1.1, LogNormal(0,1) utilities,
w ~ U(0.5,1.5)) at n = 10000 buyers, m = 1000 goods, nnz ~ 1e6 (1/1000 of the
benchmark), with the FP32 utilities the GPU's MIXED path reads (widened exactly
to FP64), solved by the oracle's PDHCG to relative KKT 1e-9.  Only p and t are
stored (unique, Fact 1).

Run from the repository root.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import certify, fisher as F  # noqa: E402
from paper_2506_06258_gb300 import synth as S  # noqa: E402

OUT = os.path.join(HERE, "c1_equilibrium.txt")


C3LAW = dict(n=10_000, m=1_000, nnz_target=1_000_000)
OUT_C3LAW = os.path.join(HERE, "c3law_equilibrium.txt")


def c3law_market():
    return S.config3(fp32=True, **C3LAW)


def main_c3law():
    mk = c3law_market()
    val = mk.val.astype(np.float64)
    r = F.pdhcg_solve(mk.row_ptr, mk.col, val, mk.w, mk.m, F.Params(tol=1e-9, max_iter=5_000_000))
    if not r.converged:
        raise SystemExit("oracle did not reach KKT 1e-9")
    cert = certify.certificate(mk.row_ptr, mk.col, val, mk.w, mk.m, r.x, r.p)
    with open(OUT_C3LAW, "w") as f:
        f.write("# skewed benchmark law at n=10000, m=1000, nnz~1e6: FP64 oracle PDHCG (Alg. 2) to relative KKT 1e-9\n")
        f.write(f"# market: synth.config3(n={C3LAW['n']}, m={C3LAW['m']}, nnz_target={C3LAW['nnz_target']}, fp32=True)"
                " (FP32 utilities widened to FP64)\n")
        f.write("# written by tests/golden/make_golden.py c3law; p and t are unique (Fact 1)\n")
        f.write(f"# n {mk.n} m {mk.m} nnz {mk.nnz} kkt {r.kkt.kkt:.3e} iters {r.iters}\n")
        f.write("# certificate " + " ".join(f"{k} {v:.3e}" for k, v in sorted(cert.items()) if k != "t") + "\n")
        for name, arr in (("p", r.p), ("t", r.t)):
            f.write(f"{name} {len(arr)}\n")
            for v in arr:
                f.write(f"{v:.17g}\n")
    print(f"wrote {OUT_C3LAW}: kkt {r.kkt.kkt:.3e} iters {r.iters}")


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
    main_c3law() if sys.argv[1:] == ["c3law"] else main()
