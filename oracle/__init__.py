"""FP64 CPU oracle for the linear Fisher / Arrow-Debreu market equilibrium.

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the CUDA
solver: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and its ``--impl reference`` arm) may import it.  The
product path (the C-ABI library and its Python binding) never imports, links or
executes anything here, and this package never imports the product path.  The
two share no code; only the seeded input generator
(``paper_2506_06258_gb300.synth``, which holds none of the method's arithmetic)
serves both.

Everything is plain numpy in float64, written from the paper (Liu, Huang, Li,
Ge, Ye, "PDHCG: A Scalable First-Order Method for Large-Scale Competitive
Market Equilibrium Computation"):

* ``fisher``   -- the Eisenberg-Gale program, Alg. 2 (restarted PDHCG) with the
                  Section 5 enhancements, the exact row subproblem, Alg. 3 and the
                  32-section search, and the relative KKT error of Section 5.
* ``closed``   -- closed-form equilibria (n=1, m=1, rank-one, 2x2) and a
                  brute-force basic-solution enumeration for tiny markets.
* ``certify``  -- the equilibrium certificate (market clearing, budgets,
                  sum p = sum w, bang-per-buck, complementarity).
* ``prd``      -- proportional-response dynamics, an independent published
                  method used only to cross-check the PDHCG oracle.
* ``arrow``    -- Alg. 4 (fixed-point iteration for Arrow-Debreu).
* ``adjoint``  -- implicit derivatives of equilibrium prices/utilities.

Parity status: the converged equilibrium (prices and utilities, unique by
Fact 1) is pinned by closed forms, brute force and proportional response; the
PDHCG iterate *trajectory* is "parity unpinned" (the paper prints no worked
example), so only converged results and single-step operators are compared.
"""
