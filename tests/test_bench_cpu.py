"""bench.py's reference arm (the FP64 oracle on the host cores) runs without a
GPU and prints one JSON line with the keys the bench contract requires."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_a_complete_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_all_core_oracle_harness_matches_one_process():
    """The all-core CPU baseline splits the buyers into row blocks, one spawned
    process each; after a few iterations its prices and column sums equal those
    of the oracle run in one process (the row subproblems are independent
    given the prices, so only the summation order of the column sums differs)."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from paper_2506_06258_gb300 import synth as S
    mk = S.config3(n=2000, m=300, nnz_target=60_000, fp32=False)
    one, two = bench.OracleIterations(mk, 1), bench.OracleIterations(mk, 3)
    try:
        for _ in range(4):
            one.step()
            two.step()
        assert np.allclose(one.p, two.p, rtol=1e-12, atol=1e-14)
        assert np.allclose(one.c, two.c, rtol=1e-12, atol=1e-14)
    finally:
        one.close()
        two.close()


def test_bench_names_resolve_and_stored_equilibrium_reads():
    """Every module-level name bench.py's GPU path calls exists (the GPU path
    cannot run here), and the stored oracle equilibrium it compares with reads."""
    import ast
    sys.path.insert(0, ROOT)
    import bench
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    defined = {n.name for n in tree.body if isinstance(n, (ast.FunctionDef, ast.ClassDef))}
    called = {n.func.id for n in ast.walk(tree) if isinstance(n, ast.Call) and isinstance(n.func, ast.Name)
              and n.func.id.startswith("_")}
    assert called <= defined, called - defined
    g = bench._stored_equilibrium("c3law_equilibrium.txt")
    assert len(g["p"]) == 1000 and len(g["t"]) == 10000
