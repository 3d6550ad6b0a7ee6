"""The reference arm of bench.py (the oracle on the host cores) keeps the one-line JSON contract,
and under several ranks only rank 0 works and prints (CPU only)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                          env=env, timeout=600, cwd=ROOT)


def test_reference_arm_prints_one_json_line():
    out = _run({})
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["higher_is_better"] is True
    assert d["unit"] == "device evals+stamps/s" and d["value"] > 0
    assert d["steps"] == 1 and d["ms_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "277778" in d["config"]["workload"]   # the ~1M-FET random logic, as the GPU arm


def test_reference_arm_other_ranks_exit_without_work():
    out = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_bench_parity_record_on_the_oracle_itself():
    # the bench's full-size parity record, fed the oracle's own step: zero error; one entry
    # moved by 1e-9 of its size: the cancellation-aware error sees it and the record fails
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import netgen
    import oracle
    net = netgen.random_logic(300, seed=3)
    x = netgen.random_x(net)
    o = oracle.Oracle(net, netgen.default_cards())
    r = o.eval_stamp(x, want_q=True)
    rec = bench.parity_vs_oracle(o, x, r["A"].copy(), r["b"].copy(), r["q"].reshape(-1).copy())
    assert rec["pass"] and rec["A"]["max_err"] == 0 and rec["b"]["max_plain"] == 0
    assert rec["q"]["max_err"] == 0 and rec["A"]["entries"] == r["A"].size
    A = r["A"].copy()
    k = int(np.argmax(np.abs(A)))
    A[k] *= 1 + 1e-9
    bad = bench.parity_vs_oracle(o, x, A, r["b"].copy(), r["q"].reshape(-1).copy())
    assert not bad["pass"] and 1e-10 < bad["A"]["max_err"] <= 1e-9 * (1 + 1e-6)
    assert abs(bad["A"]["max_plain"] - 1e-9) < 1e-12
