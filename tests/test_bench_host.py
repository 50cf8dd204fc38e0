"""bench.py's host side on CPU: the reference arm's JSON line, the recorded-traffic
lookup and its source hash, the FLOP model."""
import importlib.util
import json

import numpy as np
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "small",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["config"]["workload"].startswith("df-20atom")


def test_flop_model():
    b = _bench()
    w = b.workload("large")
    assert b.flops_K(w) == 4.0 * 1200 ** 2 * 3600 * 250


def test_recorded_traffic_is_tied_to_the_sources():
    b = _bench()
    sha = b.kernel_source_sha()
    assert len(sha) == 64
    recs = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.txt")))
    first = [r for r in recs if r["kernel"] == "slice_gemm (X = B C)"][0]
    got = b.recorded_traffic("slice_gemm (X = B C)", first["workload"], first["nslices"], first["cluster_pairs"])
    if first["source_sha256"] == sha:
        assert got == first["dram_bytes_per_launch"]
    else:
        assert got is None                          # stale record: reported as null, never reused
    assert b.recorded_traffic("slice_gemm (X = B C)", first["workload"], first["nslices"] + 1, 1) is None


def test_oracle_gate_on_the_small_molecule():
    """The bench's accuracy gate: the oracle's per-block K and J sum to the whole-molecule
    build, an exact K passes, and a K off by 2e-10 max|K| fails."""
    b = _bench()
    sys.path.insert(0, ROOT)
    from oracle import df_oracle as O
    from paper_2601_08077_gb300 import inputs
    w = inputs.SMALL
    mol, B, C, D = inputs.make_inputs(w)
    base, K, J, rho = b.oracle_reference(B, C, D, w)
    assert base["kind"] == "oracle" and base["value"] > 0 and "all 3 auxiliary blocks" in base["sample"]
    K_full = O.exchange(B, C)
    J_full = O.coulomb(B, O.rho(B, D))
    assert np.max(np.abs(K - K_full)) <= 1e-13 * np.max(np.abs(K_full))
    assert np.max(np.abs(J - J_full)) <= 1e-13 * np.max(np.abs(J_full))
    EJ, EK = O.energies(D, J, K)
    g = b.oracle_gate(K_full, J_full, (EJ, 0.0, EK), K, J, D)
    assert g["gate_vs_oracle"] and g["dE_vs_oracle"] < 1e-10
    Kbad = K_full.copy()
    Kbad[3, 5] += 2e-10 * np.max(np.abs(K_full))
    assert not b.oracle_gate(Kbad, J_full, (EJ, 0.0, EK), K, J, D)["gate_vs_oracle"]
