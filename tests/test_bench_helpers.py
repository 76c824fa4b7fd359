"""Host-side helpers of bench.py: the algorithmic-bytes model, the committed
DRAM-capture record, and the parallel oracle baseline (spawned workers over
graphs in shared memory must compute what the oracle computes in-process)."""
import numpy as np
import pytest

import bench
import oracle
from paper_2105_06145_gb300 import graphgen as gg


def test_algorithmic_bytes_per_unit():
    # per queued vertex per step 16 B, per extracted vertex 32 B, per scanned
    # edge 16 B, per successful update 8 B
    assert bench.algorithmic_bytes({"queued": 1, "extracted": 0, "edges": 0, "updates": 0}) == 16
    assert bench.algorithmic_bytes({"queued": 0, "extracted": 1, "edges": 0, "updates": 0}) == 32
    assert bench.algorithmic_bytes({"queued": 0, "extracted": 0, "edges": 1, "updates": 0}) == 16
    assert bench.algorithmic_bytes({"queued": 0, "extracted": 0, "edges": 0, "updates": 1}) == 8


def test_captured_traffic_record_matches_kernel_hash_or_is_absent():
    cap = bench.captured_traffic()
    if cap is not None:
        nbytes, edges = cap
        # one RMAT scale-22 launch scans 1-4.5 m edges and moves 8-16 B of DRAM per edge
        assert 1 * 128e6 < edges < 4.5 * 128e6
        assert 8 * edges < nbytes < 16 * edges


def test_oracle_parallel_equals_in_process_oracle():
    g1 = gg.rmat(12, 8, gen_seed=1, wseed=2)
    g2 = gg.grid(40, 40, wseed=3)
    g3 = gg.road(30, 0.75, seed=4)
    tasks = [(g1, s) for s in gg.pick_sources(g1, 5, 6)] + [(g2, 0), (g2, 799), (g3, 17)]
    r = bench.oracle_parallel(tasks, with_digests=True)
    want = [int(np.bitwise_xor.reduce(oracle.dijkstra(h, s))) for h, s in tasks]
    assert r["digests"] == want
    assert r["cores"] >= 1 and r["value"] > 0 and r["kind"] == "oracle"


def test_reference_arm_prints_one_json_line():
    """`bench.py --impl reference` (the oracle on host cores) runs without a GPU
    and prints the contract's line: impl, metric, value, cpu_baseline, e2e."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.check_output([sys.executable, "bench.py", "--impl", "reference", "--scale", "12",
                                   "--steps", "2", "--warmup", "1"], cwd=root, text=True, timeout=600)
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GTEPS" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
