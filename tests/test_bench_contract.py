"""The reference arm of bench.py (the FP64 oracle on the host cores) prints one
JSON line with the keys the benchmark contract asks for, on rank 0 only."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)

    class A:
        steps, warmup, gpus = 1, 0, 1
    assert bench.run_reference(A()) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["metric"] == bench.METRIC and d["config"]["workload"] == bench.WORKLOAD["name"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_traffic_record_is_gated(monkeypatch):
    """The roofline's DRAM traffic comes from the committed ncu record only while
    the walk source and the leaf population are those of the capture; it is the
    block's launch mix (one full walk, k - 1 electron walks)."""
    sys.path.insert(0, ROOT)
    import hashlib
    import bench
    rec = {}
    for line in open(os.path.join(ROOT, "profiles", "walk_fp32c_traffic.txt")):
        if ":" in line:
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
    src = os.path.join(ROOT, "paper_0709_3331_gb300", "csrc", "ucp_walk.cu")
    same = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == rec["walk_source_sha256_16"]
    got = bench.traffic_record()
    if same and rec.get("leaf_cap") == str(bench.WORKLOAD["leaf_cap"]):
        k = bench.WORKLOAD["k"]
        want = (float(rec["dram_bytes_per_full_walk"]) +
                (k - 1) * float(rec["dram_bytes_per_electron_walk"])) / k
        assert got == want
    else:
        assert got is None
    monkeypatch.setitem(bench.WORKLOAD, "leaf_cap", bench.WORKLOAD["leaf_cap"] + 1)
    assert bench.traffic_record() is None
