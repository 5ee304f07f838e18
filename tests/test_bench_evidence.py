"""The benchmark's evidence plumbing, on the host: the slice kernel's source
list names real files, and the committed DRAM summary of the slice kernel
parses into every field the benchmark reads (it quotes the traffic only while
the sources still hash as recorded)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_slice_sources_exist():
    for f in bench.SLICE_SOURCES:
        assert os.path.exists(os.path.join(ROOT, "paper_1307_2982_gb300", "csrc", f)), f
    assert len(bench.source_sha256()) == 64


def test_dram_summary_fields():
    path = os.path.join(ROOT, "profiles", "search_stream_1Bx128_k100_dram.txt")
    kv = {}
    with open(path) as fh:
        for line in fh:
            if "=" in line and not line.startswith(" "):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
    for key in ("source_sha256", "n", "q", "m", "codes", "dram_bytes_per_launch"):
        assert key in kv, key
    assert len(kv["source_sha256"]) == 64
    assert float(kv["dram_bytes_per_launch"]) > 0
    # the traffic is quoted for exactly the workload the summary names
    got = bench.slice_traffic({}, 1, {}, 1, int(kv["q"]), kv["codes"], int(kv["n"]), int(kv["m"]))
    if kv["source_sha256"] == bench.source_sha256():
        assert got[0] == float(kv["dram_bytes_per_launch"])
    else:
        assert got == (None, None)
    assert bench.slice_traffic({}, 1, {}, 1, int(kv["q"]), kv["codes"], int(kv["n"]) + 1, int(kv["m"])) == (None, None)


def test_reference_arm_prints_its_line():
    """`bench.py --impl reference` (the oracle timed on the host) prints one
    JSON line with the contract's keys, on a small database."""
    import json
    import subprocess

    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "20000",
                          "--steps", "1", "--warmup", "3", "--cpu-sample", "4"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "queries/s" and line["value"] > 0
    for key in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config"):
        assert key in line, key
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
