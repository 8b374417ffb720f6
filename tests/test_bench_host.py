"""Host-side logic of bench.py (no GPU): the traffic figures read from the
committed ncu summaries and their source-hash check, the NUMA binding helper,
and the reference arm's JSON line on a small oracle sample."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_committed_profiles_match_their_sources():
    # every summary the bench reads names its kernel sources and their hash
    for name in ("scan_dense_ppvbs_sweep", "lookup_ppvbs_k2_sweep", "fused_ppvbs_k2_sweep"):
        path = os.path.join(ROOT, "profiles", name + ".md")
        fields = {}
        with open(path) as f:
            for line in f:
                if line.startswith("- ") and ":" in line:
                    k, v = line[2:].split(":", 1)
                    fields[k.strip()] = v.strip().strip("`")
        h = hashlib.sha256()
        for src in fields["sources"].split(","):
            with open(os.path.join(ROOT, src.strip()), "rb") as f:
                h.update(f.read())
        traffic = bench.profile_traffic(name)
        if h.hexdigest() == fields["sources_sha256"]:
            assert traffic == int(fields["traffic_bytes_full_launch"])
        else:
            assert traffic is None


def test_profile_traffic_rejects_stale_and_missing(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    digest = hashlib.sha256(b"kernel v1\n").hexdigest()
    (prof / "k.md").write_text("- sources: k.cu\n- sources_sha256: `%s`\n- traffic_bytes_full_launch: 1234\n" % digest)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("k") == 1234
    src.write_text("kernel v2\n")  # the kernel changed after the capture
    assert bench.profile_traffic("k") is None
    assert bench.profile_traffic("absent") is None


def test_cpulist_parsing():
    assert bench._cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench._cpulist("5") == {5}
    assert bench._cpulist("") == set()


def test_bind_near_gpu_leaves_affinity_alone_without_a_gpu(monkeypatch):
    before = os.sched_getaffinity(0)

    def no_smi(*a, **k):
        raise FileNotFoundError("nvidia-smi")

    monkeypatch.setattr(subprocess, "run", no_smi)
    assert bench.bind_near_gpu(0) is None
    assert os.sched_getaffinity(0) == before


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--ref-rows", str(1 << 16)],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "Grows/s" and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_oracle_sample_on_several_threads_agrees():
    # the all-core oracle timing splits rows into ranges run by the oracle's
    # own sequential code; the values found equal one sequential pass
    values, lit = bench.make_column(1 << 18, 0)
    rows = 200_003
    _, m1, _, t1 = bench.oracle_sample(values, lit, rows, 1)
    _, m4, _, t4 = bench.oracle_sample(values, lit, rows, 4)
    assert t1 == 1 and t4 == 4
    assert m1 == m4 == int((values[:rows] < lit).sum())
