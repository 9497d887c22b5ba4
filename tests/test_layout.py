"""Structure of the product path, checked on the CPU: the package and its
CUDA sources never reach the oracle, and the benchmark's traffic lookup
refuses a capture whose kernel sources changed."""
import hashlib
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1501_05810_gb300")


def _files(top, exts):
    for d, _, fs in os.walk(top):
        if "__pycache__" in d or "_build" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_never_imports_the_oracle():
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)|nbgs_oracle|liboracle", re.M)
    hits = [p for p in _files(PKG, (".py", ".cu", ".cuh", ".h", ".cpp")) if pat.search(open(p).read())]
    hits += [p for p in _files(os.path.join(ROOT, "include"), (".h",)) if pat.search(open(p).read())]
    assert not hits, hits


def test_oracle_never_includes_the_library():
    pat = re.compile(r"^\s*(from\s+paper_1501_05810_gb300|import\s+paper_1501_05810_gb300)|"
                     r"#\s*include\s*[<\"][^>\"]*(nbgs_internal|nbgs\.h)|libnbgs", re.M)
    hits = [p for p in _files(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")) if pat.search(open(p).read())]
    assert not hits, hits


def test_nothing_committed_reaches_scratch():
    pat = re.compile(r"(?<![\w])_work(/|['\"])")
    tops = [PKG, os.path.join(ROOT, "oracle"), os.path.join(ROOT, "include"), os.path.join(ROOT, "tests")]
    hits = [p for t in tops for p in _files(t, (".py", ".cu", ".cuh", ".h", ".c"))
            if p != os.path.abspath(__file__) and pat.search(open(p).read())]
    for f in ("bench.py", "__graft_entry__.py"):
        if pat.search(open(os.path.join(ROOT, f)).read()):
            hits.append(f)
    assert not hits, hits


def test_traffic_lookup_follows_the_kernel_sources(tmp_path, monkeypatch):
    import bench
    entry = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for key, d in entry.items():
        assert abs(d["dram_bytes_per_update"] * d["contact_updates_per_launch"] - d["dram_bytes_per_launch"]) \
            <= 1e-6 * d["dram_bytes_per_launch"], key
    d = entry["k_solve_persistent<float> dense1m"]
    h = hashlib.sha256(b"".join(open(os.path.join(PKG, "csrc", f), "rb").read()
                                for f in ("solve.cu", "nbgs_internal.cuh"))).hexdigest()[:16]
    got = bench.measured_traffic("fp32", 1000, 10, workload="dense1m")
    if h == d["source_sha256_16"]:
        assert abs(got - d["dram_bytes_per_update"] * 1000 * 10) <= 1e-9 * got
    else:
        assert got is None          # a capture of other sources is not reported
    assert bench.measured_traffic("fp64", 1000, 10, workload="dense1m") is None   # no FP64 capture
    assert bench.measured_traffic("fp32", 1000, 10, workload="no such workload") is None
    # a changed source invalidates the capture
    fake = tmp_path / "repo"
    (fake / "profiles").mkdir(parents=True)
    (fake / "paper_1501_05810_gb300" / "csrc").mkdir(parents=True)
    json.dump(entry, open(fake / "profiles" / "traffic.json", "w"))
    for f in ("solve.cu", "nbgs_internal.cuh"):
        data = open(os.path.join(PKG, "csrc", f), "rb").read()
        open(fake / "paper_1501_05810_gb300" / "csrc" / f, "wb").write(data + (b"\n" if f == "solve.cu" else b""))
    monkeypatch.setattr(bench, "ROOT", str(fake))
    assert bench.measured_traffic("fp32", 1000, 10, workload="dense1m") is None
