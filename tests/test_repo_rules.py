"""Static checks of the product sources (no GPU): the product never reaches the
oracle, and bench.py's traffic and peak helpers behave as documented."""
import ast
import hashlib
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1712_02533_gb300")


def _py_files(d):
    for base, _, files in os.walk(d):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def test_product_never_imports_the_oracle():
    for path in _py_files(PKG):
        tree = ast.parse(open(path).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""]
            else:
                continue
            assert not any(n == "oracle" or n.startswith("oracle.") for n in names), (path, names)


def test_cuda_sources_include_nothing_from_the_oracle():
    for base, _, files in os.walk(os.path.join(PKG, "csrc")):
        for f in files:
            src = open(os.path.join(base, f)).read()
            assert "oracle" not in src.lower() or f.endswith(".md"), f


def test_traffic_is_reported_only_for_the_captured_kernel_source():
    import bench
    src = os.path.join(PKG, "csrc", "kernels.cu")
    sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
    if sha == bench.TRAFFIC_CAPTURE["kernels_cu_sha1"]:
        assert bench._traffic("trial", 1000.0) == round(bench.TRAFFIC_CAPTURE["trial"] * 1000.0)
    else:
        assert bench._traffic("trial", 1000.0) is None
    assert bench._traffic("prolong", 1000.0) is None


def test_peaks_come_from_the_measured_file_or_the_stated_fallback(tmp_path, monkeypatch):
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 1234.5}))
    assert bench._peaks() == (1234.5, "measured")
