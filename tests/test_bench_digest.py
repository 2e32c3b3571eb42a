"""The bench's captured-traffic bookkeeping on the CPU: the DRAM traffic recorded from one ncu
capture of the dominant kernel is reported only while the code of the kernel's sources is the
code that was captured (comments and whitespace do not count)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _write(path, text):
    with open(path, "w", encoding="utf-8") as f:
        f.write(text)


def test_digest_ignores_comments_and_whitespace_but_not_code(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _write(tmp_path / "a.cu", "int f(int x) {\n    return x + 1;   // one\n}\n")
    d0 = bench.source_digest(("a.cu",))
    _write(tmp_path / "a.cu", "/* block\n comment */ int f(int x) { return x + 1; }  // other words\n")
    assert bench.source_digest(("a.cu",)) == d0
    _write(tmp_path / "a.cu", "int f(int x) { return x + 2; }\n")
    assert bench.source_digest(("a.cu",)) != d0


def test_captured_traffic_only_for_the_captured_kernel_and_code(monkeypatch):
    for (prec, kernel), (traffic, digest) in bench.CAPTURED_TRAFFIC.items():
        assert bench.captured_traffic("fp64" if prec == "fp32" else "fp32", kernel) is None
        assert bench.captured_traffic(prec, "fwd_last") is None
        monkeypatch.setattr(bench, "source_digest", lambda files=None, d=digest: d)
        assert bench.captured_traffic(prec, kernel) == traffic
        monkeypatch.setattr(bench, "source_digest", lambda files=None: "0" * 16)
        assert bench.captured_traffic(prec, kernel) is None

