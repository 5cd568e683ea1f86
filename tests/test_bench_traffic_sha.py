"""bench.py ties a recorded ncu traffic figure to one kernel's source text: the
hash covers that kernel from its __global__ line to its closing brace, so it
changes with the kernel and not with the rest of the file (CPU only)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = """// two kernels
template <int CP>
__global__ void __launch_bounds__(256, 4) k_a(Args a) {
    if (a.x) { a.y = 1; }
}

__global__ void k_b(Args a) { a.z = 2; }
"""


def _sha(tmp_path, monkeypatch, text, kernel):
    d = tmp_path / "paper_2408_10982_gb300" / "csrc"
    d.mkdir(parents=True, exist_ok=True)
    (d / "x.cu").write_text(text)
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return bench.kernel_sha("x.cu", kernel)


def test_kernel_sha_follows_only_its_kernel(tmp_path, monkeypatch):
    a0 = _sha(tmp_path, monkeypatch, SRC, "k_a")
    b0 = _sha(tmp_path, monkeypatch, SRC, "k_b")
    assert a0 != b0 and len(a0) == 16
    other = SRC.replace("a.z = 2", "a.z = 3")            # k_b's body changes
    assert _sha(tmp_path, monkeypatch, other, "k_a") == a0
    assert _sha(tmp_path, monkeypatch, other, "k_b") != b0
    mine = SRC.replace("a.y = 1", "a.y = 4")             # k_a's nested body changes
    assert _sha(tmp_path, monkeypatch, mine, "k_a") != a0
    bounds = SRC.replace("(256, 4)", "(256, 5)")         # so do its launch bounds
    assert _sha(tmp_path, monkeypatch, bounds, "k_a") != a0
    comment = "// a comment above\n" + SRC               # text outside it does not count
    assert _sha(tmp_path, monkeypatch, comment, "k_a") == a0


def test_recorded_traffic_names_a_kernel_of_the_source():
    sys.path.insert(0, ROOT)
    import bench
    for name, rec in bench.TRAFFIC.items():
        assert name == "sample_lt"
        assert len(rec["src_sha"]) == 16 and rec["bytes_per_launch"] > 0
        bench.kernel_sha("sample.cu", "k_sample_lt1")     # the kernel exists and parses
