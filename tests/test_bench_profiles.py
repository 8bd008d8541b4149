"""The bench's link to the committed ncu summaries: a figure is used only
while the hash of the kernel code (comments and whitespace removed) matches
the one recorded with the capture (host only)."""
import bench


def test_code_only_drops_comments_and_whitespace():
    src = "int a = 1;  // one\n/* block\n comment */\n\nint b = 2;\n   // only a comment\n"
    assert bench._code_only(src) == "inta=1;intb=2;"


def test_profiled_follows_the_code_hash(tmp_path, monkeypatch):
    (tmp_path / "k.cuh").write_text("// header\n__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_hash(["k.cuh"])
    (tmp_path / "profiles" / "k_step_w.md").write_text(
        f"kernel_sources_sha256_16: {h}\ntraffic_bytes_per_launch: 123.5\n")
    assert bench.profiled("w", "traffic_bytes_per_launch", sources=["k.cuh"]) == 123.5
    # a comment or layout edit keeps the capture valid
    (tmp_path / "k.cuh").write_text("// a new header\n__global__ void\n    k() {}  // same code\n")
    assert bench.profiled("w", "traffic_bytes_per_launch", sources=["k.cuh"]) == 123.5
    # a code change does not
    (tmp_path / "k.cuh").write_text("__global__ void k() { return; }\n")
    assert bench.profiled("w", "traffic_bytes_per_launch", sources=["k.cuh"]) is None
    assert bench.profiled("missing", "traffic_bytes_per_launch", sources=["k.cuh"]) is None
