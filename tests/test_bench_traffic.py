"""bench.py's DRAM-traffic figure for the roofline line comes from a committed
ncu capture and is tied to the kernel's source files by a hash: any change to
any of them makes the figure null until it is captured again."""
import bench


def test_source_hash_covers_every_file(tmp_path, monkeypatch):
    (tmp_path / "a.cu").write_text("kernel a")
    (tmp_path / "b.cuh").write_text("body b")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h1 = bench.kernel_source_hash(["a.cu", "b.cuh"])
    assert len(h1) == 16 and int(h1, 16) >= 0
    assert bench.kernel_source_hash(["a.cu", "b.cuh"]) == h1
    (tmp_path / "b.cuh").write_text("body b changed")
    assert bench.kernel_source_hash(["a.cu", "b.cuh"]) != h1
    assert bench.kernel_source_hash(["a.cu", "missing.cuh"]) is None


def test_traffic_is_null_unless_the_sources_match(tmp_path, monkeypatch):
    (tmp_path / "k.cu").write_text("kernel")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    cap = dict(bench.TRAFFIC_CAPTURE, sources=["k.cu"], sha256_16="0" * 16, bytes_per_launch=1234.0)
    monkeypatch.setattr(bench, "TRAFFIC_CAPTURE", cap)
    traffic, note = bench._capture_traffic()
    assert traffic is None and "changed" in note
    cap["sha256_16"] = bench.kernel_source_hash(["k.cu"])
    traffic, note = bench._capture_traffic()
    assert traffic == 1234.0


def test_committed_capture_names_existing_sources():
    for src in bench.TRAFFIC_CAPTURE["sources"]:
        assert bench.kernel_source_hash([src]) is not None, src
