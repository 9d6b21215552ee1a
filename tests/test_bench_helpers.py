"""Host helpers of bench.py (CPU): the ncu traffic figure is reported only
while the kernel source matches the capture (hash) and the capture is of
the workload being timed; the roofline peak falls back to the stated
figures when the measured file is absent."""
import hashlib
import os

import bench


def _setup(tmp_path, src_text: str, recorded_sha: str, key: str):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_text(src_text)
    (tmp_path / "profiles" / "k.md").write_text(
        "# capture\n\ndram_bytes_per_launch_full_size = 123456789\n"
        f"source_sha256 = {recorded_sha}\napplies_to = {key}\n")


def test_traffic_needs_matching_source_and_workload(tmp_path, monkeypatch):
    src = "__global__ void k() {}\n"
    sha = hashlib.sha256(src.encode()).hexdigest()[:16]
    _setup(tmp_path, src, sha, "3d 256^3 r32 T32")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("k.md", "k.cu", "3d 256^3 r32 T32") == 123456789.0
    assert bench.profile_traffic("k.md", "k.cu", "3d 128^3 r32 T32") is None  # another workload
    assert bench.profile_traffic("missing.md", "k.cu", "3d 256^3 r32 T32") is None
    (tmp_path / "k.cu").write_text(src + "// changed\n")  # the source changed since the capture
    assert bench.profile_traffic("k.md", "k.cu", "3d 256^3 r32 T32") is None


def test_peak_fallback_without_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    hbm, bf16, kind = bench.measured_peaks()
    assert (hbm, bf16, kind) == (6800.0, 1900.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6698.5, "bf16_tflops": 1938.1}')
    assert bench.measured_peaks() == (6698.5, 1938.1, "measured")


def test_committed_profiles_parse():
    """Every committed capture summary names its figure, source hash and workload."""
    root = os.path.dirname(os.path.abspath(bench.__file__))
    for f in ("stencil_step_3d_256cubed.md", "probe_gemm_3d_256cubed.md"):
        text = open(os.path.join(root, "profiles", f)).read()
        for field in ("dram_bytes_per_launch_full_size", "source_sha256", "applies_to", "ncu "):
            assert field in text, (f, field)
        assert "--clock-control none" in text


def test_every_profile_gives_its_ncu_command():
    """Each summary under profiles/ states the ncu command that made it, with
    the clocks left alone (--clock-control none on every ncu line)."""
    root = os.path.join(os.path.dirname(os.path.abspath(bench.__file__)), "profiles")
    names = sorted(f for f in os.listdir(root) if f.endswith(".md"))
    assert len(names) >= 5
    for f in names:
        lines = open(os.path.join(root, f)).read().splitlines()
        cmds, cur = [], None  # commands with their backslash-continued lines joined
        for ln in lines:
            if cur is None and ln.lstrip().startswith("ncu "):
                cur = ""
            if cur is not None:
                cur += " " + ln.rstrip().rstrip("\\")
                if not ln.rstrip().endswith("\\"):
                    cmds.append(cur)
                    cur = None
        assert cmds, f
        assert all("--clock-control none" in c for c in cmds), f
