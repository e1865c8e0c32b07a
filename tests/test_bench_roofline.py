"""The bench's roofline objects on the CPU: achieved = algorithmic work per build over the kernel's
measured time, frac = achieved over the measured peak, and the leaf kernel's DRAM traffic taken
from its committed ncu summary only while that summary's source hash matches the kernel source."""
import hashlib
import os

import pytest

import bench
import synth


def _stats(builds, **kw):
    base = dict(leaf_pairs=2.0e12, ms_leaf_kernel=1000.0, leaf_kernel_launches=12, reservoir_slots=4.0e9,
                ms_prune_kernel=1000.0)
    base.update(kw)
    return [dict(base) for _ in range(builds)]


def test_leaf_roofline_arithmetic():
    peaks, _ = bench.measured_peaks()
    r = bench.leaf_roofline(_stats(3), 128, "simt", "leaf_tc.cu", "no-such-profile.md")
    # 2e12 pairs x 128 flops per pair in 1 s
    assert r["achieved"] == pytest.approx(2.0e12 * 128 / 1e12)
    assert r["peak"] == peaks["bf16_tflops"]
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["launches_per_build"] == 12 and r["ms_per_build"] == 1000.0
    assert r["traffic"] is None and r["bound"] == "tensor" and r["unit"] == "TFLOP/s"


def test_leaf_traffic_follows_the_profile_only_for_the_profiled_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2602_21247_gb300" / "csrc"
    prof = tmp_path / "profiles"
    csrc.mkdir(parents=True)
    prof.mkdir()
    src = b"// a kernel\n"
    (csrc / "k.cu").write_bytes(src)
    sha = hashlib.sha256(src).hexdigest()[:16]
    (prof / "k.md").write_text(f"kernel_source_sha256_16: {sha}\n\ndram_bytes_per_build: 2.4e+12\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    r = bench.leaf_roofline(_stats(2), 128, "tc", "k.cu", "k.md")
    assert r["traffic"] == pytest.approx(2.4e12 / 12)
    # the source changed since the capture: no traffic figure
    (csrc / "k.cu").write_bytes(src + b"// changed\n")
    assert bench.leaf_roofline(_stats(2), 128, "tc", "k.cu", "k.md")["traffic"] is None


def test_committed_leaf_profiles_parse():
    # every committed leaf summary names a source hash and a per-build DRAM figure
    for name in ("leaf_gram_tc_spacev-like-i8.md", "leaf_gram_tc_bigann-like-u8.md"):
        text = open(os.path.join(bench.ROOT, "profiles", name)).read()
        assert "kernel_source_sha256_16:" in text and "dram_bytes_per_build:" in text


def test_prune_roofline_arithmetic():
    w = dict(synth.WORKLOADS["spacev-like-i8"])
    n = 1000
    peaks, _ = bench.measured_peaks()
    r = bench.prune_roofline(_stats(2, reservoir_slots=5000.0, ms_prune_kernel=2.0), w, n)
    per_build = 5000 * (8 + 128) + n * (128 + 4 + 64 * 4 + 4)
    assert r["algorithmic_bytes_per_build"] == per_build
    assert r["achieved"] == pytest.approx(per_build / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / peaks["hbm_gbs"])
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
