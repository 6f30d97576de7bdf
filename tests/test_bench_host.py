"""Host-side arithmetic of bench.py (no GPU): the algorithmic bytes per stage against their
closed forms, the roofline fractions, the views of the spreading kernel built from a committed
ncu summary, and that the summary the headline roofline reads was taken on the current kernel
source."""
import os

import pytest

import bench

RADIAL = {"N": (512, 512), "n": (1024, 1024), "name": "2d_radial_N512_M1048576_m4"}
M = 1048576


def test_algorithmic_bytes_closed_forms():
    # per node: 2 offsets (8 B) + cell index and permutation (8 B) + complex value (8 B)
    node = M * 24
    G = 1024 * 1024 * 8
    assert bench.algorithmic_bytes("interp", 2, RADIAL["N"], RADIAL["n"], M, 4) == node + G
    assert bench.algorithmic_bytes("spread", 2, RADIAL["N"], RADIAL["n"], M, 4) == node + 2 * G
    # FFT: compact coefficients + full grid + the pruned intermediate written and read
    fft = 512 * 512 * 8 + G + 2 * 512 * 1024 * 8
    assert bench.algorithmic_bytes("fft_forward", 2, RADIAL["N"], RADIAL["n"], M, 4) == fft
    assert bench.algorithmic_bytes("fft_adjoint", 2, RADIAL["N"], RADIAL["n"], M, 4) == fft
    # FP64 doubles the offsets, values and grid cells, not the 4-byte cell index and permutation;
    # 3-D adds the second pruned intermediate
    assert bench.algorithmic_bytes("spread", 2, RADIAL["N"], RADIAL["n"], M, 8) == \
        M * (16 + 8 + 16) + 2 * 2 * G
    N3, n3 = (128,) * 3, (256,) * 3
    inter = 128 * 128 * 256 + 128 * 256 * 256
    assert bench.algorithmic_bytes("fft_forward", 3, N3, n3, 10, 4) == \
        (128 ** 3 + 256 ** 3 + 2 * inter) * 8


def test_roofline_of_picks_the_dominant_kernel():
    stages = {"fft_forward": {"ms_per_launch": 0.021}, "interp": {"ms_per_launch": 0.039},
              "zero_grid": {"ms_per_launch": 0.006}, "spread": {"ms_per_launch": 0.057},
              "fft_adjoint": {"ms_per_launch": 0.021}}
    r = bench.roofline_of(stages, RADIAL, M, 4, 6780.0, "measured")
    assert r["kernel"] == "spread"
    alg = bench.algorithmic_bytes("spread", 2, RADIAL["N"], RADIAL["n"], M, 4)
    assert r["achieved"] == pytest.approx(alg / 0.057e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6780.0)
    shares = [v["share"] for k, v in stages.items() if k != "zero_grid"]
    assert sum(shares) == pytest.approx(1.0)


def test_spreading_views_from_the_committed_summary():
    v = bench.onchip_roofline("spread", RADIAL, M, 4, 0.057, {"sm_mhz": 2070.0})
    peak = bench.NUM_SMS * 2.07e9
    assert v["peak_wavefronts_per_s"] == pytest.approx(peak)
    assert v["tap_floor_wavefronts"] == pytest.approx(M * 64 * 16 / 128)
    assert "issue" in v and 0 < v["issue"]["frac"] < 1.2
    assert v["issue"]["peak_per_s"] == pytest.approx(bench.NUM_SMS * 4 * 2.07e9)
    assert bench.onchip_roofline("interp", RADIAL, M, 4, 0.039, None) is None


def test_headline_profile_matches_the_kernel_source():
    """The summary whose DRAM traffic the headline roofline reports was captured on the
    spreading source as it is now (else bench reports no traffic)."""
    path = os.path.join(bench.ROOT, "profiles", f"spread_{RADIAL['name']}.txt")
    vals = dict(line.split(":", 1) for line in open(path) if ":" in line)
    assert vals["kernel_source_sha"].strip() == bench.source_sha(bench.STAGE_SOURCES["spread"])
    assert bench.profiled_traffic("spread", RADIAL["name"]) > 0
