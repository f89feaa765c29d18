"""Host-side arithmetic of bench.py (CPU only): the roofline figures, the normwise error
and the traffic lookup that the JSON line reports."""
import os

import numpy as np
import pytest

import bench


def test_roofline_of_the_contraction_by_hand():
    """8 flops per path-sample over the kernel's own time, against the peak it is given.
    18,068,275,200 path-samples in 0.23477 ms is 615.7 TFLOP/s, 0.323 of 1904.1; the split
    tiers execute three products per path-sample."""
    samples = 18_068_275_200
    r = bench._roofline("split_fp16", 2 * 0.23477, 2, samples, {"bf16_tflops": 1904.1}, "measured")
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s" and r["kernel"] == "umma_contract"
    assert r["achieved"] == pytest.approx(615.69, abs=0.01)
    assert r["frac"] == pytest.approx(615.69 / 1904.1, abs=1e-4)
    assert r["executed_tflops"] == pytest.approx(3 * 615.69, abs=0.05)
    assert r["kernel_ms"] == pytest.approx(0.23477)
    plain = bench._roofline("bf16", 0.1, 1, samples, {"bf16_tflops": 1904.1}, "measured")
    assert plain["executed_tflops"] == pytest.approx(plain["achieved"], rel=1e-3)


def test_roofline_of_the_direct_sum_uses_the_fma_peak():
    """FP32 direct sum: 152 SMs x 128 lanes x 2 flops at the maximum SM clock."""
    r = bench._roofline("fp32", 2.8, 1, 10 ** 10, {"sm_max_mhz": 2070.0}, "measured")
    assert r["bound"] == "alu" and r["kernel"] == "direct_sum"
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12, abs=1e-3)
    assert r["achieved"] == pytest.approx(8e10 / 2.8e-3 / 1e12, abs=1e-3)


def test_rel_l2_is_normwise():
    """||got - ref|| / ||ref|| over the whole array (the absolute norm when ref is zero); a
    mean of per-entry relative errors would give 0.05 on the last pair, not 0.00995."""
    assert bench._rel_l2(np.array([3 + 4j]), np.array([0j])) == pytest.approx(5.0)
    assert bench._rel_l2(np.array([1 + 1j, 0]), np.array([1, 0])) == pytest.approx(1.0)
    x = np.array([[1 + 2j, -3j], [0.5, 4]])
    assert bench._rel_l2(x, x) == 0.0
    assert bench._rel_l2(np.array([1.1, 10.0]), np.array([1.0, 10.0])) == pytest.approx(0.1 / np.sqrt(101.0))


def test_traffic_lookup_follows_the_kernel_source(tmp_path, monkeypatch):
    """A recorded DRAM byte count is reported only while the kernel source still has the
    hash it was captured at; comment lines and other tiers are ignored."""
    csrc = tmp_path / "paper_2307_09226_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = csrc / "k_umma.cu"
    src.write_text("// kernel v1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash("split_fp16")
    assert len(h) == 12
    (tmp_path / "profiles" / "traffic.txt").write_text(
        f"# split_fp16 {h} 1\nsplit_bf16 {h} 2\nsplit_fp16 {h} 107215616\n")
    assert bench._load_traffic("split_fp16") == 107215616.0
    assert bench._load_traffic("split_bf16") == 2.0
    src.write_text("// kernel v2\n")
    assert bench._load_traffic("split_fp16") is None
    os.remove(tmp_path / "profiles" / "traffic.txt")
    assert bench._load_traffic("split_fp16") is None
