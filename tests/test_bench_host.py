"""Host arithmetic of bench.py that its reported figures rest on, without a
GPU: the flop count of a factorisation block against its closed form, the
blocks the recursive factorisation of the fit's M = 2000 Gram matrix hands
to the block kernel, the number of moduli the exact Gram matrix and the
congruences need, the CUDA-core rooflines' arithmetic, and the clock
sampler's reading of an nvidia-smi log (a fake log: nothing is run)."""
import os
import sys
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("m", [1, 2, 3, 17, 32, 64])
def test_block_flops_closed_form(m):
    """Elimination on [A | I]: step k updates rows i > k on (m - i) + (k + 1)
    live columns.  Summed, sum_k sum_{i>k} (m - i) = sum_k (k + 1)(m - k - 1)
    = (m - 1) m (m + 1) / 6 each, so the flops are 2 (m^3 - m) / 3."""
    assert bench.block_flops(m) == pytest.approx(2.0 * (m ** 3 - m) / 3.0, rel=0, abs=0)


def test_factorisation_blocks_of_the_fit():
    blocks = bench.chol_blocks(2000)
    assert sum(blocks) == 2000 and max(blocks) <= 64 and len(blocks) == 32
    assert bench.block_flops(64) == pytest.approx(0.17e6, rel=0.03)
    assert bench.chol_blocks(64) == [64] and bench.chol_blocks(65) == [32, 33]  # halves, rounded to 32


def test_moduli_of_the_fit():
    """16 moduli <= 256 (125.4 bits) hold the exact pass-1 Gram matrix of the
    fit's 75,176 + 2,000 stacked rows (< 2^(107 + log2 m)); the congruences
    need 31 (the 16 plus primes up to 509)."""
    T1, T2 = bench.crt_moduli_counts(77176, 2001)
    assert (T1, T2) == (16, 31)
    assert sum(np.log2(bench.CRT_MODULI[:16])) == pytest.approx(125.4, abs=0.05)


def test_alu_roofline_arithmetic():
    per = {"expansion": 0.5, "pairforce": 0.25, "knm_jacobian": 2.0, "solve_block": 0.075}
    r = bench.alu_rooflines(per, n_atoms=1000, n_pairs=30000, n_max=8, l_max=6, D=252, M=2000, fp32_peak=80.0,
                            fp64_peak=1.2, hbm=6800.0, n_sm=152, n_fact=2)
    for st in ("expansion", "pairforce", "knm_jacobian"):
        e = r[st]
        assert e["achieved_tflops"] == pytest.approx(e["flops"] / (per[st] * 1e-3) / 1e12)
        assert e["frac"] == pytest.approx(e["achieved_tflops"] / 80.0)
        assert e["hbm_frac"] == pytest.approx(e["hbm_bytes"] / (per[st] * 1e-3) / 1e9 / 6800.0)
    # Jacobian rows: 3 (N + P) rows x 2 BF16 planes x D16 x 2 bytes
    assert r["knm_jacobian"]["hbm_bytes"] == 3 * (1000 + 30000) * 2 * 256 * 2
    b = r["solve_block"]
    assert b["blocks_per_factorisation"] == 32
    assert b["peak_tflops"] == pytest.approx(1.2 / 152) and b["frac_of_chip"] == pytest.approx(b["frac"] / 152)


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    s.f.write("\n".join(lines) + "\n")
    s.f.flush()
    s.p = _Done()
    return s


def test_clock_log_reading():
    na = "Not Active"
    rows = [f"0, {mhz}, 2070, 900.5, 0x0000000000000000, {na}, {na}, {na}, {cap}"
            for mhz, cap in ((2070, na), (2055, "Active"), (2070, na), (1980, na))]
    out = _sampler(rows + ["garbage line"]).stop()
    assert out["sm_mhz"] == pytest.approx(2062.5) and out["sm_max_mhz"] == 2070.0 and out["samples"] == 4
    assert out["reasons"] == ["sw_power_cap"]
    hot = _sampler([f"0, 1500, 2070, 1400.0, 0x48, {na}, Active, {na}, {na}"]).stop()
    assert hot["reasons"] == ["hw_thermal_slowdown"]
