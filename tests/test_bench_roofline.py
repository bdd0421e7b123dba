"""The FMA-rate roofline bench.py reports for the FP32 SIMT step: FMA count per step from the
contractions' definition (k per element for the projection; k or 2k for the back-projection
with or without split batches) and the peak from the unit count and clock. CPU only."""
import bench


def test_fma_roofline_counts_and_peak():
    r = bench.fma_roofline(b=4096, d=32768, k=32, ms=1.0, n_sms=152, sm_mhz=2070.0)
    assert r["bound"] == "alu" and r["unit"] == "TFMA/s"
    assert r["fma_per_step"] == 2 * 4096 * 32768 * 32
    assert abs(r["peak"] - 152 * 128 * 2.07e9 / 1e12) < 1e-9
    assert abs(r["achieved"] - r["fma_per_step"] / 1e-3 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12


def test_fma_roofline_unsplit_back_projection_doubles():
    split = bench.fma_roofline(8, 10, 2, 1.0, 1, 1000.0, split=True)["fma_per_step"]
    unsplit = bench.fma_roofline(8, 10, 2, 1.0, 1, 1000.0, split=False)["fma_per_step"]
    assert (split, unsplit) == (2 * 8 * 10 * 2, 3 * 8 * 10 * 2)
