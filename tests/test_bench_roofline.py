"""The benchmark's roofline arithmetic on the CPU: every `frac` it prints must reproduce from the
context's sizes (nls_sizes) and the kernel's average launch time, with the algorithmic counts the
measurement plan defines -- and not from the implementation's own storage formats.

* k_local_apply: bytes = the band factors of every subdomain read once (total_factor_entries x the
  factor size), the local Jacobian with its boundary columns (12 bytes per nonzero: value + column
  index) and three global vectors (3 N x 8 bytes), against the measured HBM copy bandwidth; the packed
  solve operands only as a reported overhead ratio.
* k_local_newton: flops = lu_flops x (full steps per subdomain + 1 refactorisation) + solve_flops x full
  steps per subdomain; without the refactorisation term when it runs in k_local_factor.
* k_local_factor: flops = lu_flops per launch.
* the tensor-core tile products: 3 TF32 passes of 2 x 128^3 per tile, against the sustained bf16 peak
  times 1.1 / 2.25.
"""
import types

import pytest

import bench

PEAKS = {"hbm_gbs": 6000.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1600.0, "sm_max_mhz": 2000.0}


def sizes(**kw):
    base = dict(n_dofs=1000, n_sub=10, total_factor_entries=50000, factor_bytes=4, total_local_nnz=20000,
                total_solve_entries=70000, lu_flops=3.0e6, solve_flops=4.0e5, n_coarse_dofs=1000,
                coarse_half_band=300)
    base.update(kw)
    return types.SimpleNamespace(**base)


def test_local_apply_counts_the_band_not_the_packed_operands():
    sz = sizes()
    r = bench.roofline_for("k_local_apply<float>", launches=4, ms=2.0, sizes=sz, peaks=PEAKS, peak_kind="measured")
    alg = 50000 * 4 + 20000 * 12 + 3 * 1000 * 8
    avg_s = 2.0e-3 / 4
    assert r["algorithmic_bytes_per_launch"] == alg
    assert r["achieved"] == pytest.approx(alg / avg_s / 1e9, rel=1e-12)
    assert r["frac"] == pytest.approx(alg / avg_s / 1e9 / 6000.0, rel=1e-12)
    assert r["operand_format_overhead"] == pytest.approx(70000 / 50000, rel=1e-12)
    assert r["bound"] == "hbm" and r["peak"] == 6000.0


@pytest.mark.parametrize("split", [False, True])
def test_local_newton_flops_follow_the_refactorisation_split(split):
    sz = sizes()
    steps_per_launch = 25.0  # full local Newton steps of one launch, all subdomains
    r = bench.roofline_for("k_local_newton<neohooke, float, 256>", launches=2, ms=10.0, sizes=sz, peaks=PEAKS,
                           peak_kind="measured", steps_per_launch=steps_per_launch, split_factor=split)
    per_sub = steps_per_launch / 10
    flops = 3.0e6 * (per_sub + (0.0 if split else 1.0)) + 4.0e5 * per_sub
    peak = bench.fp32_peak_tflops(PEAKS)
    assert r["algorithmic_flops_per_launch"] == pytest.approx(flops, rel=1e-12)
    assert r["frac"] == pytest.approx(flops / 5.0e-3 / 1e12 / peak, rel=1e-12)
    # 152 SMs x 128 FP32 lanes x 2 flops x the maximum SM clock
    assert peak == pytest.approx(152 * 128 * 2 * 2000.0e6 / 1e12, rel=1e-12)


def test_local_factor_counts_one_lu_per_subdomain():
    sz = sizes()
    r = bench.roofline_for("k_local_factor<float>", launches=3, ms=6.0, sizes=sz, peaks=PEAKS, peak_kind="measured")
    assert r["algorithmic_flops_per_launch"] == 3.0e6
    assert r["achieved"] == pytest.approx(3.0e6 / 2.0e-3 / 1e12, rel=1e-12)


def test_tensor_products_use_the_sustained_peak():
    sz = sizes()
    r = bench.roofline_for("k_tile_solve_products", launches=1, ms=0.1, sizes=sz, peaks=PEAKS, peak_kind="measured")
    NT, TB = 8, 3  # ceil(1000 / 128), ceil(300 / 128)
    tiles = sum(1 for t in range(NT) for k in range(1, TB + 1) if t - k >= 0) + \
        sum(1 for t in range(NT) for k in range(1, TB + 1) if t + k < NT)
    flops = 3 * 2 * 128 ** 3 * tiles
    assert r["tf32_flops_per_launch"] == flops
    assert r["peak"] == pytest.approx(1600.0 * 1.1 / 2.25, rel=1e-12)
    assert r["frac"] == pytest.approx(flops / 1e-4 / 1e12 / r["peak"], rel=1e-12)
