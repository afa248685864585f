"""Host-side arithmetic of bench.py (no GPU): the per-step roofline derived from step times, and the
CPU description of the baseline record."""
import math

import pytest

import bench

STEPS = ["cholesky", "invert", "multiply", "to_band", "to_tridiag", "solve", "back_tridiag", "back_band", "mult",
         "refine"]
MP = {"bf16_tflops_sustained": 1764.7}


def fake_ms(v=100.0):
    return {s: v for s in STEPS}


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("emulated", [False, True])
@pytest.mark.parametrize("fp32_products", [-1, 0, 3, 6])
def test_steps_roofline_every_combination(complex_, mixed, emulated, fp32_products):
    r = bench.steps_roofline(fake_ms(), 1024, 256, 64, complex_, mixed, emulated, 2, fp32_products, MP)
    assert ("refine" in r) == mixed
    for step, row in r.items():
        assert row["ms"] == 100.0 and isinstance(row["engine"], str)
        if step == "solve":
            assert "tflops" not in row
            continue
        assert row["tflops"] > 0 and math.isclose(row["frac"], row["tflops"] / row["peak_tflops"])


def test_steps_roofline_counts():
    n, k, b = 2000, 500, 64
    r = bench.steps_roofline(fake_ms(1000.0), n, k, b, False, False, True, 0, -1, MP)
    # one second per step: TFLOP/s = flops / 1e12
    assert math.isclose(r["multiply"]["tflops"], n ** 3 / 1e12)
    assert math.isclose(r["cholesky"]["tflops"], 2 * n ** 3 / 3 / 1e12)
    assert math.isclose(r["to_band"]["tflops"], 4 * n ** 3 / 3 / 1e12)
    assert math.isclose(r["to_tridiag"]["tflops"], 6 * b * n * n / 1e12)
    assert math.isclose(r["back_tridiag"]["tflops"], 2 * n * n * k / 1e12)
    assert math.isclose(r["mult"]["tflops"], n * n * k / 1e12)
    # emulated FP64 products: 36 BF16 products per FP64 product
    assert math.isclose(r["multiply"]["peak_tflops"], 1764.7 / 36)
    rc = bench.steps_roofline(fake_ms(1000.0), n, k, b, True, False, True, 0, -1, MP)
    assert math.isclose(rc["multiply"]["tflops"], 4 * r["multiply"]["tflops"])
    rm = bench.steps_roofline(fake_ms(1000.0), n, k, b, False, True, True, 3, 6, MP)
    assert math.isclose(rm["refine"]["tflops"], 3 * (2 * n * n * k + 3 * n * k * k) / 1e12)
    assert math.isclose(rm["to_band"]["peak_tflops"], 1764.7 / 6)
    # the mixed form back-transforms all n FP32 vectors; the plain emulated form's back-transform 2 runs on
    # the tensor-core product engine, the native one on the FP64 FMA pipe
    assert math.isclose(rm["back_tridiag"]["tflops"], 2 * n ** 3 / 1e12)
    assert math.isclose(rm["back_band"]["tflops"], 2 * n ** 3 / 1e12)
    assert math.isclose(r["back_tridiag"]["peak_tflops"], 1764.7 / 36)
    rn = bench.steps_roofline(fake_ms(1000.0), n, k, b, False, False, False, 0, -1, MP)
    assert "FMA" in rn["back_tridiag"]["engine"]


def test_steps_roofline_zero_time_has_no_rate():
    r = bench.steps_roofline({"multiply": 0.0}, 64, 16, 16, False, False, True, 0, -1, MP)
    assert "tflops" not in r["multiply"] and r["cholesky"]["ms"] == 0.0


def test_cpu_model_is_a_string():
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
