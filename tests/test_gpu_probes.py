"""GPU checks of the two probes the library exports for measurement and accuracy:
the FP32 throughput probe that gives the tracking kernel's roofline its measured
denominator, and the FP64 exponential behind the EPIC fit weights (Tang's
table-driven method), against an extended-precision reference exponential."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_09971_gb300 as m
    return m.load()


def stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def exp_neg_gpu(lib, y):
    yd = torch.from_numpy(np.ascontiguousarray(y, np.float64)).cuda()
    out = torch.empty_like(yd)
    assert lib.dgf_epic_exp_neg(ctypes.c_void_p(yd.data_ptr()), ctypes.c_void_p(out.data_ptr()), len(y), stream()) == 0
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_exp_neg_against_an_extended_precision_exp(lib):
    """exp(-y) for y in [0, 745.2) within 2 ulps of the double result (so within
    4.5e-16 relative while the result is a normal double, up to y = 708.39, and within
    two units of the smallest subnormal below that; measured 1.93 and 1.27); zero from
    745.2 on, where exp(-y) is below half the smallest subnormal."""
    rng = np.random.default_rng(0)
    y = np.concatenate([np.linspace(0.0, 745.2, 1_000_001)[:-1], rng.uniform(0, 745.2, 1_000_000),
                        rng.uniform(0, 1e-3, 100_000), np.ldexp(1.0, -np.arange(1, 1075)),
                        [0.0, 5e-324, 708.3964185322641, 708.3964185322642, 744.44, 745.13, 745.1332]])
    g = exp_neg_gpu(lib, y)
    ref = np.exp(-y.astype(np.longdouble))  # 80-bit (x86) or 128-bit (Arm) long double
    ulp = np.spacing(ref.astype(np.float64)).astype(np.longdouble)  # the smallest subnormal below 2^-1022
    err_ulp = np.abs(g.astype(np.longdouble) - ref) / ulp
    normal = ref >= np.finfo(np.float64).tiny
    print(f"exp(-y): max error {float(err_ulp[normal].max()):.3f} ulp on {normal.sum()} normal results, "
          f"{float(err_ulp[~normal].max()):.3f} on {(~normal).sum()} subnormal ones")
    assert float(err_ulp.max()) <= 2.0
    assert np.all(exp_neg_gpu(lib, np.array([745.2, 746.0, 800.0, 1e4, 1e300])) == 0.0)
    assert exp_neg_gpu(lib, np.array([0.0]))[0] == 1.0


def test_fp32_probe_measures_a_plausible_rate(lib):
    """The probe runs on every SM and reports a rate in the range a GB300 can reach
    (scalar and packed FMA; the packed form issues two FMAs per lane)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, threads, iters = sms * 8, 256, 2000
    out = torch.empty(blocks * threads, dtype=torch.float32, device="cuda")
    rates = {}
    for packed in (0, 1):
        assert lib.dgf_fp32_probe(ctypes.c_void_p(out.data_ptr()), blocks, threads, iters, packed, stream()) == 0
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        assert lib.dgf_fp32_probe(ctypes.c_void_p(out.data_ptr()), blocks, threads, iters, packed, stream()) == 0
        b.record()
        b.synchronize()
        rates[packed] = lib.dgf_fp32_probe_flops(blocks, threads, iters, packed) / (a.elapsed_time(b) * 1e-3) / 1e12
    print(f"FP32 probe on {sms} SMs: scalar {rates[0]:.1f} TFLOP/s, packed {rates[1]:.1f} TFLOP/s")
    assert 10.0 < rates[0] < 400.0 and 10.0 < rates[1] < 400.0
    v = out.cpu().numpy()
    assert np.all(np.isfinite(v))  # v <- v/2 + 1 stays near 2 in every chain
