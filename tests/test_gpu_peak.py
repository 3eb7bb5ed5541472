"""The FMA-throughput launch behind the ALU roofline (sph_fma_peak).

Each of its chains iterates a <- 0.999 a + 1e-3 from a0 = (t mod 16)/16 + k,
so after n rounds a = 1 + 0.999^n (a0 - 1): the sink holds the sum of the 8
chains, and the reported operations are 2 x 8 x threads x rounds."""
import numpy as np
import pytest
import torch

import paper_2411_13992_gb300 as sph

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,dtype,rtol", [(32, torch.float32, 1e-4), (64, torch.float64, 1e-12)])
def test_fma_peak_launch_computes_the_recurrence(precision, dtype, rtol):
    blocks, iters = 3, 500
    sink = torch.zeros(blocks * 256, dtype=dtype, device="cuda")
    flops = sph.sph_fma_peak(precision, blocks, iters, sink)
    torch.cuda.synchronize()
    assert flops == 2.0 * 8 * blocks * 256 * iters
    t = np.arange(blocks * 256)
    a0 = (t % 16)[:, None] * 0.0625 + np.arange(8)[None, :]
    expect = (1.0 + 0.999 ** iters * (a0 - 1.0)).sum(axis=1)
    np.testing.assert_allclose(sink.cpu().numpy(), expect, rtol=rtol)


def test_fp32_fma_peak_is_near_the_unit_count_bound():
    """Measured FP32 FMA rate between 50 % and 105 % of 152 SMs x 128 lanes x
    2 flops x the maximum SM clock (80.5 TFLOP/s)."""
    import bench
    rate = bench.measured_fma_peak(torch, sph, 32, target_ms=10.0)
    bound = bench.fp32_peak_tflops(bench.SM_MAX_MHZ)
    print("FP32 FMA %.1f TFLOP/s of %.1f; FP64 FMA %.2f TFLOP/s" % (rate, bound,
          bench.measured_fma_peak(torch, sph, 64, target_ms=10.0)))
    assert 0.5 * bound < rate < 1.05 * bound
