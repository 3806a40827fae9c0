"""FMA throughput probes (spai_measure_fp64_rate, spai_measure_fp32_rate): the measured
counterparts of the derived ALU roofs the benchmark reports kernels against.

GB300 nominal rates: FP64 152 SM x 2 FMA/clk x 2 flop x 2.07 GHz = 1.26 TFLOP/s; FP32
152 SM x 128 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s.  A chain of FMAs on every SM
reaches a large part of either (clocks under load may sit below the maximum), never more.
"""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1809_06574_gb300 as sg
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = sg.spai_ctx_create(torch.cuda.current_stream().cuda_stream, 0)
    yield c
    sg.spai_ctx_destroy(c)


def test_fma_probes_plausible(ctx):
    import paper_1809_06574_gb300 as sg
    fp64 = max(sg.spai_measure_fp64_rate(ctx) for _ in range(3))
    fp32 = max(sg.spai_measure_fp32_rate(ctx) for _ in range(3))
    assert 0.3 < fp64 < 1.3, fp64
    assert 20.0 < fp32 < 82.0, fp32
    # the FP32 pipe is 64 lanes per FP64 lane on this part; with the clocks of a short probe
    # the measured ratio stays well above 16
    assert fp32 / fp64 > 16.0, (fp32, fp64)


def test_fma_probes_reject_null(ctx):
    import paper_1809_06574_gb300 as sg
    assert sg.lib().spai_measure_fp32_rate(None, None) == sg.SPAI_EINVAL
    assert sg.lib().spai_measure_fp32_rate(ctx, None) == sg.SPAI_EINVAL
    assert sg.lib().spai_measure_fp64_rate(ctx, None) == sg.SPAI_EINVAL
