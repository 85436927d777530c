"""The FMA-throughput microbenchmark (jf_fma_peak) that gives the measured
ALU roofline beside the derived one (SMs x 128 FP32 lanes x 2 x clock)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_13760_gb300 import jf  # noqa: E402


def test_fma_peak_fp32_near_the_unit_count():
    props = torch.cuda.get_device_properties(0)
    derived = props.multi_processor_count * 128 * 2 * 2.07e9  # lanes x FMA x maximum SM clock
    measured = jf.fma_peak("f32", iters=3000)
    assert 0.5 * derived < measured < 1.05 * derived, (measured, derived)


def test_fma_peak_fp64_below_fp32():
    f32 = jf.fma_peak("f32", iters=3000)
    f64 = jf.fma_peak("f64", iters=100)
    assert 0.0 < f64 < f32 / 4, (f64, f32)
