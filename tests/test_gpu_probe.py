"""The FMA-throughput probe behind the roofline denominators: it runs,
rejects bad arguments, and its two figures are plausible for GB300 (FP32 FMA
at most the 152 SMs x 128 lanes x 2 flop x 2.1 GHz of the part; FP64 below
the nominal 1.26 TFLOP/s and far below FP32)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1711_03590_gb300 as dgp  # noqa: E402


def test_peak_probe():
    dgp.build()
    f64 = dgp.dg_peak_probe(0)
    f32 = dgp.dg_peak_probe(1)
    assert 0.3 < f64 < 1.3
    assert 20.0 < f32 < 152 * 128 * 2 * 2.1e9 / 1e12
    assert f32 > 20 * f64
    with pytest.raises(dgp.DGError):
        dgp.dg_peak_probe(2)
