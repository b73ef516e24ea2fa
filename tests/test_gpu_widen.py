"""The exact FP32 -> FP64 widening the refinement kernels apply to FP32
matrices (integer operations instead of the conversion instruction, which
runs at the FP64 rate on this GPU), through hqr_widen_f32, against the
conversion instruction (torch's float -> double) over every FP32 bit
pattern: zeros, subnormals, normal numbers, infinities and NaNs."""
import pytest

torch = pytest.importorskip("torch")
hqr = pytest.importorskip("paper_1110_1553_gb300.hqr")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1110_1553_gb300 import _build
    _build.build()
    hqr.load()


def test_widen_every_fp32_bit_pattern():
    chunk = 1 << 27
    quiet = 1 << 51  # a signalling NaN stays signalling in the integer form
    y = torch.empty(chunk, dtype=torch.float64, device="cuda")
    for start in range(0, 1 << 32, chunk):
        bits = torch.arange(start, start + chunk, dtype=torch.int64, device="cuda")
        x = torch.where(bits >= (1 << 31), bits - (1 << 32), bits).to(torch.int32).view(torch.float32)
        hqr.widen_f32(x, y)
        ref = x.double()
        yb, rb = y.view(torch.int64), ref.view(torch.int64)
        nan = torch.isnan(x)
        assert torch.equal(yb[~nan], rb[~nan]), hex(start)
        assert bool(torch.isnan(y[nan]).all())
        assert torch.equal(yb[nan] | quiet, rb[nan] | quiet), hex(start)
    torch.cuda.synchronize()


def test_widen_argument_errors():
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    y = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        hqr.widen_f32(x, y)
    lib = hqr.load()
    assert lib.hqr_widen_f32(None, None, -1, None) == -3
    assert lib.hqr_widen_f32(None, None, 0, None) == 0
