"""The FP32-bulk kernels convert FP64 values to FP32 (and FP32 results back)
on the integer pipe, with the library's own IEEE 754 conversion.  It must
round exactly like the hardware conversion (to nearest, ties to even), so the
FP32-bulk results do not depend on which unit converted them: checked bit for
bit against PyTorch's (hardware) conversion on special values, ties, the
binary32 subnormal and overflow ranges, random bit patterns of every
exponent, and the value ranges of the flow states."""
import numpy as np
import pytest

from gpu_util import gpu_or_skip

pytestmark = pytest.mark.gpu


def _inputs():
    rng = np.random.default_rng(11)
    f32max = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    sub = 2.0 ** -149
    special = [0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, f32max, -f32max, f32max * (1 + 2 ** -25),
               f32max * (1 + 2 ** -24), f32max * 2, tiny, -tiny, tiny * (1 - 2 ** -30), sub, -sub, sub / 2,
               sub * 1.5, sub * 2.5, sub * 0.75, sub / 4, 1e-300, -1e-300, 1e300, 2.0 ** -1074, 3.0, 0.1]
    # exact ties: 1 + (2k + 1) 2^-24 lies halfway between two binary32 values
    ties = [(1.0 + (2 * k + 1) * 2.0 ** -24) * 2.0 ** s for k in range(8) for s in (-130, -20, 0, 7, 100)]
    bits = rng.integers(0, 2 ** 63, size=200000, dtype=np.int64).view(np.float64)
    bits = bits[np.isfinite(bits)]
    expo = (rng.uniform(-1.0, 1.0, 100000) * 2.0 ** rng.integers(-160, 140, 100000)).astype(np.float64)
    flow = np.concatenate([rng.uniform(0.1, 3.0, 50000), rng.normal(0.0, 1e-3, 50000), rng.uniform(50, 300, 50000),
                           rng.normal(0.0, 1e-9, 50000)])
    return np.concatenate([np.array(special + ties), bits, expo, flow])


def test_integer_pipe_conversions_match_the_hardware():
    torch, dg = gpu_or_skip()
    x = torch.from_numpy(_inputs()).cuda()
    out, back = dg.convert_check(x)
    ref = x.float()
    torch.cuda.synchronize()
    a = out.view(torch.int32).cpu().numpy()
    r = ref.view(torch.int32).cpu().numpy()
    nan = np.isnan(ref.cpu().numpy())
    assert np.array_equal(np.isnan(out.cpu().numpy()), nan)
    mism = np.nonzero((a != r) & ~nan)[0]
    assert mism.size == 0, (x.cpu().numpy()[mism[:5]], a[mism[:5]], r[mism[:5]])
    b = back.view(torch.int64).cpu().numpy()
    rb = out.double().view(torch.int64).cpu().numpy()
    bn = np.isnan(out.cpu().numpy())
    assert np.array_equal(b[~bn], rb[~bn])
    # NaN inputs come out as NaN
    xn = torch.tensor([float("nan"), -float("nan")], dtype=torch.float64, device="cuda")
    o, bk = dg.convert_check(xn)
    assert torch.isnan(o).all() and torch.isnan(bk).all()
