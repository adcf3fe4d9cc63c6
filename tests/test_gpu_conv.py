"""GPU parity of the tensor-core 3x3 convolution (tcgen05, BF16 operands,
FP32 accumulation) against the FP64 oracle on the same bf16 inputs: whole
outputs on ragged images (tiles of 16 x 8 pixels that leave the image), both
channel-block widths, bias and SiLU, bf16 output, a single pixel, and sampled
outputs of the benchmark launch (152 x 70 x 70, 128 -> 128 channels)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import conv as C  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_16393_gb300 import api as A
    return A


def bf16_inputs(seed, n, h, w, cin, cout, scale=1.0):
    """bf16 tensors on the device and the same values in float64 (rounded on the host)."""
    rng = np.random.default_rng(seed)
    x = torch.tensor(rng.standard_normal((n, h, w, cin), dtype=np.float32)).to(torch.bfloat16)
    wt = torch.tensor(scale * rng.standard_normal((cout, 3, 3, cin), dtype=np.float32) /
                      np.sqrt(9 * cin)).to(torch.bfloat16)
    b = torch.tensor(rng.standard_normal(cout, dtype=np.float32))
    return (x.to(DEV), wt.to(DEV), b.to(DEV),
            x.double().numpy(), wt.double().numpy(), b.double().numpy())


def bound(x, w, y_ref, cin, out_bf16, act):
    """Rounding bound: any order of the 9 cin FP32 additions of exact bf16
    products errs by at most 9 cin 2^-23 sum |x w| (truncating adds), SiLU's
    slope is below 1.1, and a bf16 output adds half an ulp (2^-9 relative)."""
    e = 9 * cin * 2.0 ** -23 * C.abs_sum(x, w)
    if act:
        e = 1.1 * e
    if out_bf16:
        e = e + 2.0 ** -8 * np.abs(y_ref)
    return e + 1e-30


@pytest.mark.parametrize("n,h,w,cin,cout,act,use_bias,out_bf16", [
    (2, 70, 70, 64, 64, 0, False, False),      # 70 = 4 x 16 + 6 and 8 x 8 + 6: ragged tiles
    (1, 13, 37, 128, 128, 1, True, False),     # 128-channel blocks, bias + SiLU
    (1, 9, 20, 192, 192, 0, True, True),       # a 128-channel block + a 64-channel remainder
    (1, 1, 1, 64, 64, 0, False, False),        # one pixel: the centre tap only
    (3, 64, 64, 64, 128, 1, True, False),      # tiles cover the image exactly
    (1, 9, 20, 128, 384, 1, True, True),       # three 128-channel blocks, pixels as the MMA's N
    (1, 21, 19, 256, 256, 1, True, True),      # 256-channel blocks (the widest MMA)
    (2, 16, 24, 64, 512, 0, True, False),      # two 256-channel blocks from 64 input channels
])
def test_conv_matches_oracle(api, n, h, w, cin, cout, act, use_bias, out_bf16):
    x, wt, b, xo, wo, bo = bf16_inputs(n * 1000 + cin, n, h, w, cin, cout)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    y = api.conv3x3(x, wt, b if use_bias else None, act,
                    torch.bfloat16 if out_bf16 else torch.float32, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    y_ref = C.conv3x3(xo, wo, bo if use_bias else None, act)
    err = np.abs(y.double().cpu().numpy() - y_ref)
    lim = bound(xo, wo, y_ref, cin, out_bf16, act)
    assert np.all(err <= lim), float((err / lim).max())
    # the bound is tight enough to see a wrong tap or a transposed operand
    assert float(np.abs(y_ref).max()) > 100 * float(lim.max())


def test_conv_benchmark_launch_sampled(api):
    n, h, w, c = 152, 70, 70, 128
    x, wt, b, xo, wo, bo = bf16_inputs(77, n, h, w, c, c)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    y = api.conv3x3(x, wt, b, 1, torch.bfloat16, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    rng = np.random.default_rng(5)
    pix = [(0, 0, 0), (n - 1, h - 1, w - 1), (3, 0, w - 1), (100, h - 1, 0)] + \
        [(int(rng.integers(n)), int(rng.integers(h)), int(rng.integers(w))) for _ in range(60)]
    ch = list(range(c))
    ref = C.conv3x3_at(xo, wo, bo, 1, pix, ch)
    yh = y.float().cpu().numpy()
    got = np.stack([yh[bb, iy, ix] for bb, iy, ix in pix])
    # per-sample bound: |x| |w| summed over the 3 x 3 x cin window
    xa, wa = np.abs(xo), np.abs(wo)
    for k, (bb, iy, ix) in enumerate(pix):
        s = C.conv3x3_at(xa, wa, None, 0, [(bb, iy, ix)], ch)[0]
        lim = 1.1 * 9 * c * 2.0 ** -23 * s + 2.0 ** -8 * np.abs(ref[k]) + 1e-30
        assert np.all(np.abs(got[k] - ref[k]) <= lim), (k, float((np.abs(got[k] - ref[k]) / lim).max()))
    assert np.isfinite(yh).all()


@pytest.mark.parametrize("cout", [64, 128, 256])
def test_bounded_waits_report_a_timeout_and_leave_the_device_usable(api, cout):
    # failure detection without a fault: the self-check launch never loads
    # the weights, every device-side wait runs out (20 ms), the kernel drains
    # its own copies, frees its tensor memory and reports the timeout
    x, wt, b, xo, wo, bo = bf16_inputs(9, 1, 20, 24, 128, cout)
    y = torch.full((1, 20, 24, cout), 7.0, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    api.fwi_conv3x3_bf16_wait_check(x, wt, y, status)
    torch.cuda.synchronize()
    assert int(status.item()) == api.FWI_ERR_DEVICE_TIMEOUT
    assert bool((y == 7.0).all())
    status.zero_()
    y2 = api.conv3x3(x, wt, b, 0, torch.float32, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = C.conv3x3(xo, wo, bo)
    assert np.all(np.abs(y2.double().cpu().numpy() - ref) <= bound(xo, wo, ref, 128, False, 0))
