"""Surrogate kernels (GPU, through the C-ABI) against the FP64 reference.

Inputs are rounded to BF16 first and the reference gets the rounded values,
so the comparison measures the kernels' own error: FP32 accumulation and a
BF16-rounded output, relative error <= 1e-2 of the output's scale.  Channel
slices (a stride wider than the channel count, an offset first channel) are
exercised on purpose, as the decoder's concatenation buffers use them.
"""

import math

import numpy as np
import pytest

from oracle import surrogate_ref as R
from paper_1908_08386_gb300 import surrogate as S
from paper_1908_08386_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def bf(a):
    """Host array -> device BF16 tensor, and the rounded values back in FP64."""
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().to(torch.bfloat16)
    return t, t.to(torch.float64).cpu().numpy()


def f64(t):
    return t.to(torch.float64).cpu().numpy()


def rel(got, want):
    return np.abs(got - want).max() / max(np.abs(want).max(), 1e-30)


def sync():
    torch.cuda.synchronize()


@pytest.mark.parametrize("mode", [S.LINEAR, S.LEAKY, S.DLEAKY])
def test_conv3x3_matches_the_reference(mode):
    rng = np.random.default_rng(1)
    B, H, W, cin, cout = 2, 16, 32, 48, 64
    wide, xw = bf(rng.standard_normal((B, H, W, cin + 16)))  # x = channels 16.. of a wider tensor
    w, wr = bf(rng.standard_normal((cout, 9, cin)) / math.sqrt(9 * cin))
    bias = torch.from_numpy(rng.standard_normal(cout).astype(np.float32)).cuda()
    m, mr = bf(rng.standard_normal((B, H, W, cout)))
    y = torch.zeros(B, H, W, cout + 32, dtype=torch.bfloat16, device="cuda")  # y = channels 32..
    S.conv3x3(S.View(wide, 16), w.data_ptr(), bias.data_ptr(), S.View(y, 32), B, H, W, cin, cout, mode,
              S.View(m) if mode == S.DLEAKY else None)
    sync()
    ref = R.conv3x3(xw[..., 16:], wr.reshape(cout, 3, 3, cin), 0.0 if mode == S.DLEAKY else f64(bias))
    if mode == S.LEAKY:
        ref = R.leaky(ref)
    if mode == S.DLEAKY:
        ref = R.leaky_backward(mr, ref)
    got = f64(y)
    assert rel(got[..., 32:], ref) <= 1e-2
    assert np.all(got[..., :32] == 0.0)  # nothing outside the slice


# a block takes up to four 128-position tiles, each with its own
# tensor-memory accumulator (two at 160 and 256 output channels): full blocks,
# a last block with fewer tiles (W = 128: nine tiles per image), images of
# fewer tiles than a block holds
@pytest.mark.parametrize("B,H,W,cin,cout", [(3, 8, 16, 16, 32), (1, 8, 128, 32, 32), (2, 16, 16, 160, 160),
                                             (1, 8, 32, 256, 96), (1, 8, 64, 96, 256), (2, 24, 48, 64, 64),
                                             (18, 128, 128, 16, 32), (32, 64, 64, 32, 64), (64, 32, 32, 32, 96),
                                             (32, 32, 32, 256, 96)])
def test_tensor_core_conv3x3_covers_the_network_shapes(B, H, W, cin, cout):
    """The tcgen05 convolution on the widths, depths and image sizes of the
    network (tiles of 128 padded positions that cross image rows and, for
    W = 16, several rows; the adjoint's 256 output channels; a 16-channel
    input; blocks of several tiles), each output element against the FP64
    reference; the status word of the bounded waits stays clear."""
    rng = np.random.default_rng(B * 1000 + W + cin + cout)
    x, xr = bf(rng.standard_normal((B, H, W, cin)))
    w, wr = bf(rng.standard_normal((cout, 9, cin)) / math.sqrt(9 * cin))
    bias = torch.from_numpy(rng.standard_normal(cout).astype(np.float32)).cuda()
    y = torch.full((B, H, W, cout), float("nan"), dtype=torch.bfloat16, device="cuda")
    S.conv3x3(S.View(x), w.data_ptr(), bias.data_ptr(), S.View(y), B, H, W, cin, cout, S.LEAKY)
    S.check()
    ref = R.leaky(R.conv3x3(xr, wr.reshape(cout, 3, 3, cin), f64(bias)))
    got = f64(y)
    assert np.isfinite(got).all()  # every output position written
    assert rel(got, ref) <= 1e-2


def test_adjoint_and_weight_gradient_match_the_reference():
    rng = np.random.default_rng(2)
    B, H, W, cin, cout = 2, 16, 32, 32, 64
    x, xr = bf(rng.standard_normal((B, H, W, cin)))
    w, wr = bf(rng.standard_normal((cout, 9, cin)) / math.sqrt(9 * cin))
    dy, dyr = bf(rng.standard_normal((B, H, W, cout)))
    wt = torch.zeros(cin * 9 * cout, dtype=torch.bfloat16, device="cuda")
    S.call("lbmfvm_sg_flip", w.data_ptr(), wt.data_ptr(), cin, cout, S._stream())
    dx = torch.zeros(B, H, W, cin, dtype=torch.bfloat16, device="cuda")
    S.conv3x3(S.View(dy), wt.data_ptr(), None, S.View(dx), B, H, W, cout, cin, S.LINEAR)
    dw = torch.zeros(cout * 9 * cin, dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    S.call("lbmfvm_sg_conv3x3_wgrad", x.data_ptr(), cin, dy.data_ptr(), cout, dw.data_ptr(), db.data_ptr(), B, H, W,
           cin, cout, S._stream())
    sync()
    rdx, rdw, rdb = R.conv3x3_backward(xr, wr.reshape(cout, 3, 3, cin), dyr)
    assert rel(f64(dx), rdx) <= 1e-2
    assert rel(f64(dw).reshape(cout, 3, 3, cin), rdw) <= 1e-4  # FP32 sums of exact BF16 products
    assert rel(f64(db), rdb) <= 1e-4


def test_pooling_and_upsampling_match_the_reference():
    rng = np.random.default_rng(3)
    B, H, W, C = 2, 16, 32, 32
    x, xr = bf(rng.standard_normal((B, H, W, C)))
    y = torch.zeros(B, H // 2, W // 2, C, dtype=torch.bfloat16, device="cuda")
    S.call("lbmfvm_sg_pool2", x.data_ptr(), C, y.data_ptr(), C, B, H, W, C, S._stream())
    dy, dyr = bf(rng.standard_normal((B, H // 2, W // 2, C)))
    add, addr = bf(rng.standard_normal((B, H, W, C)))
    m, mr = bf(rng.standard_normal((B, H, W, C)))
    dx = torch.zeros(B, H, W, C, dtype=torch.bfloat16, device="cuda")
    S.call("lbmfvm_sg_pool2_backward", dy.data_ptr(), C, add.data_ptr(), C, m.data_ptr(), C, dx.data_ptr(), C, B, H, W,
           C, S._stream())
    up = torch.zeros(B, H, W, C, dtype=torch.bfloat16, device="cuda")
    S.call("lbmfvm_sg_upsample2", dy.data_ptr(), C, up.data_ptr(), C, B, H // 2, W // 2, C, S._stream())
    dup = torch.zeros(B, H // 2, W // 2, C, dtype=torch.bfloat16, device="cuda")
    mc, mcr = bf(rng.standard_normal((B, H // 2, W // 2, C)))
    S.call("lbmfvm_sg_upsample2_backward", add.data_ptr(), C, mc.data_ptr(), C, dup.data_ptr(), C, B, H // 2, W // 2, C,
           S._stream())
    sync()
    assert rel(f64(y), R.avgpool2(xr)) <= 1e-2
    assert rel(f64(dx), R.leaky_backward(mr, R.avgpool2_backward(dyr) + addr)) <= 1e-2
    assert np.array_equal(f64(up), R.upsample2(dyr))
    assert rel(f64(dup), R.leaky_backward(mcr, R.upsample2_backward(addr))) <= 1e-2


def test_output_layer_loss_and_adam_match_the_reference():
    rng = np.random.default_rng(4)
    B, H, W, C = 2, 16, 16, 32
    P = B * H * W
    x, xr = bf(np.abs(rng.standard_normal((B, H, W, C))) * np.sign(rng.standard_normal((B, H, W, C))))
    w = torch.from_numpy(rng.standard_normal((3, C)).astype(np.float32)).cuda()
    b = torch.from_numpy(rng.standard_normal(3).astype(np.float32)).cuda()
    y = torch.zeros(B, H, W, 3, dtype=torch.float32, device="cuda")
    S.call("lbmfvm_sg_conv1x1", x.data_ptr(), C, w.data_ptr(), b.data_ptr(), y.data_ptr(), P, C, 3, S._stream())
    target = torch.from_numpy(rng.standard_normal((B, H, W, 3)).astype(np.float32)).cuda()
    fluid_np = (rng.random((B, H, W)) > 0.25).astype(np.uint8)
    fluid = torch.from_numpy(fluid_np).cuda()
    dpred = torch.zeros_like(y)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    n = int(fluid_np.sum())
    S.call("lbmfvm_sg_mse", y.data_ptr(), target.data_ptr(), fluid.data_ptr(), P, 3, 1.0 / (3 * n), dpred.data_ptr(),
           loss.data_ptr(), S._stream())
    dx = torch.zeros(B, H, W, C, dtype=torch.bfloat16, device="cuda")
    dw = torch.zeros(3, C, dtype=torch.float32, device="cuda")
    db = torch.zeros(3, dtype=torch.float32, device="cuda")
    S.call("lbmfvm_sg_conv1x1_backward", x.data_ptr(), C, w.data_ptr(), dpred.data_ptr(), dx.data_ptr(), C,
           dw.data_ptr(), db.data_ptr(), P, C, 3, S._stream())
    sync()
    ref_y = R.conv1x1(xr, f64(w), f64(b))
    assert rel(f64(y), ref_y) <= 1e-5
    ref_loss, ref_d = R.masked_mse(f64(y), f64(target), fluid_np)
    assert loss.item() == pytest.approx(ref_loss, rel=1e-6)
    assert rel(f64(dpred), ref_d) <= 1e-6
    rdx, rdw, rdb = R.conv1x1_backward(xr, f64(w), f64(dpred))
    assert rel(f64(dx), R.leaky_backward(xr, rdx)) <= 1e-2
    assert rel(f64(dw), rdw) <= 1e-5 and rel(f64(db), rdb) <= 1e-5
    # Adam, three steps
    p0 = rng.standard_normal(1000)
    p = torch.from_numpy(p0.astype(np.float32)).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    pb = torch.zeros(1000, dtype=torch.bfloat16, device="cuda")
    rp, rm, rv = p0.astype(np.float32).astype(np.float64), np.zeros(1000), np.zeros(1000)
    for t in (1, 2, 3):
        g = rng.standard_normal(1000)
        gt = torch.from_numpy(g.astype(np.float32)).cuda()
        S.call("lbmfvm_sg_adam", p.data_ptr(), gt.data_ptr(), m.data_ptr(), v.data_ptr(), pb.data_ptr(), 1000, 1e-2,
               0.9, 0.999, 1e-8, t, S._stream())
        rp, rm, rv = R.adam_step(rp, g.astype(np.float32).astype(np.float64), rm, rv, t, 1e-2)
    sync()
    assert np.abs(f64(p) - rp).max() <= 1e-5
    assert np.array_equal(f64(pb), f64(p.to(torch.bfloat16)))


def test_network_forward_and_backward_match_the_reference():
    widths, B, H = (32, 64), 2, 32
    params = WL.surrogate_init(widths, seed=7)
    net = S.Surrogate(widths, params=params)
    rng = np.random.default_rng(8)
    masks_np = (rng.random((B, H, H)) > 0.8).astype(np.uint8)
    scal_np = rng.uniform(-1, 1, (B, 2)).astype(np.float32)
    net.encode(torch.from_numpy(masks_np).cuda(), torch.from_numpy(scal_np).cuda(), B, H)
    pred = net.forward(B, H)
    target_np = rng.standard_normal((B, H, H, 3)).astype(np.float32)
    fluid_np = (1 - masks_np).astype(np.uint8)
    net.loss(B, H, torch.from_numpy(target_np).cuda(), torch.from_numpy(fluid_np).cuda(), int(fluid_np.sum()))
    net.backward(B, H)
    sync()
    # the reference with the network's own BF16-rounded 3x3 weights and input
    rparams = [p.copy() for p in params]
    for i in range(0, len(rparams) - 2, 2):
        rparams[i] = torch.from_numpy(rparams[i].astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    x = f64(net.buffers(B, H)["x"])[..., :3]
    out, acts = R.forward(rparams, x, widths)
    _, dout = R.masked_mse(out, target_np.astype(np.float64), fluid_np)
    grads, _ = R.backward(rparams, acts, dout, widths)
    assert rel(f64(pred), out) <= 3e-2
    flat = f64(net.g)
    errs = []
    for i, ((kind, creal, cin, cout), (w0, b0)) in enumerate(zip(net.layers, net.offsets)):
        if kind == "c3":
            gw = flat[w0:b0].reshape(cout, 9, cin)[:, :, :creal].reshape(cout, 3, 3, creal)
        else:
            gw = flat[w0:b0].reshape(cout, cin)
        gb = flat[b0:b0 + cout]
        for got, want in ((gw, grads[2 * i]), (gb, grads[2 * i + 1])):
            err = np.linalg.norm(got - want) / np.linalg.norm(want)
            cos = np.sum(got * want) / (np.linalg.norm(got) * np.linalg.norm(want))
            errs.append((i, kind, round(float(err), 4), round(float(cos), 5)))
    print(errs)
    # BF16 activations round at every layer (and flip the leaky ReLU's slope
    # where a pre-activation is near zero), so gradients of the BF16 layers
    # sit a few per cent from the FP64 recomputation, in the same direction;
    # a wrong or missing term would turn their direction.  The FP32 output
    # layer, fed by the last activation only, is held tighter.
    assert all(c >= 0.995 and e <= 0.1 for _, k, e, c in errs if k == "c3"), errs
    assert all(e <= 1e-2 for _, k, e, _ in errs if k == "c1"), errs


def test_training_reduces_the_loss():
    widths, B, H = (32, 64), 4, 32
    net = S.Surrogate(widths, seed=1)
    rng = np.random.default_rng(9)
    masks = torch.from_numpy((rng.random((B, H, H)) > 0.9).astype(np.uint8)).cuda()
    scal = torch.from_numpy(rng.uniform(-1, 1, (B, 2)).astype(np.float32)).cuda()
    yy, xx = np.meshgrid(np.linspace(0, 1, H), np.linspace(0, 1, H), indexing="ij")
    target_np = np.stack([np.sin(np.pi * xx) * yy, xx * (1 - xx), 1 - xx], -1)[None].repeat(B, 0).astype(np.float32)
    target = torch.from_numpy(target_np).cuda()
    fluid = 1 - masks
    n = int(fluid.sum().item())
    net.encode(masks, scal, B, H)
    losses = []
    for it in range(60):
        bufs = net.buffers(B, H)
        bufs["loss"].zero_()
        net.forward(B, H)
        net.loss(B, H, target, fluid, n)
        net.backward(B, H)
        net.adam(2e-3)
        losses.append(bufs["loss"].item())
    assert losses[-1] < 0.2 * losses[0], losses[::10]


def test_encode_and_resampling_follow_their_definitions():
    rng = np.random.default_rng(10)
    net_in = torch.zeros(1, 32, 32, 16, dtype=torch.bfloat16, device="cuda")
    mask_np = (rng.random((1, 32, 32)) > 0.5).astype(np.uint8)
    mask_d = torch.from_numpy(mask_np).cuda()
    scal_d = torch.tensor([0.25, -0.5], device="cuda")
    S.call("lbmfvm_sg_encode", mask_d.data_ptr(), scal_d.data_ptr(), net_in.data_ptr(), 1, 32, 32, S._stream())
    nx, ny = 97, 49
    big = (rng.random((ny, nx)) > 0.7).astype(np.uint8)
    small = torch.zeros(16, 16, dtype=torch.uint8, device="cuda")
    bigt = torch.from_numpy(big).cuda()
    S.call("lbmfvm_sg_resample_mask", bigt.data_ptr(), nx, ny, small.data_ptr(), 16, 16, S._stream())
    pred_np = rng.standard_normal((16, 16, 3)).astype(np.float32)
    pred = torch.from_numpy(pred_np).cuda()
    u, v, T = (torch.zeros(ny, nx, dtype=torch.float32, device="cuda") for _ in range(3))
    S.call("lbmfvm_sg_resample_fields", pred.data_ptr(), 16, 16, bigt.data_ptr(), nx, ny, 0.05, u.data_ptr(),
           v.data_ptr(), T.data_ptr(), S._stream())
    sync()
    x = f64(net_in)
    assert np.array_equal(x[0, :, :, 0], mask_np[0].astype(np.float64))
    assert np.all(x[0, :, :, 1] == 0.25) and np.all(x[0, :, :, 2] == -0.5) and np.all(x[0, :, :, 3:] == 0)
    sy = np.minimum(((np.arange(16) + 0.5) * ny / 16).astype(int), ny - 1)
    sx = np.minimum(((np.arange(16) + 0.5) * nx / 16).astype(int), nx - 1)
    assert np.array_equal(small.cpu().numpy(), big[sy][:, sx])
    # bilinear interpolation at one interior fluid node, by hand
    j, i = 20, 41
    fx = min(max((i + 0.5) * 16 / nx - 0.5, 0), 15)
    fy = min(max((j + 0.5) * 16 / ny - 0.5, 0), 15)
    x0, y0 = int(fx), int(fy)
    ax, ay = fx - x0, fy - y0
    val = (1 - ay) * ((1 - ax) * pred_np[y0, x0] + ax * pred_np[y0, x0 + 1]) + \
        ay * ((1 - ax) * pred_np[y0 + 1, x0] + ax * pred_np[y0 + 1, x0 + 1])
    un, vn, Tn = f64(u), f64(v), f64(T)
    if not big[j, i]:
        assert un[j, i] == pytest.approx(0.05 * val[0], rel=1e-5, abs=1e-7)
        assert vn[j, i] == pytest.approx(0.05 * val[1], rel=1e-5, abs=1e-7)
    assert Tn[j, i] == pytest.approx(min(max(val[2], 0.0), 1.0), rel=1e-5, abs=1e-7)
    assert np.all(un[big == 1] == 0) and np.all(un[0, :] == 0) and np.all(un[:, -1] == 0)
    assert Tn.min() >= 0.0 and Tn.max() <= 1.0


def test_convolution_waits_give_up_and_report_without_a_fault():
    """A staged load that never comes (injected on the host: block 0 skips
    it) makes the convolution's bounded waits run out: the status word
    reports it (-4), nothing faults, and the next convolution on the same
    context is correct."""
    rng = np.random.default_rng(9)
    B, H, W, cin, cout = 2, 16, 32, 32, 64
    x, xr = bf(rng.standard_normal((B, H, W, cin)))
    w, wr = bf(rng.standard_normal((cout, 9, cin)) / math.sqrt(9 * cin))
    y = torch.zeros(B, H, W, cout, dtype=torch.bfloat16, device="cuda")
    S.check()
    S.call("lbmfvm_sg_inject_stall")
    S.conv3x3(S.View(x), w.data_ptr(), None, S.View(y), B, H, W, cin, cout, S.LINEAR)
    with pytest.raises(S.LbmfvmError) as e:
        S.check()
    assert e.value.code == -4
    S.check()  # the word was cleared
    S.conv3x3(S.View(x), w.data_ptr(), None, S.View(y), B, H, W, cin, cout, S.LINEAR)
    S.check()
    ref = R.conv3x3(xr, wr.reshape(cout, 3, 3, cin), 0.0)
    assert rel(f64(y), ref) <= 1e-2
