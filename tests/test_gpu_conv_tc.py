"""The tensor-core (tcgen05) 3x3x3 convolution against the FP64 reference of
the network (oracle/warmnet_ref.py) and against the mma.sync layer.

Inputs and weights are BF16 values (exact in both), accumulation is FP32, so
the tensor-core result differs from the FP64 reference by accumulation
rounding only: bound 1e-3 of the output scale, as for the mma.sync layer;
the two GPU layers agree to FP32 summation order (1e-5 of the scale).  Every
case also checks that no block's bounded wait expired.
"""
import math

import numpy as np
import pytest

from oracle import warmnet_ref as R
from paper_1503_08718_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_08718_gb300 import build
    build.build()
    lbm.load()
    lbm.lbm_nn_tc_error(True)
    return t


def _bf16_round(a):
    import torch as T
    return T.from_numpy(np.asarray(a, np.float32)).to(T.bfloat16).to(T.float64).numpy()


def _case(cin, cout, vol, seed):
    rng = np.random.default_rng(seed)
    n, d, h, w = vol
    x = _bf16_round(rng.standard_normal((n, d, h, w, cin)))
    wt = _bf16_round(rng.standard_normal((cout, cin, 3, 3, 3)) / math.sqrt(cin * 27))
    b = rng.standard_normal(cout)
    return x, wt, b


def _dev(torch, x, wt, b):
    cout, cin = wt.shape[:2]
    dev = torch.device("cuda")
    xg = torch.from_numpy(x.reshape(-1, cin)).to(torch.bfloat16).to(dev)
    wg = torch.from_numpy(np.transpose(wt.reshape(cout, cin, 27), (2, 1, 0)).copy()).to(torch.bfloat16).to(dev)
    bg = torch.from_numpy(b.astype(np.float32)).to(dev)
    return xg, wg, bg


@pytest.mark.parametrize("cin,cout,vol", [
    (16, 32, (2, 4, 16, 8)), (32, 32, (1, 3, 32, 16)), (32, 64, (1, 5, 16, 24)),
    (64, 64, (2, 4, 16, 16)), (96, 32, (1, 4, 16, 8)), (64, 128, (1, 3, 16, 8)),
    (128, 128, (1, 2, 16, 8)), (192, 64, (1, 3, 32, 8)), (16, 256, (1, 2, 16, 8))])
def test_tc_conv_forward_matches_reference_and_mma_sync(torch, cin, cout, vol):
    n, d, h, w = vol
    assert lbm.lbm_nn_conv3d_tc_supported(cin, cout, n, d, h, w) == 1
    x, wt, b = _case(cin, cout, vol, 11 * cin + cout)
    ref = R.conv3_np(x, wt, b)
    xg, wg, bg = _dev(torch, x, wt, b)
    V = n * d * h * w
    wk = torch.empty((27, cout, cin), dtype=torch.bfloat16, device="cuda")
    assert lbm.lbm_nn_weights_kmajor(wg.data_ptr(), wk.data_ptr(), cin, cout, 0, None) == lbm.LBM_OK
    y = torch.empty((V, cout), dtype=torch.float32, device="cuda")
    st = lbm.lbm_nn_conv3d_tc(xg.data_ptr(), cin, wk.data_ptr(), bg.data_ptr(), y.data_ptr(), cout,
                              n, d, h, w, 0, 1, None)
    assert st == lbm.LBM_OK
    torch.cuda.synchronize()
    assert lbm.lbm_nn_tc_error(True) == 0
    got = y.cpu().numpy().reshape(ref.shape)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= 1e-3 * scale
    y2 = torch.empty((V, cout), dtype=torch.float32, device="cuda")
    assert lbm.lbm_nn_conv3d(xg.data_ptr(), cin, wg.data_ptr(), bg.data_ptr(), y2.data_ptr(), cout,
                             n, d, h, w, 3, 0, 1, None) == lbm.LBM_OK
    assert np.max(np.abs(y2.cpu().numpy().reshape(ref.shape) - got)) <= 1e-5 * scale
    # fused leaky ReLU with BF16 output
    yb = torch.empty((V, cout), dtype=torch.bfloat16, device="cuda")
    assert lbm.lbm_nn_conv3d_tc(xg.data_ptr(), cin, wk.data_ptr(), bg.data_ptr(), yb.data_ptr(), cout,
                                n, d, h, w, 1, 0, None) == lbm.LBM_OK
    leaky = np.where(ref > 0, ref, 0.01 * ref)
    assert np.max(np.abs(yb.float().cpu().numpy().reshape(ref.shape) - leaky)) <= 1e-2 * scale
    assert lbm.lbm_nn_tc_error(True) == 0


@pytest.mark.parametrize("cin,cout,tz", [(64, 64, 2), (32, 128, 1), (64, 32, 4)])
def test_tc_conv_persistent_blocks_walk_many_tiles(torch, cin, cout, tz):
    """Cells with far more tiles than SMs: every persistent block walks many
    tiles, both accumulator buffers and every ring stage wrap around several
    times.  Against the mma.sync layer (same BF16 operands, FP32
    accumulation: FP32 summation order apart) on every output, and against
    the FP64 reference on sampled voxels."""
    n, d, h, w = 2, 16, 64, 64
    rng = np.random.default_rng(7 * cin + cout + tz)
    x = _bf16_round(rng.standard_normal((n, d, h, w, cin)))
    wt = _bf16_round(rng.standard_normal((cout, cin, 3, 3, 3)) / math.sqrt(cin * 27))
    b = rng.standard_normal(cout)
    xg, wg, bg = _dev(torch, x, wt, b)
    V = n * d * h * w
    wk = torch.empty((27, cout, cin), dtype=torch.bfloat16, device="cuda")
    assert lbm.lbm_nn_weights_kmajor(wg.data_ptr(), wk.data_ptr(), cin, cout, 0, None) == lbm.LBM_OK
    y = torch.empty((V, cout), dtype=torch.float32, device="cuda")
    assert lbm.lbm_nn_conv3d_tc_cfg(xg.data_ptr(), cin, wk.data_ptr(), bg.data_ptr(), y.data_ptr(), cout,
                                    n, d, h, w, 1, 1, tz, 0, None) == lbm.LBM_OK
    y2 = torch.empty((V, cout), dtype=torch.float32, device="cuda")
    assert lbm.lbm_nn_conv3d(xg.data_ptr(), cin, wg.data_ptr(), bg.data_ptr(), y2.data_ptr(), cout,
                             n, d, h, w, 3, 1, 1, None) == lbm.LBM_OK
    torch.cuda.synchronize()
    assert lbm.lbm_nn_tc_error(True) == 0
    got = y.cpu().numpy().reshape(n, d, h, w, cout)
    other = y2.cpu().numpy().reshape(n, d, h, w, cout)
    scale = np.max(np.abs(other))
    assert np.max(np.abs(got - other)) <= 1e-5 * scale
    # sampled voxels against the FP64 definition (periodic in x, y; zero in z)
    for _ in range(64):
        c, z, yy, xx = (int(rng.integers(0, s)) for s in (n, d, h, w))
        acc = b.copy()
        for dz in (-1, 0, 1):
            if not 0 <= z + dz < d:
                continue
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    acc += wt[:, :, dz + 1, dy + 1, dx + 1] @ x[c, z + dz, (yy + dy) % h, (xx + dx) % w]
        leaky = np.where(acc > 0, acc, 0.01 * acc)
        assert np.max(np.abs(got[c, z, yy, xx] - leaky)) <= 1e-3 * scale


@pytest.mark.parametrize("tz,ns", [(1, 2), (1, 4), (2, 2), (2, 4), (4, 2), (4, 4)])
@pytest.mark.parametrize("cin,cout", [(64, 64), (32, 128), (128, 64)])
def test_tc_conv_every_launch_configuration(torch, cin, cout, tz, ns):
    """Every kernel variant (output planes per block x weight stages) against
    the FP64 reference."""
    vol = (1, 4, 16, 16)
    n, d, h, w = vol
    cols = 32
    while cols < cout:
        cols *= 2
    if tz * cols > 256:
        pytest.skip("the accumulators of this many planes exceed 256 tensor-memory columns")
    x, wt, b = _case(cin, cout, vol, 3 * tz + ns)
    ref = R.conv3_np(x, wt, b)
    xg, wg, bg = _dev(torch, x, wt, b)
    wk = torch.empty((27, cout, cin), dtype=torch.bfloat16, device="cuda")
    assert lbm.lbm_nn_weights_kmajor(wg.data_ptr(), wk.data_ptr(), cin, cout, 0, None) == lbm.LBM_OK
    y = torch.empty((n * d * h * w, cout), dtype=torch.float32, device="cuda")
    st = lbm.lbm_nn_conv3d_tc_cfg(xg.data_ptr(), cin, wk.data_ptr(), bg.data_ptr(), y.data_ptr(), cout,
                                  n, d, h, w, 0, 1, tz, ns, None)
    assert st == lbm.LBM_OK
    torch.cuda.synchronize()
    assert lbm.lbm_nn_tc_error(True) == 0
    got = y.cpu().numpy().reshape(ref.shape)
    assert np.max(np.abs(got - ref)) <= 1e-3 * np.max(np.abs(ref))


@pytest.mark.parametrize("cin,cout", [(32, 64), (64, 32)])
def test_tc_data_gradient_weights(torch, cin, cout):
    """With the flipped K-major weights the tensor-core conv of the output
    gradient is the data gradient, as the mma.sync layer computes it from
    lbm_nn_flip_weights."""
    vol = (1, 4, 16, 16)
    n, d, h, w = vol
    x, wt, b = _case(cin, cout, vol, 5)
    g = _bf16_round(np.random.default_rng(6).standard_normal((n, d, h, w, cout)))
    _, wg, _ = _dev(torch, x, wt, b)
    gg = torch.from_numpy(g.reshape(-1, cout)).to(torch.bfloat16).to("cuda")
    V = n * d * h * w
    wf = torch.empty((27, cout, cin), dtype=torch.bfloat16, device="cuda")
    lbm.lbm_nn_flip_weights(wg.data_ptr(), wf.data_ptr(), cin, cout, 3, None)
    dx_ref = torch.empty((V, cin), dtype=torch.float32, device="cuda")
    lbm.lbm_nn_conv3d(gg.data_ptr(), cout, wf.data_ptr(), None, dx_ref.data_ptr(), cin, n, d, h, w, 3, 0, 1,
                      None)
    wkf = torch.empty((27, cin, cout), dtype=torch.bfloat16, device="cuda")
    assert lbm.lbm_nn_weights_kmajor(wg.data_ptr(), wkf.data_ptr(), cin, cout, 1, None) == lbm.LBM_OK
    dx = torch.empty((V, cin), dtype=torch.float32, device="cuda")
    assert lbm.lbm_nn_conv3d_tc(gg.data_ptr(), cout, wkf.data_ptr(), None, dx.data_ptr(), cin,
                                n, d, h, w, 0, 1, None) == lbm.LBM_OK
    a, r = dx.cpu().numpy(), dx_ref.cpu().numpy()
    assert np.max(np.abs(a - r)) <= 1e-5 * np.max(np.abs(r))
    assert lbm.lbm_nn_tc_error(True) == 0


def test_tc_conv_rejects_unsupported_sizes(torch):
    assert lbm.lbm_nn_conv3d_tc_supported(16, 32, 1, 4, 12, 8) == 0     # h not a multiple of 16
    assert lbm.lbm_nn_conv3d_tc_supported(16, 32, 1, 4, 16, 12) == 0    # w not a multiple of 8
    assert lbm.lbm_nn_conv3d_tc_supported(8, 32, 1, 4, 16, 8) == 0      # cin below 16
    assert lbm.lbm_nn_conv3d_tc_supported(16, 264, 1, 4, 16, 8) == 0    # cout above 256
    st = lbm.lbm_nn_conv3d_tc(1, 16, 1, None, 1, 32, 1, 4, 12, 8, 0, 0, None)
    assert st == lbm.LBM_ERR_INVALID_ARG


def test_network_on_tensor_cores_matches_mma_sync(torch):
    """The whole warm-start network with its 3x3x3 convolutions and data
    gradients on the tcgen05 kernel (where the 16 x 8 tiles fit) against the
    same network on the mma.sync kernel: the BF16 activations may round
    differently after FP32 sums in another order, so the prediction is held
    to 1e-3 of its scale and the gradients by direction (cosine >= 0.999)."""
    from paper_1503_08718_gb300 import inputs as I
    from paper_1503_08718_gb300.warmstart import WarmNet
    rng = np.random.default_rng(4)
    n, d, h, w = 2, 16, 32, 32
    phases = rng.integers(0, 3, size=(n, d, h, w), dtype=np.uint8)
    lams = [np.stack([I.random_spd(rng) for _ in range(3)]) for _ in range(n)]
    target = rng.uniform(0, 1, size=(n, d, h, w)).astype(np.float32)
    out = []
    for use_tc in (True, False):
        net = WarmNet(seed=3, use_tc=use_tc)
        x0, tl = net.make_input(phases, lams)
        tgt = torch.from_numpy(target.reshape(-1)).to(net.dev)
        pred, loss = net.forward(x0, (n, d, h, w), tl, tgt)
        net.backward()
        torch.cuda.synchronize()
        out.append((pred.cpu().numpy(), float(loss.item()),
                    np.concatenate([g.cpu().numpy().ravel() for g in net.gW])))
    assert lbm.lbm_nn_tc_error(True) == 0
    (p1, l1, g1), (p0, l0, g0) = out
    assert np.max(np.abs(p1 - p0)) <= 1e-3 * max(1.0, float(np.max(np.abs(p0))))
    assert l1 == pytest.approx(l0, rel=1e-2)
    cos = float(g1 @ g0 / (np.linalg.norm(g1) * np.linalg.norm(g0)))
    assert cos >= 0.999, cos


@pytest.mark.parametrize("cin,cout,vol", [(16, 32, (1, 3, 16, 8)), (32, 64, (2, 2, 16, 16)),
                                          (64, 64, (1, 4, 32, 8)), (96, 32, (1, 2, 16, 8)),
                                          (128, 128, (1, 2, 16, 16)), (192, 64, (1, 2, 16, 8)),
                                          (32, 40, (1, 2, 16, 24)), (16, 8, (1, 3, 16, 8))])
def test_tc_weight_gradient_matches_reference(torch, cin, cout, vol):
    """dW of the tensor-core kernel (both operands MN-major, accumulators in
    tensor memory; with cout <= 64 the M = 128 rows hold two or three
    x-shifted copies of the output gradient, so that one MMA gives two or
    three taps) against reverse-mode differentiation of the FP64 reference
    conv; FP32 accumulation, bound 1e-4 of the scale as for the mma.sync
    weight gradient."""
    import torch as T
    n, d, h, w = vol
    assert lbm.lbm_nn_conv3d_wgrad_tc_supported(cin, cout, n, d, h, w) == 1
    rng = np.random.default_rng(7 * cin + cout)
    x = _bf16_round(rng.standard_normal((n, d, h, w, cin)))
    g = _bf16_round(rng.standard_normal((n, d, h, w, cout)))
    W = T.zeros((cout, cin, 3, 3, 3), dtype=T.float64, requires_grad=True)
    y = R.conv3(T.from_numpy(np.moveaxis(x, -1, 1)), W, None)
    (y * T.from_numpy(np.moveaxis(g, -1, 1))).sum().backward()
    ref = np.transpose(W.grad.numpy().reshape(cout, cin, 27), (2, 1, 0))
    xg = torch.from_numpy(x.reshape(-1, cin)).to(torch.bfloat16).to("cuda")
    gg = torch.from_numpy(g.reshape(-1, cout)).to(torch.bfloat16).to("cuda")
    dw = torch.zeros((27, cin, cout), dtype=torch.float32, device="cuda")
    assert lbm.lbm_nn_conv3d_wgrad_tc(xg.data_ptr(), cin, gg.data_ptr(), cout, dw.data_ptr(),
                                      n, d, h, w, None) == lbm.LBM_OK
    torch.cuda.synchronize()
    assert lbm.lbm_nn_tc_error(True) == 0
    assert np.max(np.abs(dw.cpu().numpy() - ref)) <= 1e-4 * np.max(np.abs(ref))
