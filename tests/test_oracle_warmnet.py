"""Pins of the FP64 network reference (oracle/warmnet_ref.py) to something
other than itself: its 3x3x3 convolution against the definition written out
as loops (circular padding in x and y, zero padding in z, cross-correlation
with bias), its pooling and upsampling against their definitions, and the
whole network's reverse-mode gradients against central finite differences."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import warmnet_ref as R  # noqa: E402


def _conv3_loops(x, w, b):
    """y[n,o,z,y,x] = b[o] + sum_{c,dz,dy,dx} w[o,c,dz,dy,dx] x[n,c,z+dz-1,(y+dy-1)%H,(x+dx-1)%W],
    with x = 0 outside 0 <= z < D."""
    N, C, D, H, W = x.shape
    O = w.shape[0]
    y = np.zeros((N, O, D, H, W))
    for n in range(N):
        for o in range(O):
            for z in range(D):
                for yy in range(H):
                    for xx in range(W):
                        acc = b[o]
                        for dz in range(3):
                            zz = z + dz - 1
                            if zz < 0 or zz >= D:
                                continue
                            for dy in range(3):
                                for dx in range(3):
                                    acc += np.dot(w[o, :, dz, dy, dx],
                                                  x[n, :, zz, (yy + dy - 1) % H, (xx + dx - 1) % W])
                        y[n, o, z, yy, xx] = acc
    return y


def test_conv3_is_the_written_definition():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 2, 3, 4, 5))
    w = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    got = R.conv3(torch.from_numpy(x), torch.from_numpy(w), torch.from_numpy(b)).numpy()
    assert np.max(np.abs(got - _conv3_loops(x, w, b))) < 1e-12
    # the channels-last helper is the same layer
    got_nl = R.conv3_np(np.moveaxis(x, 1, -1), w, b)
    assert np.max(np.abs(np.moveaxis(got_nl, -1, 1) - got)) < 1e-12


def test_pool_and_upsample_are_block_mean_and_nearest():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 2, 4, 6, 8))
    pooled = torch.nn.functional.avg_pool3d(torch.from_numpy(x), 2).numpy()
    blocks = x.reshape(1, 2, 2, 2, 3, 2, 4, 2).mean(axis=(3, 5, 7))
    assert np.max(np.abs(pooled - blocks)) < 1e-15
    up = torch.nn.functional.interpolate(torch.from_numpy(pooled), scale_factor=2, mode="nearest").numpy()
    rep = pooled.repeat(2, axis=2).repeat(2, axis=3).repeat(2, axis=4)
    assert np.array_equal(up, rep)


def test_network_gradients_match_finite_differences():
    """A two-level network (channels 32, 16) on a 4^3 cell: the reverse-mode
    gradient of the loss equals central differences for weights and biases
    of every layer (FP64, step 1e-6)."""
    chans = (32, 16)
    rng = np.random.default_rng(2)
    params = R.init_params(seed=3, chans=chans)
    params = [(w, 0.1 * rng.standard_normal(b.shape)) for w, b in params]
    x = rng.standard_normal((1, 7, 4, 4, 4))
    t_lin = np.broadcast_to(np.linspace(0.9, 0.1, 4)[None, None, :, None, None], (1, 1, 4, 4, 4)).copy()
    target = rng.uniform(0, 1, (1, 1, 4, 4, 4))
    loss, grads = R.loss_and_grads(params, x, t_lin, target, chans)

    def loss_at(p):
        return R.loss_and_grads(p, x, t_lin, target, chans)[0]

    h = 1e-6
    for layer in range(len(params)):
        w, b = params[layer]
        for kind, arr, g in (("w", w, grads[layer][0]), ("b", b, grads[layer][1])):
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            plus = [(ww.copy(), bb.copy()) for ww, bb in params]
            minus = [(ww.copy(), bb.copy()) for ww, bb in params]
            (plus[layer][0] if kind == "w" else plus[layer][1])[idx] += h
            (minus[layer][0] if kind == "w" else minus[layer][1])[idx] -= h
            fd = (loss_at(plus) - loss_at(minus)) / (2 * h)
            assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), (layer, kind, idx)
    assert loss > 0
