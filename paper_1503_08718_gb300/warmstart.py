"""Learned warm start for the steady lattice Boltzmann solve.

A small 3D convolutional encoder-decoder predicts a cell's steady temperature
from its material field (6 tensor components and the linear profile between
the walls, temperature difference along z); the solve then starts from the
equilibrium of that field instead of the linear profile.  The converged
lattice Boltzmann result is unchanged (the iteration has one fixed point),
only the number of iterations to reach it changes.

Every layer runs in the library's CUDA kernels (lbm_nn_*: BF16 implicit-GEMM
convolutions on the tensor cores, FP32 accumulation); this module only
allocates buffers (torch), sequences the layer calls and keeps the optimiser
state.  Training targets come from the library's own solver.

Architecture (weights [taps][cin][cout], activations channels-last):
  conv3 16(7)->32, conv3 32->32 = s1 | pool | conv3 32->64, conv3 64->64 = s2 |
  pool | conv3 64->128, conv3 128->128 | up, cat s2 | conv3 192->64,
  conv3 64->64 | up, cat s1 | conv3 96->32 | conv1 32->1 head: T = T_lin + out
"""
from __future__ import annotations

import math

import numpy as np

from . import inputs as I
from . import lbm

CONV3 = [(16, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (192, 64), (64, 64),
         (96, 32)]
IN_CHANNELS = 7           # 6 tensor components + linear profile (padded to 16)
HEAD_C = 32


def _torch():
    import torch
    return torch


def material_table(lam: np.ndarray) -> np.ndarray:
    """Per-phase network features: the six tensor components divided by the
    cell's largest diagonal conductivity."""
    lam = np.asarray(lam, dtype=np.float64).reshape(-1, 6)
    return (lam / lam[:, :3].max()).astype(np.float32)


def linear_profile(d: int, t_hot: float = 1.0, t_cold: float = 0.0) -> np.ndarray:
    z = np.arange(d, dtype=np.float64)
    return (t_hot + (t_cold - t_hot) * (z + 0.5) / d).astype(np.float32)


class WarmNet:
    """Parameters and optimiser state on the GPU; forward and backward passes
    over a batch of n cells of d x h x w (all multiples of 4)."""

    def __init__(self, seed: int = 0, device: int = 0):
        torch = _torch()
        self.torch = torch
        self.dev = torch.device("cuda", device)
        g = np.random.default_rng(seed)
        self.W, self.Wb, self.b = [], [], []
        for cin, cout in CONV3:
            fan_in = 27 * (IN_CHANNELS if cin == 16 else cin)
            w = np.zeros((27, cin, cout), np.float32)
            live = IN_CHANNELS if cin == 16 else cin
            w[:, :live, :] = g.standard_normal((27, live, cout)) * math.sqrt(2.0 / fan_in)
            self.W.append(torch.from_numpy(w).to(self.dev))
            self.b.append(torch.zeros(cout, dtype=torch.float32, device=self.dev))
        self.hw = torch.from_numpy((g.standard_normal(HEAD_C) * math.sqrt(1.0 / HEAD_C) * 0.1)
                                   .astype(np.float32)).to(self.dev)
        self.hb = torch.zeros(1, dtype=torch.float32, device=self.dev)
        self._sync_bf16()
        self.params = self.W + self.b + [self.hw, self.hb]
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.t = 0

    # ---- parameters ----------------------------------------------------
    def _sync_bf16(self):
        torch = self.torch
        self.Wb = [w.to(torch.bfloat16).contiguous() for w in self.W]

    def set_reference_params(self, params):
        """Loads weights given as [(w [cout, cin, 3, 3, 3], b), ..., head]."""
        torch = self.torch
        for l, (w, b) in enumerate(params[: len(CONV3)]):
            cin_pad, cout = CONV3[l]
            wt = np.zeros((27, cin_pad, cout), np.float32)
            wt[:, : w.shape[1], :] = np.transpose(np.asarray(w).reshape(cout, w.shape[1], 27), (2, 1, 0))
            self.W[l].copy_(torch.from_numpy(wt))
            self.b[l].copy_(torch.from_numpy(np.asarray(b, np.float32)))
        hw, hb = params[-1]
        self.hw.copy_(torch.from_numpy(np.asarray(hw, np.float32).reshape(-1)))
        self.hb.copy_(torch.from_numpy(np.asarray(hb, np.float32).reshape(-1)))
        self._sync_bf16()

    def save(self, path: str):
        arrs = {f"W{l}": w.cpu().numpy() for l, w in enumerate(self.W)}
        arrs.update({f"b{l}": b.cpu().numpy() for l, b in enumerate(self.b)})
        arrs["hw"] = self.hw.cpu().numpy()
        arrs["hb"] = self.hb.cpu().numpy()
        np.savez(path, **arrs)

    def load(self, path: str):
        torch = self.torch
        z = np.load(path)
        for l in range(len(CONV3)):
            self.W[l].copy_(torch.from_numpy(z[f"W{l}"]))
            self.b[l].copy_(torch.from_numpy(z[f"b{l}"]))
        self.hw.copy_(torch.from_numpy(z["hw"]))
        self.hb.copy_(torch.from_numpy(z["hb"]))
        self._sync_bf16()

    # ---- passes --------------------------------------------------------
    def _stream(self):
        return self.torch.cuda.current_stream(self.dev).cuda_stream

    @staticmethod
    def _ok(st, what):
        if st != lbm.LBM_OK:
            raise lbm.LBMError(st, what)

    def _conv(self, l, x, vol, relu=True):
        torch = self.torch
        n, d, h, w = vol
        cin, cout = CONV3[l]
        y = torch.empty((n * d * h * w, cout), dtype=torch.bfloat16, device=self.dev)
        self._ok(lbm.lbm_nn_conv3d(x.data_ptr(), cin, self.Wb[l].data_ptr(), self.b[l].data_ptr(),
                                   y.data_ptr(), cout, n, d, h, w, 3, int(relu), 0, self._stream()),
                 f"conv layer {l}")
        return y

    def _pool(self, x, c, vol):
        torch = self.torch
        n, d, h, w = vol
        y = torch.empty((n * d * h * w // 8, c), dtype=torch.bfloat16, device=self.dev)
        self._ok(lbm.lbm_nn_pool2(x.data_ptr(), y.data_ptr(), c, n, d, h, w, 0.125, self._stream()),
                 "pool")
        return y

    def _up(self, x, c, vol_out, scale=1.0):
        torch = self.torch
        n, d, h, w = vol_out
        y = torch.empty((n * d * h * w, c), dtype=torch.bfloat16, device=self.dev)
        self._ok(lbm.lbm_nn_upsample2(x.data_ptr(), y.data_ptr(), c, n, d, h, w, float(scale),
                                      self._stream()), "upsample")
        return y

    def _cat(self, a, ca, b, cb):
        torch = self.torch
        y = torch.empty((a.shape[0], ca + cb), dtype=torch.bfloat16, device=self.dev)
        self._ok(lbm.lbm_nn_concat(a.data_ptr(), ca, b.data_ptr(), cb, y.data_ptr(), a.shape[0],
                                   self._stream()), "concat")
        return y

    def forward(self, x0, vol, t_lin, target=None):
        """x0 [V, 16] BF16 input, t_lin [V] FP32; returns pred [V] FP32 (and
        keeps the activations for backward).  With a target, also the loss
        and the head's gradients."""
        torch = self.torch
        n, d, h, w = vol
        v2 = (n, d // 2, h // 2, w // 2)
        v4 = (n, d // 4, h // 4, w // 4)
        A = {"x0": x0}
        A["a1"] = self._conv(0, x0, vol)
        A["s1"] = self._conv(1, A["a1"], vol)
        A["p1"] = self._pool(A["s1"], 32, vol)
        A["a3"] = self._conv(2, A["p1"], v2)
        A["s2"] = self._conv(3, A["a3"], v2)
        A["p2"] = self._pool(A["s2"], 64, v2)
        A["a5"] = self._conv(4, A["p2"], v4)
        A["a6"] = self._conv(5, A["a5"], v4)
        A["u1"] = self._up(A["a6"], 128, v2)
        A["c1"] = self._cat(A["u1"], 128, A["s2"], 64)
        A["a7"] = self._conv(6, A["c1"], v2)
        A["a8"] = self._conv(7, A["a7"], v2)
        A["u2"] = self._up(A["a8"], 64, vol)
        A["c2"] = self._cat(A["u2"], 64, A["s1"], 32)
        A["a9"] = self._conv(8, A["c2"], vol)
        V = n * d * h * w
        pred = torch.empty(V, dtype=torch.float32, device=self.dev)
        self.vol, self.A = vol, A
        if target is None:
            self._ok(lbm.lbm_nn_head(A["a9"].data_ptr(), self.hw.data_ptr(), self.hb.data_ptr(),
                                     t_lin.data_ptr(), None, pred.data_ptr(), None, None, None,
                                     None, V, self._stream()), "head")
            return pred, None
        self.g_hw = torch.zeros_like(self.hw)
        self.g_hb = torch.zeros_like(self.hb)
        loss = torch.zeros(1, dtype=torch.float64, device=self.dev)
        self.dh9 = torch.empty((V, HEAD_C), dtype=torch.bfloat16, device=self.dev)
        self._ok(lbm.lbm_nn_head(A["a9"].data_ptr(), self.hw.data_ptr(), self.hb.data_ptr(),
                                 t_lin.data_ptr(), target.data_ptr(), pred.data_ptr(),
                                 self.dh9.data_ptr(), self.g_hw.data_ptr(), self.g_hb.data_ptr(),
                                 loss.data_ptr(), V, self._stream()), "head")
        return pred, loss

    def _back_conv(self, l, g_out, x_in, vol, need_dx=True):
        """Weight, bias and (optionally) input gradients of conv layer l."""
        torch = self.torch
        n, d, h, w = vol
        cin, cout = CONV3[l]
        V = n * d * h * w
        self.gW[l].zero_()
        self.gb[l].zero_()
        s = self._stream()
        self._ok(lbm.lbm_nn_conv3d_wgrad(x_in.data_ptr(), cin, g_out.data_ptr(), cout,
                                         self.gW[l].data_ptr(), n, d, h, w, 3, s), "wgrad")
        self._ok(lbm.lbm_nn_bias_grad(g_out.data_ptr(), cout, V, self.gb[l].data_ptr(), s), "bgrad")
        if not need_dx:
            return None
        wf = torch.empty((27, cout, cin), dtype=torch.bfloat16, device=self.dev)
        self._ok(lbm.lbm_nn_flip_weights(self.Wb[l].data_ptr(), wf.data_ptr(), cin, cout, 3, s), "flip")
        dx = torch.empty((V, cin), dtype=torch.bfloat16, device=self.dev)
        self._ok(lbm.lbm_nn_conv3d(g_out.data_ptr(), cout, wf.data_ptr(), None, dx.data_ptr(), cin,
                                   n, d, h, w, 3, 0, 0, s), "dgrad")
        return dx

    def _mask(self, dy, y):
        g = self.torch.empty_like(dy)
        self._ok(lbm.lbm_nn_relu_mask(dy.data_ptr(), y.data_ptr(), g.data_ptr(), dy.numel(),
                                      self._stream()), "relu mask")
        return g

    def _slice(self, src, csrc, off, c, dst=None):
        torch = self.torch
        acc = dst is not None
        if dst is None:
            dst = torch.empty((src.shape[0], c), dtype=torch.bfloat16, device=self.dev)
        self._ok(lbm.lbm_nn_slice(src.data_ptr(), csrc, off, dst.data_ptr(), c, src.shape[0],
                                  int(acc), self._stream()), "slice")
        return dst

    def backward(self):
        """Gradients of the loss of the last forward into gW, gb, g_hw, g_hb."""
        torch = self.torch
        A, vol = self.A, self.vol
        n, d, h, w = vol
        v2 = (n, d // 2, h // 2, w // 2)
        v4 = (n, d // 4, h // 4, w // 4)
        if not hasattr(self, "gW"):
            self.gW = [torch.zeros_like(x) for x in self.W]
            self.gb = [torch.zeros_like(x) for x in self.b]
        g9 = self._mask(self.dh9, A["a9"])
        dc2 = self._back_conv(8, g9, A["c2"], vol)
        du2 = self._slice(dc2, 96, 0, 64)
        ds1_cat = self._slice(dc2, 96, 64, 32)
        s = self._stream()
        da8 = torch.empty((A["a8"].shape[0], 64), dtype=torch.bfloat16, device=self.dev)
        self._ok(lbm.lbm_nn_pool2(du2.data_ptr(), da8.data_ptr(), 64, n, d, h, w, 1.0, s), "up bwd")
        g8 = self._mask(da8, A["a8"])
        da7 = self._back_conv(7, g8, A["a7"], v2)
        g7 = self._mask(da7, A["a7"])
        dc1 = self._back_conv(6, g7, A["c1"], v2)
        du1 = self._slice(dc1, 192, 0, 128)
        ds2 = self._slice(dc1, 192, 128, 64)
        da6 = torch.empty((A["a6"].shape[0], 128), dtype=torch.bfloat16, device=self.dev)
        self._ok(lbm.lbm_nn_pool2(du1.data_ptr(), da6.data_ptr(), 128, *v2, 1.0, s), "up bwd")
        g6 = self._mask(da6, A["a6"])
        da5 = self._back_conv(5, g6, A["a5"], v4)
        g5 = self._mask(da5, A["a5"])
        dp2 = self._back_conv(4, g5, A["p2"], v4)
        dp2u = self._up(dp2, 64, v2, 0.125)
        self._slice(dp2u, 64, 0, 64, dst=ds2)
        g4 = self._mask(ds2, A["s2"])
        da3 = self._back_conv(3, g4, A["a3"], v2)
        g3 = self._mask(da3, A["a3"])
        dp1 = self._back_conv(2, g3, A["p1"], v2)
        dp1u = self._up(dp1, 32, vol, 0.125)
        self._slice(dp1u, 32, 0, 32, dst=ds1_cat)
        g2 = self._mask(ds1_cat, A["s1"])
        da1 = self._back_conv(1, g2, A["a1"], vol)
        g1 = self._mask(da1, A["a1"])
        self._back_conv(0, g1, A["x0"], vol, need_dx=False)

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.t += 1
        grads = self.gW + self.gb + [self.g_hw, self.g_hb]
        s = self._stream()
        for i, (p, g) in enumerate(zip(self.params, grads)):
            pb = self.Wb[i].data_ptr() if i < len(CONV3) else None
            self._ok(lbm.lbm_nn_adam(p.data_ptr(), g.data_ptr(), self.m[i].data_ptr(),
                                     self.v[i].data_ptr(), pb, p.numel(), lr, beta1, beta2, eps,
                                     self.t, s), "adam")

    # ---- helpers ---------------------------------------------------------
    def make_input(self, phases, lams, t_hot=1.0, t_cold=0.0):
        """Device input and linear profile for n cells of equal size
        (phases uint8 [n, d, h, w] on the host, one tensor table per cell)."""
        torch = self.torch
        phases = np.ascontiguousarray(phases, dtype=np.uint8)
        n, d, h, w = phases.shape
        V = n * d * h * w
        x0 = torch.empty((V, 16), dtype=torch.bfloat16, device=self.dev)
        prof = linear_profile(d, t_hot, t_cold)
        tl = torch.from_numpy(np.broadcast_to(prof[None, :, None, None], (n, d, h, w)).reshape(-1)
                              .copy()).to(self.dev)
        tz = torch.from_numpy(prof).to(self.dev)
        for i in range(n):
            ph = torch.from_numpy(phases[i].reshape(-1)).to(self.dev)
            tab = torch.from_numpy(material_table(lams[i]).reshape(-1)).to(self.dev)
            sub = x0[i * d * h * w:(i + 1) * d * h * w]
            self._ok(lbm.lbm_nn_input(ph.data_ptr(), tab.data_ptr(), tz.data_ptr(), sub.data_ptr(),
                                      1, d, h, w, self._stream()), "input")
        return x0, tl

    def predict(self, phase, lam, t_hot=1.0, t_cold=0.0) -> np.ndarray:
        """Predicted temperature [d, h, w] of one cell (z = temperature axis)."""
        d, h, w = phase.shape
        x0, tl = self.make_input(phase[None], [lam], t_hot, t_cold)
        pred, _ = self.forward(x0, (1, d, h, w), tl)
        return pred.view(d, h, w).cpu().numpy()


def generate_cells(seeds, n=64, g_range=(20.0, 45.0), phi_range=(0.30, 0.60), A=10.0, B=6.0,
                   tol=1e-7, max_iters=400_000, device=0):
    """Seeded braided n^3 cells and their steady temperatures from the
    library's batched solver (z axis, periodic laterals, FP32)."""
    phases, lams = [], []
    for s in seeds:
        r = I.SplitMix64(10_000 + int(s))
        g = g_range[0] + (g_range[1] - g_range[0]) * r.uniform()
        phi = phi_range[0] + (phi_range[1] - phi_range[0]) * r.uniform()
        with lbm.Solver(n, n, n, device) as S:
            S.set_geometry_braid(math.radians(g), I.braid_anchors(n, n, int(s), n_max=256), phi, A, B)
            phases.append(S.geometry())
        lams.append(I.braid_tensors(g))
    B_ = lbm.Batch(device)
    for ph, lam in zip(phases, lams):
        B_.add(ph, lam, 2)
    B_.solve(0, lbm.Solver.opts(tol=tol, max_iters=max_iters))
    temps = np.stack([B_.temperature(i) for i in range(len(phases))])
    k = np.array([B_.result(i).k_eff for i in range(len(phases))])
    B_.close()
    return np.stack(phases), lams, temps, k


def train(net: WarmNet, phases, lams, temps, epochs=10, batch=4, lr=1e-3, seed=0, log=None):
    """Adam on the mean squared error of the predicted temperature."""
    torch = net.torch
    rng = np.random.default_rng(seed)
    n = len(phases)
    _, d, h, w = phases.shape
    history = []
    for ep in range(epochs):
        order = rng.permutation(n)
        tot = 0.0
        for i in range(0, n - batch + 1, batch):
            idx = order[i:i + batch]
            x0, tl = net.make_input(phases[idx], [lams[j] for j in idx])
            tgt = torch.from_numpy(temps[idx].reshape(-1).astype(np.float32)).to(net.dev)
            _, loss = net.forward(x0, (len(idx), d, h, w), tl, tgt)
            net.backward()
            net.adam_step(lr)
            tot += float(loss.item()) / (len(idx) * d * h * w)
        history.append(tot / max(1, n // batch))
        if log:
            log(f"epoch {ep}: mse {history[-1]:.3e}")
    return history
