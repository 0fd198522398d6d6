"""Learned warm start: binding and driver of the surrogate network.

The network maps a cavity's obstacle mask, normalised log10 Ra and Pr (three
input planes at 128 x 128) to (u/U0, v/U0, T) through a 4-level
encoder-decoder: per level two 3x3 convolutions with the leaky ReLU, 2x2
average pooling down, nearest-neighbour up-sampling and skip concatenation on
the way up, a 1x1 output layer.  Every arithmetic step of training and
inference runs in the CUDA kernels of liblbmfvm.so (include/surrogate.h);
this module owns the buffers (PyTorch device memory), orders the kernel calls
and marshals their arguments.

Activations are BF16 NHWC; the encoder writes each level's output straight
into the decoder's concatenation buffer of that resolution (channels after
the up-sampled ones).  Parameters are kept in FP32 (Adam's master copy) with
BF16 copies of the 3x3 weights for the tensor cores.
"""

from __future__ import annotations

import ctypes
import math

import numpy as np

from . import LbmfvmError, lib

LINEAR, LEAKY, DLEAKY = 0, 1, 2
IN_CHANNELS = 16  # the three input planes padded to one 16-channel K step

# Every entry point include/surrogate.h declares (checked by the test-suite).
SG_EXPORTS = (
    "lbmfvm_sg_conv3x3", "lbmfvm_sg_flip", "lbmfvm_sg_conv3x3_wgrad", "lbmfvm_sg_pool2", "lbmfvm_sg_pool2_backward",
    "lbmfvm_sg_upsample2", "lbmfvm_sg_upsample2_backward", "lbmfvm_sg_conv1x1", "lbmfvm_sg_conv1x1_backward",
    "lbmfvm_sg_mse", "lbmfvm_sg_adam", "lbmfvm_sg_encode", "lbmfvm_sg_resample_mask", "lbmfvm_sg_resample_fields",
    "lbmfvm_sg_check", "lbmfvm_sg_inject_stall", "lbmfvm_sg_last_error",
)

_ready = False


def _lib():
    global _ready
    L = lib()
    if not _ready:
        vp, i32, i64, f, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
        sig = {
            "lbmfvm_sg_conv3x3": [vp, i32, vp, vp, vp, i32, vp, i32, i32, i32, i32, i32, i32, i32, vp],
            "lbmfvm_sg_flip": [vp, vp, i32, i32, vp],
            "lbmfvm_sg_conv3x3_wgrad": [vp, i32, vp, i32, vp, vp, i32, i32, i32, i32, i32, vp],
            "lbmfvm_sg_pool2": [vp, i32, vp, i32, i32, i32, i32, i32, vp],
            "lbmfvm_sg_pool2_backward": [vp, i32, vp, i32, vp, i32, vp, i32, i32, i32, i32, i32, vp],
            "lbmfvm_sg_upsample2": [vp, i32, vp, i32, i32, i32, i32, i32, vp],
            "lbmfvm_sg_upsample2_backward": [vp, i32, vp, i32, vp, i32, i32, i32, i32, i32, vp],
            "lbmfvm_sg_conv1x1": [vp, i32, vp, vp, vp, i64, i32, i32, vp],
            "lbmfvm_sg_conv1x1_backward": [vp, i32, vp, vp, vp, i32, vp, vp, i64, i32, i32, vp],
            "lbmfvm_sg_mse": [vp, vp, vp, i64, i32, d, vp, vp, vp],
            "lbmfvm_sg_adam": [vp, vp, vp, vp, vp, i64, f, f, f, f, i32, vp],
            "lbmfvm_sg_encode": [vp, vp, vp, i32, i32, i32, vp],
            "lbmfvm_sg_resample_mask": [vp, i32, i32, vp, i32, i32, vp],
            "lbmfvm_sg_resample_fields": [vp, i32, i32, vp, i32, i32, f, vp, vp, vp, vp],
            "lbmfvm_sg_check": [vp],
            "lbmfvm_sg_inject_stall": [],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.restype = ctypes.c_int
            fn.argtypes = args
        L.lbmfvm_sg_last_error.restype = ctypes.c_char_p
        L.lbmfvm_sg_last_error.argtypes = []
        _ready = True
    return L


def call(name, *args):
    """Call one surrogate entry point; raise LbmfvmError on a non-zero status."""
    L = _lib()
    r = getattr(L, name)(*args)
    if r != 0:
        raise LbmfvmError(r, L.lbmfvm_sg_last_error().decode())


def check():
    """Synchronise the current stream; raise if a bounded device wait of the
    tensor-core convolution ran out since the last check."""
    call("lbmfvm_sg_check", _stream())


def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class View:
    """A channel slice of an NHWC tensor: pointer to its first channel and the
    tensor's channel stride."""

    def __init__(self, t, c0=0, c=None):
        self.t = t
        self.ld = int(t.shape[-1])
        self.c = self.ld - c0 if c is None else c
        self.ptr = t.data_ptr() + c0 * t.element_size()


def conv3x3(x: View, w_ptr, bias_ptr, y: View, B, H, W, cin, cout, mode, m: View | None = None):
    call("lbmfvm_sg_conv3x3", x.ptr, x.ld, w_ptr, bias_ptr, y.ptr, y.ld, m.ptr if m else None, m.ld if m else 0,
         B, H, W, cin, cout, mode, _stream())


def input_scalars(Ra, Pr):
    """Normalised (log10 Ra, Pr) of the network input (Ra in [1e3, 1e6] and Pr
    in [0.71, 7.0] map to [-1, 1])."""
    return np.array([(math.log10(Ra) - 4.5) / 1.5, (Pr - 3.855) / 3.145], dtype=np.float32)


class Surrogate:
    """The warm-start network on the current CUDA device.

    ``params``: list of numpy arrays in the layer order and shapes of
    ``workloads.surrogate_init`` (3x3 weights [Co, 3, 3, Ci], biases, 1x1
    weights [Co, Ci]); defaults to that function's seeded initialisation.
    """

    def __init__(self, widths=(32, 64, 96, 160), params=None, seed=0, device=None):
        import torch

        from . import workloads

        self.torch = torch
        self.dev = torch.device("cuda" if device is None else device)
        self.widths = tuple(int(w) for w in widths)
        for w in self.widths:
            if w % 32:
                raise ValueError("level widths must be multiples of 32")
        L = len(self.widths)
        # layers: (kind, real input channels, staged input channels, outputs)
        self.layers = []
        c = 3
        for w in self.widths:
            self.layers += [("c3", c, IN_CHANNELS if c == 3 else c, w), ("c3", w, w, w)]
            c = w
        for lvl in range(L - 2, -1, -1):
            w = self.widths[lvl]
            cin = self.widths[lvl + 1] + w
            self.layers += [("c3", cin, cin, w), ("c3", w, w, w)]
        self.layers.append(("c1", self.widths[0], self.widths[0], 3))
        # flat parameter buffers: per layer its weights then its biases
        self.offsets = []
        n = 0
        for kind, _, cin, cout in self.layers:
            nw = cout * 9 * cin if kind == "c3" else cout * cin
            self.offsets.append((n, n + nw))
            n += nw + cout
        n = (n + 7) // 8 * 8  # keeps every BF16 weight block 16-byte aligned below
        self.n = n
        f32 = dict(dtype=torch.float32, device=self.dev)
        self.p = torch.zeros(n, **f32)
        self.g = torch.zeros(n, **f32)
        self.m = torch.zeros(n, **f32)
        self.v = torch.zeros(n, **f32)
        self.pb = torch.zeros(n, dtype=torch.bfloat16, device=self.dev)  # BF16 copy
        self.pt = torch.zeros(n, dtype=torch.bfloat16, device=self.dev)  # adjoint (flipped) 3x3 weights
        for (kind, _, cin, _), (w0, _) in zip(self.layers, self.offsets):
            if kind == "c3" and (w0 * 2) % 16:
                raise AssertionError("unaligned weight block")
        self.t = 0
        self._bufs = {}
        self.set_params(params if params is not None else workloads.surrogate_init(self.widths, seed))

    # -- parameters ---------------------------------------------------------
    def _ptr(self, buf, off):
        return buf.data_ptr() + off * buf.element_size()

    def set_params(self, params):
        if len(params) != 2 * len(self.layers):
            raise ValueError("expected %d parameter arrays" % (2 * len(self.layers)))
        flat = np.zeros(self.n, dtype=np.float32)
        for i, ((kind, creal, cin, cout), (w0, b0)) in enumerate(zip(self.layers, self.offsets)):
            w = np.asarray(params[2 * i], dtype=np.float64)
            if kind == "c3":
                full = np.zeros((cout, 9, cin))
                full[:, :, :creal] = w.reshape(cout, 9, creal)
                flat[w0:b0] = full.ravel()
            else:
                flat[w0:b0] = w.ravel()
            flat[b0:b0 + cout] = np.asarray(params[2 * i + 1]).ravel()
        self.p.copy_(self.torch.from_numpy(flat))
        self.pb.copy_(self.p.to(self.torch.bfloat16))
        self.m.zero_()
        self.v.zero_()
        self.t = 0

    def get_params(self):
        flat = self.p.cpu().numpy().astype(np.float64)
        out = []
        for (kind, creal, cin, cout), (w0, b0) in zip(self.layers, self.offsets):
            if kind == "c3":
                out.append(flat[w0:b0].reshape(cout, 9, cin)[:, :, :creal].reshape(cout, 3, 3, creal).copy())
            else:
                out.append(flat[w0:b0].reshape(cout, cin).copy())
            out.append(flat[b0:b0 + cout].copy())
        return out

    def save(self, path):
        np.savez(path, widths=np.array(self.widths), *[p.astype(np.float32) for p in self.get_params()])

    @classmethod
    def load(cls, path, device=None):
        z = np.load(path)
        widths = tuple(int(w) for w in z["widths"])
        n = len([k for k in z.files if k.startswith("arr_")])
        return cls(widths, params=[z["arr_%d" % i] for i in range(n)], device=device)

    # -- buffers -------------------------------------------------------------
    def buffers(self, B, H):
        key = (B, H)
        if key in self._bufs:
            return self._bufs[key]
        torch = self.torch
        L = len(self.widths)
        if H % (16 << (L - 1)):
            raise ValueError("input size must be a multiple of %d" % (16 << (L - 1)))
        bf = dict(dtype=torch.bfloat16, device=self.dev)
        w = self.widths
        Hs = [H >> l for l in range(L)]
        z = lambda *s: torch.zeros(*s, **bf)
        bufs = {"x": z(B, H, H, IN_CHANNELS), "pred": torch.zeros(B, H, H, 3, dtype=torch.float32, device=self.dev),
                "dpred": torch.zeros(B, H, H, 3, dtype=torch.float32, device=self.dev),
                "loss": torch.zeros(1, dtype=torch.float64, device=self.dev)}
        for l in range(L):
            h = Hs[l]
            if l > 0:
                bufs["in", l] = z(B, h, h, w[l - 1])
                bufs["gin", l] = z(B, h, h, w[l - 1])
            bufs["a1", l] = z(B, h, h, w[l])
            bufs["ge1", l] = z(B, h, h, w[l])
            bufs["ge2", l] = z(B, h, h, w[l])
            if l < L - 1:
                bufs["cat", l] = z(B, h, h, w[l + 1] + w[l])
                bufs["gcat", l] = z(B, h, h, w[l + 1] + w[l])
                bufs["d1", l] = z(B, h, h, w[l])
                bufs["d2", l] = z(B, h, h, w[l])
                bufs["g1", l] = z(B, h, h, w[l])
                bufs["g2", l] = z(B, h, h, w[l])
            else:
                bufs["a2", l] = z(B, h, h, w[l])
        self._bufs[key] = bufs
        return bufs

    def _enc_out(self, bufs, l):
        """View of encoder level l's output (inside the concatenation buffer)."""
        L = len(self.widths)
        if l == L - 1:
            return View(bufs["a2", l])
        return View(bufs["cat", l], self.widths[l + 1])

    # -- passes ---------------------------------------------------------------
    def forward(self, B, H):
        """Network output (bufs['pred'], B x H x H x 3 FP32) of bufs['x']."""
        bufs = self.buffers(B, H)
        L, w = len(self.widths), self.widths
        s = _stream()
        h = View(bufs["x"])
        k = 0
        for l in range(L):
            hh = H >> l
            for j, (src, dst) in enumerate(((h, View(bufs["a1", l])), (View(bufs["a1", l]), self._enc_out(bufs, l)))):
                _, _, cin, cout = self.layers[k]
                w0, b0 = self.offsets[k]
                conv3x3(src, self._ptr(self.pb, w0), self._ptr(self.p, b0), dst, B, hh, hh, cin, cout, LEAKY)
                k += 1
            if l < L - 1:
                e = self._enc_out(bufs, l)
                call("lbmfvm_sg_pool2", e.ptr, e.ld, bufs["in", l + 1].data_ptr(), w[l], B, hh, hh, w[l], s)
                h = View(bufs["in", l + 1])
        d = self._enc_out(bufs, L - 1)
        for l in range(L - 2, -1, -1):
            hh = H >> l
            call("lbmfvm_sg_upsample2", d.ptr, d.ld, bufs["cat", l].data_ptr(), bufs["cat", l].shape[-1], B, hh // 2,
                 hh // 2, w[l + 1], s)
            for src, dst in ((View(bufs["cat", l]), View(bufs["d1", l])), (View(bufs["d1", l]), View(bufs["d2", l]))):
                _, _, cin, cout = self.layers[k]
                w0, b0 = self.offsets[k]
                conv3x3(src, self._ptr(self.pb, w0), self._ptr(self.p, b0), dst, B, hh, hh, cin, cout, LEAKY)
                k += 1
            d = View(bufs["d2", l])
        w0, b0 = self.offsets[k]
        call("lbmfvm_sg_conv1x1", d.ptr, d.ld, self._ptr(self.p, w0), self._ptr(self.p, b0), bufs["pred"].data_ptr(),
             B * H * H, w[0], 3, s)
        return bufs["pred"]

    def _adjoint(self, k, gy: View, gx: View, B, hh, mode, m: View | None = None):
        """Input gradient of 3x3 layer k from its output gradient."""
        _, _, cin, cout = self.layers[k]
        w0, _ = self.offsets[k]
        call("lbmfvm_sg_flip", self._ptr(self.pb, w0), self._ptr(self.pt, w0), cin, cout, _stream())
        conv3x3(gy, self._ptr(self.pt, w0), None, gx, B, hh, hh, cout, cin, mode, m)

    def _wgrad(self, k, x: View, gy: View, B, hh):
        _, _, cin, cout = self.layers[k]
        w0, b0 = self.offsets[k]
        call("lbmfvm_sg_conv3x3_wgrad", x.ptr, x.ld, gy.ptr, gy.ld, self._ptr(self.g, w0), self._ptr(self.g, b0), B,
             hh, hh, cin, cout, _stream())

    def backward(self, B, H):
        """Gradients (self.g) of the loss whose output gradient is bufs['dpred'],
        after forward() of the same batch."""
        bufs = self.buffers(B, H)
        L, w = len(self.widths), self.widths
        s = _stream()
        self.g.zero_()
        nl = len(self.layers)
        w0, b0 = self.offsets[nl - 1]
        last = View(bufs["d2", 0]) if L > 1 else self._enc_out(bufs, 0)
        first_grad = View(bufs["g2", 0]) if L > 1 else View(bufs["ge2", 0])
        call("lbmfvm_sg_conv1x1_backward", last.ptr, last.ld, self._ptr(self.p, w0), bufs["dpred"].data_ptr(),
             first_grad.ptr, first_grad.ld, self._ptr(self.g, w0), self._ptr(self.g, b0), B * H * H, w[0], 3, s)
        # decoder, fine to coarse; its layers sit after the 2L encoder layers
        for l in range(0, L - 1):
            hh = H >> l
            k1 = 2 * L + 2 * (L - 2 - l)
            k2 = k1 + 1
            self._wgrad(k2, View(bufs["d1", l]), View(bufs["g2", l]), B, hh)
            self._adjoint(k2, View(bufs["g2", l]), View(bufs["g1", l]), B, hh, DLEAKY, View(bufs["d1", l]))
            self._wgrad(k1, View(bufs["cat", l]), View(bufs["g1", l]), B, hh)
            self._adjoint(k1, View(bufs["g1", l]), View(bufs["gcat", l]), B, hh, LINEAR)
            # up-sampled part: through the coarser map's activation
            coarse = View(bufs["d2", l + 1]) if l + 1 <= L - 2 else self._enc_out(bufs, L - 1)
            gcoarse = View(bufs["g2", l + 1]) if l + 1 <= L - 2 else View(bufs["ge2", L - 1])
            gc = View(bufs["gcat", l])
            call("lbmfvm_sg_upsample2_backward", gc.ptr, gc.ld, coarse.ptr, coarse.ld, gcoarse.ptr, gcoarse.ld, B,
                 hh // 2, hh // 2, w[l + 1], s)
        # encoder, coarse to fine
        for l in range(L - 1, -1, -1):
            hh = H >> l
            k1, k2 = 2 * l, 2 * l + 1
            self._wgrad(k2, View(bufs["a1", l]), View(bufs["ge2", l]), B, hh)
            self._adjoint(k2, View(bufs["ge2", l]), View(bufs["ge1", l]), B, hh, DLEAKY, View(bufs["a1", l]))
            xin = View(bufs["x"]) if l == 0 else View(bufs["in", l])
            self._wgrad(k1, xin, View(bufs["ge1", l]), B, hh)
            if l > 0:
                self._adjoint(k1, View(bufs["ge1", l]), View(bufs["gin", l]), B, hh, LINEAR)
                skip = View(bufs["gcat", l - 1], w[l])  # the encoder part of the decoder's input gradient
                e = self._enc_out(bufs, l - 1)
                gi = View(bufs["gin", l])
                gd = View(bufs["ge2", l - 1])
                call("lbmfvm_sg_pool2_backward", gi.ptr, gi.ld, skip.ptr, skip.ld, e.ptr, e.ld, gd.ptr, gd.ld, B,
                     2 * hh, 2 * hh, w[l - 1], s)
        return self.g

    def loss(self, B, H, target, fluid, n_fluid):
        """Masked MSE of bufs['pred'] against target (B x H x H x 3 FP32) over
        the pixels where fluid (B x H x H uint8) is non-zero; fills
        bufs['dpred'] and accumulates the loss into bufs['loss'] (device)."""
        bufs = self.buffers(B, H)
        call("lbmfvm_sg_mse", bufs["pred"].data_ptr(), target.data_ptr(), fluid.data_ptr(), B * H * H, 3,
             1.0 / (3.0 * n_fluid), bufs["dpred"].data_ptr(), bufs["loss"].data_ptr(), _stream())

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.t += 1
        call("lbmfvm_sg_adam", self.p.data_ptr(), self.g.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
             self.pb.data_ptr(), self.n, lr, beta1, beta2, eps, self.t, _stream())

    def encode(self, masks, scalars, B, H):
        """bufs['x'] from B masks (device uint8, B x H x H) and scalars (device
        float32, B x 2)."""
        bufs = self.buffers(B, H)
        call("lbmfvm_sg_encode", masks.data_ptr(), scalars.data_ptr(), bufs["x"].data_ptr(), B, H, H, _stream())
