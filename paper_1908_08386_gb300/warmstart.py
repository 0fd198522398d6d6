"""Learned warm start: training data from the batched solver, training, and
initial states for the LBM-FVM iteration.

The data are steady fields that the batched solver computes itself (FP32
storage, run to a residual of 1e-6, where FP32 rounding still leaves the
fields accurate far beyond what the network can learn).  The network sees a
cavity resampled to 128 x 128 and predicts (u/U0, v/U0, T) there; the
prediction is interpolated back to the cavity's nodes and handed to
lbmfvm_batch_set_state, which starts from f = f_eq(1, u) with the boundary
temperatures imposed.  The iteration then runs to the same residual as from
rest, so a poor prediction costs steps, never accuracy.
"""

from __future__ import annotations

import math
import time

import numpy as np

from . import Batch
from . import surrogate as S

RES = 128  # the network's grid


def case_arrays(cases, res=RES):
    """Masks (uint8, N x ny x nx list), scalars (N x 2) and fluid masks at the
    network's grid for cavities that are already res x res."""
    masks = np.zeros((len(cases), res, res), np.uint8)
    for i, c in enumerate(cases):
        if c.mask is not None:
            masks[i] = np.asarray(c.mask, np.uint8).reshape(c.ny, c.nx)
    scalars = np.stack([S.input_scalars(c.Ra, c.Pr) for c in cases]).astype(np.float32)
    fluid = (masks == 0).astype(np.uint8)
    fluid[:, 0, :] = fluid[:, -1, :] = 0
    fluid[:, :, 0] = fluid[:, :, -1] = 0
    return masks, scalars, fluid


def generate(cases, tol=1e-6, check_every=1000, max_steps=600000, log=print):
    """Steady (u/U0, v/U0, T) of every cavity (N x res x res x 3 float32) from
    one batched FP32 run."""
    import torch

    t0 = time.time()
    b = Batch(cases, store="f32")
    b.set_polish("f32", 0)  # stay in FP32: tol is above its floor
    steps, r = b.run(tol=tol, check_every=check_every, max_steps=max_steps)
    torch.cuda.synchronize()
    log(f"generated {len(cases)} steady fields in {time.time() - t0:.1f} s: steps {int(steps.min())}.."
        f"{int(steps.max())}, residual max {float(np.nanmax(r)):.2e}")
    targets = np.zeros((len(cases), cases[0].ny, cases[0].nx, 3), np.float32)
    for i, c in enumerate(cases):
        _, u, v, T = b.fields(i)
        U0 = c.Ma / math.sqrt(3.0)
        targets[i] = np.stack([u / U0, v / U0, T], -1)
    b.close()
    return targets, steps, r


class Dataset:
    """Network inputs and targets resident on the device."""

    def __init__(self, cases, targets):
        import torch

        masks, scalars, fluid = case_arrays(cases)
        dev = "cuda"
        self.n = len(cases)
        self.masks = torch.from_numpy(masks).to(dev)
        self.scalars = torch.from_numpy(scalars).to(dev)
        self.fluid = torch.from_numpy(fluid).to(dev)
        self.targets = torch.from_numpy(np.ascontiguousarray(targets, np.float32)).to(dev)
        self.n_fluid = fluid.reshape(self.n, -1).sum(1)

    def batch(self, idx):
        import torch

        sel = torch.as_tensor(idx, device="cuda")
        return (self.masks.index_select(0, sel).contiguous(), self.scalars.index_select(0, sel).contiguous(),
                self.targets.index_select(0, sel).contiguous(), self.fluid.index_select(0, sel).contiguous(),
                int(self.n_fluid[idx].sum()))


def train(net, data: Dataset, epochs=60, batch=32, lr=1e-3, seed=0, log=print):
    """Adam with a cosine learning-rate schedule over `epochs` passes of
    mini-batches of `batch` samples; returns the mean loss per epoch."""
    import torch

    rng = np.random.default_rng(seed)
    steps_per_epoch = data.n // batch
    total = epochs * steps_per_epoch
    history = []
    k = 0
    t0 = time.time()
    for ep in range(epochs):
        perm = rng.permutation(data.n)
        bufs = net.buffers(batch, RES)
        bufs["loss"].zero_()
        for s in range(steps_per_epoch):
            m, sc, tg, fl, nf = data.batch(perm[s * batch:(s + 1) * batch])
            net.encode(m, sc, batch, RES)
            net.forward(batch, RES)
            net.loss(batch, RES, tg, fl, nf)
            net.backward(batch, RES)
            net.adam(lr * 0.5 * (1.0 + math.cos(math.pi * k / total)))
            k += 1
        history.append(bufs["loss"].item() / steps_per_epoch)
        if ep % 10 == 0 or ep == epochs - 1:
            log(f"epoch {ep}: loss {history[-1]:.4e} ({time.time() - t0:.1f} s)")
    torch.cuda.synchronize()
    return history


def predict(net, data: Dataset, idx, batch=32):
    """Network output (len(idx) x res x res x 3, host float32)."""
    out = []
    for s in range(0, len(idx), batch):
        part = list(idx[s:s + batch])
        B = len(part)
        m, sc, _, _, _ = data.batch(part)
        net.encode(m, sc, B, RES)
        out.append(net.forward(B, RES).cpu().numpy().copy())
    return np.concatenate(out)


def errors(pred, targets, fluid):
    """RMS errors of T and of the velocity (relative to the targets' RMS speed)
    over fluid nodes."""
    f = fluid.astype(bool)
    dT = (pred[..., 2] - targets[..., 2])[f]
    du = (pred[..., :2] - targets[..., :2])[f]
    speed = targets[..., :2][f]
    return float(np.sqrt(np.mean(dT ** 2))), float(np.sqrt(np.mean(du ** 2)) / np.sqrt(np.mean(speed ** 2)))


def initial_states(net, cases, batch=32):
    """Warm-start fields (u, v, T device float32 ny x nx tensors) of arbitrary
    cavities: mask sampled to the network grid, prediction, bilinear
    interpolation back, U0 scaling, T clipped to [0, 1]."""
    import torch

    dev = "cuda"
    out = []
    for s in range(0, len(cases), batch):
        part = cases[s:s + batch]
        B = len(part)
        masks_d = []
        small = torch.zeros(B, RES, RES, dtype=torch.uint8, device=dev)
        for j, c in enumerate(part):
            m = np.zeros((c.ny, c.nx), np.uint8) if c.mask is None else np.asarray(c.mask, np.uint8).reshape(c.ny, c.nx)
            md = torch.from_numpy(np.ascontiguousarray(m)).to(dev)
            masks_d.append(md)
            S.call("lbmfvm_sg_resample_mask", md.data_ptr(), c.nx, c.ny, small[j].data_ptr(), RES, RES, S._stream())
        scal = torch.from_numpy(np.stack([S.input_scalars(c.Ra, c.Pr) for c in part])).to(dev)
        net.encode(small, scal, B, RES)
        pred = net.forward(B, RES)
        for j, c in enumerate(part):
            u, v, T = (torch.empty(c.ny, c.nx, dtype=torch.float32, device=dev) for _ in range(3))
            S.call("lbmfvm_sg_resample_fields", pred[j].data_ptr(), RES, RES, masks_d[j].data_ptr(), c.nx, c.ny,
                   c.Ma / math.sqrt(3.0), u.data_ptr(), v.data_ptr(), T.data_ptr(), S._stream())
            out.append((u, v, T))
    torch.cuda.synchronize()
    return out


def warm_start(batch: Batch, net, cases):
    """set_state of every cavity of `batch` from the network's prediction."""
    for i, (u, v, T) in enumerate(initial_states(net, cases)):
        batch.set_state(i, u, v, T)
