"""Plain PyTorch (CPU) reference of the pose-proposal CNN, for tests only.

TEST INFRASTRUCTURE ONLY: nothing in the product library imports this file.

The network, written with torch.nn.functional on float32 CPU tensors (NCHW):
input = the acquired and the simulated 64x64 patch, each normalised to zero
mean and unit population deviation over the valid pixels (invalid pixels
0), as 2 of 16 input channels; six 3x3 convolutions with padding 1, bias
and ReLU (channels 32, 32, 64, 64, 64, 64; strides 1, 2, 2, 2, 2, 1);
the 4x4x64 last activation flattened in (y, x, channel) order; a linear
layer to 6 outputs.  Loss: the
batch mean of sum_j (out_j - target_j)^2.

Parameters come as one flat float32 vector: per layer the weights
[co][ky][kx][ci] then the bias, then the head [6][1024] and its bias.
With emulate_bf16, weights, the input image, every stored activation and
every activation gradient are rounded to bfloat16 where the GPU stores them
in that format.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

LAYERS = [(16, 32, 1), (32, 32, 2), (32, 64, 2), (64, 64, 2), (64, 64, 2), (64, 64, 1)]
FEAT = 4 * 4 * 64   # flattened last activation


def _bf(t):
    return t.to(torch.bfloat16).to(torch.float32)


def unpack(flat):
    flat = torch.as_tensor(np.asarray(flat, dtype=np.float32))
    o, ws, bs = 0, [], []
    for cin, cout, _ in LAYERS:
        n = cout * 9 * cin
        ws.append(flat[o:o + n].reshape(cout, 3, 3, cin).permute(0, 3, 1, 2).contiguous())   # OIHW
        o += n
        bs.append(flat[o:o + cout].clone())
        o += cout
    hw = flat[o:o + 6 * FEAT].reshape(6, FEAT).clone()
    o += 6 * FEAT
    hb = flat[o:o + 6].clone()
    return ws, bs, hw, hb


def pack(ws, bs, hw, hb):
    parts = []
    for w, b in zip(ws, bs):
        parts += [w.permute(0, 2, 3, 1).reshape(-1), b.reshape(-1)]
    parts += [hw.reshape(-1), hb.reshape(-1)]
    return torch.cat(parts).detach().numpy()


def inputs(y, s, valid, desc):
    """Normalised input images [B, 16, 64, 64] (float32)."""
    y = np.asarray(y, np.float64)
    s = np.asarray(s, np.float64)
    valid = np.asarray(valid).astype(bool)
    B = desc.shape[0]
    img = np.zeros((B, 16, 64, 64), np.float32)
    for b in range(B):
        o = int(desc[b, 6])
        v = valid[o:o + 4096]
        for c, arr in ((0, y), (1, s)):
            a = arr[o:o + 4096]
            cnt = max(v.sum(), 1)
            m = a[v].sum() / cnt
            var = max((a[v] ** 2).sum() / cnt - m * m, 1e-6)
            img[b, c] = np.where(v, (a - m) / np.sqrt(var), 0.0).reshape(64, 64)
    return torch.from_numpy(img)


def forward(flat, img, emulate_bf16=True):
    """Returns (out [B, 6], activations) with autograd enabled on the
    parameters (the returned parameter tensors require grad)."""
    ws, bs, hw, hb = unpack(flat)
    params = []
    for t in ws + bs + [hw, hb]:
        t.requires_grad_(True)
        params.append(t)
    x = _bf(img) if emulate_bf16 else img
    for (cin, cout, st), w, b in zip(LAYERS, ws, bs):
        wq = _bf(w) if emulate_bf16 else w
        if emulate_bf16:
            wq = w + (wq - w).detach()          # rounded value, gradient of the master weight
        x = F.relu(F.conv2d(x, wq, b, stride=st, padding=1))
        if emulate_bf16:
            x = x + (_bf(x) - x).detach()
            x.register_hook(lambda g: _bf(g))
    feat = x.permute(0, 2, 3, 1).reshape(x.shape[0], FEAT)   # (y, x, channel) order
    out = feat @ hw.t() + hb
    return out, (ws, bs, hw, hb)


def loss_and_grads(flat, img, target, emulate_bf16=True):
    out, (ws, bs, hw, hb) = forward(flat, img, emulate_bf16)
    t = torch.as_tensor(np.asarray(target, np.float32))
    loss = ((out - t) ** 2).sum(dim=1).mean()
    loss.backward()
    g = pack([w.grad for w in ws], [b.grad for b in bs], hw.grad, hb.grad)
    return float(loss.detach()), out.detach().numpy(), g
