"""FP64 CPU oracle of the warm-start network (forward pass, loss, gradients).

TEST INFRASTRUCTURE.  Only the test suite may import this module; the library
never calls it.

The network is the library's own addition (the ptychopy paper's Sec. 2.2 lets
the user supply an object guess; this is a learned guess).  Architecture: 12
convolutions with 3x3 kernels and padding 1 over 6 resolution levels
(128, 64, 32, 16, 8, 4, then back up to 64), stride-2 convolutions going down,
nearest-neighbour x2 upsampling before the convolution going up, ReLU after
every layer but the last.  Input x = log(1 + max(I, 0)) / 10 of a 128 x 128
detector-centred frame; output (amplitude, phase) of the central 64 x 64
object patch.  Loss L = sum (out - target)^2 / (B * 2 * 64 * 64).

Parameter vector: for each layer, weights [co][ci][3][3] then biases [co].
Everything here is plain numpy in FP64: each convolution is a sum over the
nine taps of strided slices of the zero-padded input, and the backward pass
applies the adjoint of each of those steps in reverse order.
"""
from __future__ import annotations

import numpy as np

# (ci, co, stride, upsample, relu)
LAYERS = [
    (1, 16, 1, 0, 1), (16, 32, 2, 0, 1), (32, 64, 2, 0, 1), (64, 128, 2, 0, 1),
    (128, 256, 2, 0, 1), (256, 256, 2, 0, 1), (256, 256, 1, 0, 1),
    (256, 128, 1, 1, 1), (128, 64, 1, 1, 1), (64, 32, 1, 1, 1), (32, 16, 1, 1, 1),
    (16, 2, 1, 0, 0),
]


def layout():
    """(weight offset, bias offset) of each layer and the total size."""
    offs, o = [], 0
    for ci, co, *_ in LAYERS:
        offs.append((o, o + co * ci * 9))
        o += co * ci * 9 + co
    return offs, o


def unpack(params):
    offs, _ = layout()
    out = []
    for (ci, co, *_), (wo, bo) in zip(LAYERS, offs):
        out.append((params[wo:wo + co * ci * 9].reshape(co, ci, 3, 3), params[bo:bo + co]))
    return out


def bf16_round(x):
    """Round to the nearest BF16 value (8-bit significand, ties to even),
    returned as float64."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def net_input(I, act_bf16=False):
    x = np.log1p(np.maximum(np.asarray(I, np.float64), 0.0))[:, None] / 10.0
    return bf16_round(x) if act_bf16 else x


def conv(x, w, b, stride, up):
    """y[b,o,Y,X] = b[o] + sum_{c,dy,dx} w[o,c,dy,dx] xu[b,c,s*Y+dy-1, s*X+dx-1],
    xu = x upsampled (nearest, x2) if up, zero outside."""
    if up:
        x = x.repeat(2, axis=2).repeat(2, axis=3)
    H, W = x.shape[2], x.shape[3]
    Ho, Wo = (H - 1) // stride + 1, (W - 1) // stride + 1
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    y = np.zeros((x.shape[0], w.shape[0], Ho, Wo)) + b[None, :, None, None]
    for dy in range(3):
        for dx in range(3):
            sl = xp[:, :, dy:dy + stride * (Ho - 1) + 1:stride, dx:dx + stride * (Wo - 1) + 1:stride]
            y += np.einsum("bchw,oc->bohw", sl, w[:, :, dy, dx])
    return y


def conv_adjoint(gy, x, w, stride, up):
    """Gradients (dx, dw, db) of sum(gy * conv(x, w, b)) with respect to x, w, b."""
    xu = x.repeat(2, axis=2).repeat(2, axis=3) if up else x
    H, W = xu.shape[2], xu.shape[3]
    Ho, Wo = gy.shape[2], gy.shape[3]
    xp = np.pad(xu, ((0, 0), (0, 0), (1, 1), (1, 1)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            sy = slice(dy, dy + stride * (Ho - 1) + 1, stride)
            sx = slice(dx, dx + stride * (Wo - 1) + 1, stride)
            gw[:, :, dy, dx] = np.einsum("bohw,bchw->oc", gy, xp[:, :, sy, sx])
            gxp[:, :, sy, sx] += np.einsum("bohw,oc->bchw", gy, w[:, :, dy, dx])
    gxu = gxp[:, :, 1:H + 1, 1:W + 1]
    if up:  # adjoint of nearest upsampling: sum each 2x2 block
        gx = gxu.reshape(gxu.shape[0], gxu.shape[1], H // 2, 2, W // 2, 2).sum(axis=(3, 5))
    else:
        gx = gxu
    return gx, gw, gy.sum(axis=(0, 2, 3))


def forward(params, I, act_bf16=False):
    """Network output [B, 2, 64, 64] and the per-layer inputs/pre-activations.
    act_bf16: store the input and every hidden activation in BF16, as the
    method does (the output layer stays unrounded)."""
    x = net_input(I, act_bf16)
    cache = []
    for (w, b), (ci, co, s, up, relu) in zip(unpack(np.asarray(params, np.float64)), LAYERS):
        pre = conv(x, w, b, s, up)
        cache.append((x, pre))
        x = np.maximum(pre, 0.0) if relu else pre
        if act_bf16 and relu:
            x = bf16_round(x)
    return x, cache


def loss_and_grads(params, I, targets, act_bf16=False):
    """L = sum (out - t)^2 / (B * 2 * 64 * 64) and dL/dparams (same layout)."""
    params = np.asarray(params, np.float64)
    out, cache = forward(params, I, act_bf16)
    n = out.size
    d = out - np.asarray(targets, np.float64)
    L = float(np.sum(d * d)) / n
    g = 2.0 * d / n
    grads = np.zeros_like(params)
    offs, _ = layout()
    layers = unpack(params)
    for l in range(len(LAYERS) - 1, -1, -1):
        ci, co, s, up, relu = LAYERS[l]
        x, pre = cache[l]
        if relu:
            g = g * (pre > 0)
        gx, gw, gb = conv_adjoint(g, x, layers[l][0], s, up)
        wo, bo = offs[l]
        grads[wo:wo + gw.size] = gw.ravel()
        grads[bo:bo + gb.size] = gb
        g = gx
    return L, grads
