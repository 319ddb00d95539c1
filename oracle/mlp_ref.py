"""CPU double-precision reference of the cost model's network -- TEST INFRASTRUCTURE ONLY.

Forward and backward of the 6 -> 32 -> 32 -> 4 ReLU MLP with mean squared error,
written out with numpy in float64.  FP16 storage of weights and activations is
emulated by rounding through numpy.float16, so the only difference from the
GPU kernels is the FP32 (GPU) vs FP64 (here) accumulation.  Pinned in the tests
by central finite differences.

Parameter layout: W1[32][6], b1[32], W2[32][32], b2[32], W3[4][32], b3[4].
"""
from __future__ import annotations

import numpy as np

F, H, O = 6, 32, 4
SIZES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (O, H)), ("b3", (O,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(w: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = w[o:o + n].reshape(shape)
        o += n
    return out


def h16(x, emulate: bool):
    return x.astype(np.float16).astype(np.float64) if emulate else x


def loss_and_grad(w, feat, target, fmean, fstd, tmean, tstd, emulate_fp16: bool = True):
    """Mean squared error over samples and outputs (targets z-scored) and its gradient."""
    p = {k: h16(np.asarray(v, dtype=np.float64), emulate_fp16) for k, v in unpack(np.asarray(w)).items()}
    x = h16((np.asarray(feat, np.float64) - fmean) / fstd, emulate_fp16)          # n x F
    y = (np.asarray(target, np.float64) - tmean) / tstd                            # n x O
    a1 = x @ p["W1"].T + p["b1"]
    h1 = h16(np.maximum(a1, 0.0), emulate_fp16)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = h16(np.maximum(a2, 0.0), emulate_fp16)
    out = h2 @ p["W3"].T + p["b3"]
    n = x.shape[0]
    e = out - y
    loss = float((e ** 2).sum() / (n * O))
    g_out = 2.0 * e / (n * O)
    g = {"W3": g_out.T @ h2, "b3": g_out.sum(0)}
    g_h2 = (g_out @ p["W3"]) * (h2 > 0)
    g["W2"] = g_h2.T @ h1
    g["b2"] = g_h2.sum(0)
    g_h1 = (g_h2 @ p["W2"]) * (h1 > 0)
    g["W1"] = g_h1.T @ x
    g["b1"] = g_h1.sum(0)
    grad = np.concatenate([g[name].ravel() for name, _ in SIZES])
    return loss, grad
