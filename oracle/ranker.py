"""CPU oracle of the candidate ranker: TEST INFRASTRUCTURE.

The paper motivates ranking the many single-pulse candidates of a survey
(Sec. 1 and Sec. 2: candidates are archived and reviewed by astronomers);
this ranker is the project's own design for that step (it ranks the plain
threshold output, never replaces it).  Plain numpy in FP64, written from the
definitions below; only tests, the smoke check and the bench's reference leg
import it.  It shares no code with the CUDA library.

Snippet of a candidate (dm_idx d, start t, width w) from the normalised
series xnorm[row][s] of the search (detrended residual / sigma_ref, bad
blocks zeroed, s < Ls): a 64 x 64 DM-time image
    img[i][j] = sum_{s in bin j, 0 <= s < Ls} xnorm[d - 32 + i][s] / sqrt(f)
with f = max(1, w // 4) samples per time bin, bin j = [tc + (j - 32) f,
tc + (j - 31) f), tc = t + w // 2, and rows outside [0, ndm) all zero.

Network (NCHW here; the GPU's layout is its own):
    conv 3x3 pad 1 (1 -> 8) + bias, ReLU, max-pool 2x2      64x64 -> 32x32
    conv 3x3 pad 1 (8 -> 16) + bias, ReLU, max-pool 2x2     -> 16x16
    conv 3x3 pad 1 (16 -> 32) + bias, ReLU, max-pool 2x2    -> 8x8
    fc 2048 -> 96 + bias, ReLU   (feature index (y * 8 + x) * 32 + c)
    fc 96 -> 2 + bias            (logits; class 1 = astrophysical pulse)
Rounding points (the GPU rounds at the same places): every operand of a
product (weights, activations, back-propagated gradients) is rounded to
bfloat16 (round to nearest even); sums, bias, ReLU, pooling, softmax and the
Adam update are exact here (FP32 on the GPU).  Max-pool ties go to the first
element of the window in (0,0), (0,1), (1,0), (1,1) order.  Loss: mean
softmax cross-entropy.  Adam: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
w -= lr * (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps).
"""
import math

import numpy as np

SNIP = 64
SHAPES = {"w1": (8, 1, 3, 3), "b1": (8,), "w2": (16, 8, 3, 3), "b2": (16,),
          "w3": (32, 16, 3, 3), "b3": (32,), "w4": (96, 2048), "b4": (96,),
          "w5": (2, 96), "b5": (2,)}
ORDER = ("w1", "b1", "w2", "b2", "w3", "b3", "w4", "b4", "w5", "b5")


def bf16(x):
    """Round to bfloat16 (nearest, ties to even) and return as float64.  The
    value is first rounded to float32 (the GPU's storage type)."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(a.shape)


def time_bin(w):
    return max(1, int(w) // 4)


def snippet(xnorm, d, t, w):
    """64 x 64 DM-time image of a candidate; xnorm: float [ndm][Ls]."""
    ndm, Ls = xnorm.shape
    f = time_bin(w)
    tc = int(t) + int(w) // 2
    img = np.zeros((SNIP, SNIP))
    for i in range(SNIP):
        r = int(d) - SNIP // 2 + i
        if r < 0 or r >= ndm:
            continue
        for j in range(SNIP):
            a = tc + (j - SNIP // 2) * f
            lo, hi = max(a, 0), min(a + f, Ls)
            if hi > lo:
                img[i, j] = xnorm[r, lo:hi].sum() / math.sqrt(f)
    return img


def init_params(seed):
    """He-uniform weights, zero biases (float32 values, as on the GPU)."""
    rng = np.random.default_rng(seed)
    p = {}
    for k in ORDER:
        s = SHAPES[k]
        if k.startswith("b"):
            p[k] = np.zeros(s)
        else:
            fan_in = int(np.prod(s[1:]))
            lim = math.sqrt(6.0 / fan_in)
            p[k] = rng.uniform(-lim, lim, s).astype(np.float32).astype(np.float64)
    return p


# ------------------------------------------------------------- layer pieces

def conv3x3(a, w, b, exact=False):
    """z[b,o,y,x] = sum_{c,ky,kx} a[b,c,y+ky-1,x+kx-1] w[o,c,ky,kx] + bias[o]."""
    r = (lambda v: v) if exact else bf16
    a, w = r(a), r(w)
    B, C, H, W = a.shape
    ap = np.zeros((B, C, H + 2, W + 2))
    ap[:, :, 1:-1, 1:-1] = a
    z = np.zeros((B, w.shape[0], H, W))
    for ky in range(3):
        for kx in range(3):
            z += np.einsum("bcyx,oc->boyx", ap[:, :, ky:ky + H, kx:kx + W], w[:, :, ky, kx])
    return z + b[None, :, None, None]


def conv3x3_backward(g, a, w, exact=False):
    """Gradients of conv3x3 w.r.t. its input and weights, for output gradient g."""
    r = (lambda v: v) if exact else bf16
    g, a, w = r(g), r(a), r(w)
    B, C, H, W = a.shape
    ap = np.zeros((B, C, H + 2, W + 2))
    ap[:, :, 1:-1, 1:-1] = a
    dw = np.zeros_like(w)
    dap = np.zeros_like(ap)
    for ky in range(3):
        for kx in range(3):
            dw[:, :, ky, kx] = np.einsum("boyx,bcyx->oc", g, ap[:, :, ky:ky + H, kx:kx + W])
            dap[:, :, ky:ky + H, kx:kx + W] += np.einsum("boyx,oc->bcyx", g, w[:, :, ky, kx])
    return dap[:, :, 1:-1, 1:-1], dw


def maxpool2(h):
    """2x2 max-pool; returns the pooled map and the argmax index (0..3) per output."""
    B, C, H, W = h.shape
    v = np.stack([h[:, :, 0::2, 0::2], h[:, :, 0::2, 1::2], h[:, :, 1::2, 0::2],
                  h[:, :, 1::2, 1::2]], axis=0)
    idx = np.argmax(v, axis=0)          # first maximum wins ties
    return np.take_along_axis(v, idx[None], axis=0)[0], idx


def maxpool2_backward(gp, idx):
    B, C, H2, W2 = gp.shape
    gh = np.zeros((B, C, 2 * H2, 2 * W2))
    for k, (dy, dx) in enumerate(((0, 0), (0, 1), (1, 0), (1, 1))):
        gh[:, :, dy::2, dx::2] = np.where(idx == k, gp, 0.0)
    return gh


def flatten_hwc(a):
    """[B, C, 8, 8] -> [B, 2048] with feature index (y * 8 + x) * C + c."""
    return np.ascontiguousarray(a.transpose(0, 2, 3, 1)).reshape(a.shape[0], -1)


def unflatten_hwc(f, C, H, W):
    return f.reshape(f.shape[0], H, W, C).transpose(0, 3, 1, 2)


# -------------------------------------------------------------- the network

def forward(p, x, exact=False):
    """x: [B, 64, 64] snippets.  Returns the logits and the tape for backward."""
    r = (lambda v: v) if exact else bf16
    t = {"a0": x[:, None, :, :].astype(np.float64)}
    a = t["a0"]
    for l in (1, 2, 3):
        z = conv3x3(a, p["w%d" % l], p["b%d" % l], exact)
        pooled, idx = maxpool2(np.maximum(z, 0.0))
        t["z%d" % l], t["idx%d" % l], t["in%d" % l] = z, idx, a
        a = r(pooled)
    t["a3"] = a
    f3 = flatten_hwc(a)
    z4 = r(f3) @ r(p["w4"]).T + p["b4"]
    a4 = r(np.maximum(z4, 0.0))
    z5 = a4 @ r(p["w5"]).T + p["b5"]
    t.update(f3=f3, z4=z4, a4=a4)
    return z5, t


def loss_and_grad(p, x, y, exact=False):
    """Mean softmax cross-entropy of labels y (0/1) and the gradient of every
    parameter, following the rounding points of the module docstring."""
    r = (lambda v: v) if exact else bf16
    z5, t = forward(p, x, exact)
    B = x.shape[0]
    zm = z5 - z5.max(axis=1, keepdims=True)
    e = np.exp(zm)
    sm = e / e.sum(axis=1, keepdims=True)
    loss = float(-np.mean(np.log(sm[np.arange(B), y])))
    g5 = sm.copy()
    g5[np.arange(B), y] -= 1.0
    g5 /= B
    g = {}
    g["w5"] = r(g5).T @ t["a4"]
    g["b5"] = g5.sum(axis=0)
    ga4 = r(g5) @ r(p["w5"])
    g4 = ga4 * (t["z4"] > 0)
    g["w4"] = r(g4).T @ r(t["f3"])
    g["b4"] = g4.sum(axis=0)
    ga = unflatten_hwc(r(g4) @ r(p["w4"]), 32, 8, 8)
    for l in (3, 2, 1):
        gh = maxpool2_backward(ga, t["idx%d" % l])
        gz = gh * (t["z%d" % l] > 0)
        da, dw = conv3x3_backward(gz, t["in%d" % l], p["w%d" % l], exact)
        g["w%d" % l] = dw
        g["b%d" % l] = gz.sum(axis=(0, 2, 3))
        ga = da
    return loss, g


def adam_step(p, g, m, v, k, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step number k >= 1) of every parameter, in place."""
    for name in ORDER:
        m[name] = b1 * m[name] + (1 - b1) * g[name]
        v[name] = b2 * v[name] + (1 - b2) * g[name] ** 2
        mh = m[name] / (1 - b1 ** k)
        vh = v[name] / (1 - b2 ** k)
        p[name] = p[name] - lr * mh / (np.sqrt(vh) + eps)


def scores(p, x):
    """Ranking score: softmax probability of class 1."""
    z5, _ = forward(p, x)
    zm = z5 - z5.max(axis=1, keepdims=True)
    e = np.exp(zm)
    return e[:, 1] / e.sum(axis=1)
