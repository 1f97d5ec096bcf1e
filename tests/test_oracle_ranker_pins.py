"""Pins of the ranker oracle (oracle/ranker.py) against what fixes it
independently: hand-worked bfloat16 ties and the library's bfloat16
conversion; direct loops and torch's conv2d / max_pool2d for the layers;
central finite differences of the exact (unrounded) network for every
parameter tensor; the closed form of a first Adam step; hand-built
normalised series for the snippet."""
import math

import numpy as np
import pytest

from oracle import ranker as R


def test_bf16_rounding_hand_cases():
    one = 1.0
    assert R.bf16(np.array([one]))[0] == 1.0
    assert R.bf16(np.array([1 + 2.0 ** -8]))[0] == 1.0               # tie -> even (down)
    assert R.bf16(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6  # tie -> even (up)
    assert R.bf16(np.array([1 + 2.0 ** -8 + 2.0 ** -20]))[0] == 1 + 2.0 ** -7
    assert R.bf16(np.array([-2.5]))[0] == -2.5
    assert R.bf16(np.array([0.0]))[0] == 0.0


def test_bf16_matches_library_conversion():
    torch = pytest.importorskip("torch")
    v = np.random.default_rng(1).standard_normal(20000).astype(np.float32) * 37.0
    lib = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert (R.bf16(v) == lib).all()


def test_conv3x3_direct_loops():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((2, 3, 5, 6))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    z = R.conv3x3(a, w, b, exact=True)
    for bi in range(2):
        for o in range(4):
            for y in range(5):
                for x in range(6):
                    s = b[o]
                    for c in range(3):
                        for ky in range(3):
                            for kx in range(3):
                                yy, xx = y + ky - 1, x + kx - 1
                                if 0 <= yy < 5 and 0 <= xx < 6:
                                    s += a[bi, c, yy, xx] * w[o, c, ky, kx]
                    assert abs(z[bi, o, y, x] - s) < 1e-12


def test_layers_match_library():
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    rng = np.random.default_rng(3)
    a = rng.standard_normal((3, 8, 16, 16))
    w = rng.standard_normal((16, 8, 3, 3))
    b = rng.standard_normal(16)
    ref = F.conv2d(torch.from_numpy(a), torch.from_numpy(w), torch.from_numpy(b), padding=1)
    assert np.abs(R.conv3x3(a, w, b, exact=True) - ref.numpy()).max() < 1e-12
    h = rng.standard_normal((3, 8, 16, 16))
    pooled, idx = R.maxpool2(h)
    assert (pooled == F.max_pool2d(torch.from_numpy(h), 2).numpy()).all()


def test_maxpool_ties_go_to_first():
    h = np.zeros((1, 1, 2, 2))
    _, idx = R.maxpool2(h)
    assert idx[0, 0, 0, 0] == 0
    h[0, 0, 1, 0] = h[0, 0, 1, 1] = 5.0
    pooled, idx = R.maxpool2(h)
    assert pooled[0, 0, 0, 0] == 5.0 and idx[0, 0, 0, 0] == 2
    g = R.maxpool2_backward(np.full((1, 1, 1, 1), 7.0), idx)
    assert g[0, 0].tolist() == [[0.0, 0.0], [7.0, 0.0]]


def test_flatten_order():
    a = np.arange(2 * 32 * 8 * 8, dtype=np.float64).reshape(2, 32, 8, 8)
    f = R.flatten_hwc(a)
    for (bb, c, y, x) in [(0, 0, 0, 0), (1, 5, 3, 7), (0, 31, 7, 7)]:
        assert f[bb, (y * 8 + x) * 32 + c] == a[bb, c, y, x]
    assert (R.unflatten_hwc(f, 32, 8, 8) == a).all()


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(4)
    p = R.init_params(7)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.uniform(-0.05, 0.05, p[k].shape)
    x = rng.standard_normal((2, 64, 64))
    y = np.array([0, 1])
    loss, g = R.loss_and_grad(p, x, y, exact=True)
    assert math.isfinite(loss)
    for name in R.ORDER:
        flat = p[name].reshape(-1)
        for i in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[i]
            h = 1e-6 * max(1.0, abs(old))
            flat[i] = old + h
            lp, _ = R.loss_and_grad(p, x, y, exact=True)
            flat[i] = old - h
            lm, _ = R.loss_and_grad(p, x, y, exact=True)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-5 * max(1e-3, abs(fd)) + 1e-9, (name, i, fd, an)


def test_first_adam_step_closed_form():
    p = {k: np.ones(R.SHAPES[k]) for k in R.ORDER}
    g = {k: np.full(R.SHAPES[k], -0.25) for k in R.ORDER}
    m = {k: np.zeros(R.SHAPES[k]) for k in R.ORDER}
    v = {k: np.zeros(R.SHAPES[k]) for k in R.ORDER}
    R.adam_step(p, g, m, v, 1, lr=1e-2)
    # m_hat = g, v_hat = g^2 at the first step: w -= lr * g / (|g| + eps)
    want = 1.0 + 1e-2 * 0.25 / (0.25 + 1e-8)
    for k in R.ORDER:
        assert np.allclose(p[k], want, rtol=0, atol=1e-15)


def test_snippet_hand_built():
    ndm, Ls = 40, 3000
    xn = np.zeros((ndm, Ls))
    xn[10, 1000:1008] = 2.0          # a box of width 8 on row 10
    img = R.snippet(xn, 10, 1000, 8)   # f = 2, tc = 1004
    f = 2
    assert img.shape == (64, 64)
    # row 10 is image row 32; bins j cover [1004 + (j - 32) * 2, +2)
    row = img[32]
    want = np.zeros(64)
    for j in range(64):
        a = 1004 + (j - 32) * f
        want[j] = xn[10, max(a, 0):min(a + f, Ls)].sum() / math.sqrt(f)
    assert np.allclose(row, want)
    assert np.isclose(row.sum(), 16.0 / math.sqrt(2))
    assert (np.delete(img, 32, axis=0) == 0).all()
    # rows outside [0, ndm) are zero, time outside [0, Ls) contributes nothing
    edge = R.snippet(np.ones((5, 100)), 0, 0, 1)
    assert (edge[:32] == 0).all() and (edge[32:37, 32:] == 1).all() and (edge[37:] == 0).all()
    assert (edge[32:37, :32] == 0).all()
    assert R.time_bin(150) == 37 and R.time_bin(3) == 1
