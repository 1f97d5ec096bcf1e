"""GPU parity of the candidate ranker against its CPU oracle (oracle/ranker.py),
through the C ABI: candidate snippets from a real search; forward logits,
every parameter's gradient and three Adam steps from the same parameters;
and a small learning check.  The GPU rounds to bf16 at the oracle's points
and accumulates in FP32 where the oracle uses FP64, so the comparisons are
relative (the tolerances are stated per test)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import ranker as R  # noqa: E402


@pytest.fixture(scope="module")
def gsp():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_12749_gb300 import build, gsp as g
    build.build()
    g.lib()
    return g


def _flat(p):
    return np.concatenate([np.asarray(p[k], np.float64).reshape(-1) for k in R.ORDER])


def _split(v):
    out, o = {}, 0
    for k in R.ORDER:
        n = int(np.prod(R.SHAPES[k]))
        out[k] = v[o:o + n].reshape(R.SHAPES[k]).astype(np.float64)
        o += n
    return out


def _batch(n, seed):
    """Snippet-like inputs: unit noise, half with a bright dispersed-pulse blob."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 64, 64)).astype(np.float32)
    y = (rng.random(n) < 0.5).astype(np.int32)
    ii, jj = np.mgrid[0:64, 0:64]
    for k in np.nonzero(y)[0]:
        a = rng.uniform(2.0, 6.0)
        x[k] += (a * np.exp(-((jj - 32 - 0.2 * (ii - 32)) ** 2) / 4.0 - (ii - 32) ** 2 / 200.0)
                 ).astype(np.float32)
    return x, y


def test_snippets_match_oracle(gsp, orc):
    from paper_2110_12749_gb300 import synth
    wl = synth.WORKLOADS["tiny"]
    dl, _ = orc.delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.dms)
    n_out = wl.n_in - orc.max_delay(dl)
    x, _, _, _ = synth.workload_filterbank(
        wl, lambda dm: orc.delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, [dm])[0][0], n_out)
    desc, keep = gsp.make_desc(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_in, ndm=wl.ndm,
                               dm_lo=wl.dm_lo, dm_step=wl.dm_step, threshold=4.0)
    plan = gsp.gsp_plan_create(desc, keep)
    D = torch.zeros((wl.ndm, (n_out + 3) // 4 * 4), dtype=torch.int32, device="cuda")
    gsp.gsp_search(plan, torch.from_numpy(x).cuda(), wl.n_in, out=D)
    cands, n, st = gsp.gsp_candidates(plan)
    assert st == gsp.GSP_OK and n > 10
    cands = cands[:200]
    dc = torch.from_numpy(cands.view(np.uint8).copy()).cuda()
    out = torch.zeros((len(cands), 64, 64), dtype=torch.float32, device="cuda")
    gsp.gsp_ranker_snippets(plan, D, dc, out)
    got = out.cpu().numpy()
    Dref = orc.dedisperse(x, wl.n_in, dl)
    xn = np.stack([orc.search_row(Dref[r], threshold=4.0, detail=True)["xnorm"]
                   for r in range(wl.ndm)])
    for k, c in enumerate(cands):
        ref = R.snippet(xn, c["dm_idx"], c["t"], c["width"])
        tol = 1e-4 * (1.0 + np.abs(ref)) * np.sqrt(R.time_bin(c["width"]))
        assert (np.abs(got[k] - ref) <= tol).all(), (k, float(np.abs(got[k] - ref).max()))


@pytest.mark.parametrize("path,pad", [(1, 0), (1, 1), (2, 0), (2, 1)])
def test_snippets_crafted_candidates(gsp, orc, path, pad):
    """Snippets of placed candidates against the oracle: every default boxcar
    width (f = 1 .. 37) and two wider ones (f = 150 and 300: a row no longer
    fits half of the kernel's shared-memory ring), at the start and end of the
    searched span (rows whose aligned span leaves the series) and at the first
    and last DM rows (blank rows).  pad = 1 stores D with a row stride that is
    not a multiple of four samples, so that every row is read directly instead
    of by bulk copies; the sums must not change.  path 1 sums the samples of D
    (the direct path), path 2 differences of block-local prefix sums; both
    paths must give the same floats."""
    from paper_2110_12749_gb300 import synth
    wl = synth.WORKLOADS["tiny"]
    dl, _ = orc.delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.dms)
    n_out = wl.n_in - orc.max_delay(dl)
    x, _, _, _ = synth.workload_filterbank(
        wl, lambda dm: orc.delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, [dm])[0][0], n_out)
    desc, keep = gsp.make_desc(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_in, ndm=wl.ndm,
                               dm_lo=wl.dm_lo, dm_step=wl.dm_step, threshold=4.0)
    plan = gsp.gsp_plan_create(desc, keep)
    D4 = torch.zeros((wl.ndm, (n_out + 3) // 4 * 4), dtype=torch.int32, device="cuda")
    gsp.gsp_search(plan, torch.from_numpy(x).cuda(), wl.n_in, out=D4)
    D = torch.zeros((wl.ndm, D4.shape[1] + pad), dtype=torch.int32, device="cuda")
    D[:, :D4.shape[1]] = D4
    Dref = orc.dedisperse(x, wl.n_in, dl)
    xn = np.stack([orc.search_row(Dref[r], threshold=4.0, detail=True)["xnorm"]
                   for r in range(wl.ndm)])
    Ls = xn.shape[1]
    widths = [1, 2, 3, 4, 6, 9, 14, 20, 30, 45, 70, 100, 150, 600, 1200]
    times = [0, 3, 777, Ls // 2 + 1, Ls - 2300, Ls - 40, Ls - 1]
    rows = [0, 17, wl.ndm // 2, wl.ndm - 1]
    recs = [(d, w, t) for d in rows for w in widths for t in times]
    cands = np.zeros(len(recs), dtype=gsp.CAND_DTYPE)
    for k, (d, w, t) in enumerate(recs):
        cands[k]["dm_idx"], cands[k]["width"], cands[k]["t"] = d, w, t
        cands[k]["snr"] = 5.0
    dc = torch.from_numpy(cands.view(np.uint8).copy()).cuda()
    outs = {}
    for pth in (path, 3 - path):
        gsp.gsp_plan_set_snippet_path(plan, pth)
        out = torch.full((len(cands), 64, 64), 7.0, dtype=torch.float32, device="cuda")
        gsp.gsp_ranker_snippets(plan, D, dc, out)
        torch.cuda.synchronize()
        outs[pth] = out.cpu().numpy()
    assert np.array_equal(outs[1], outs[2])
    got = outs[path]
    for k, c in enumerate(cands):
        ref = R.snippet(xn, c["dm_idx"], c["t"], c["width"])
        tol = 1e-4 * (1.0 + np.abs(ref)) * np.sqrt(R.time_bin(c["width"]))
        assert (np.abs(got[k] - ref) <= tol).all(), (recs[k], float(np.abs(got[k] - ref).max()))
    gsp.gsp_plan_destroy(plan)


def test_snippet_prefix_follows_new_searches(gsp, orc):
    """The prefix sums are rebuilt after every search: snippets of the same
    candidates from two different beams searched by one plan match the oracle
    of each beam (path 2 forced)."""
    from paper_2110_12749_gb300 import synth
    wl = synth.WORKLOADS["tiny"]
    dl, _ = orc.delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.dms)
    n_out = wl.n_in - orc.max_delay(dl)
    desc, keep = gsp.make_desc(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_in, ndm=wl.ndm,
                               dm_lo=wl.dm_lo, dm_step=wl.dm_step, threshold=4.0)
    plan = gsp.gsp_plan_create(desc, keep)
    gsp.gsp_plan_set_snippet_path(plan, 2)
    D = torch.zeros((wl.ndm, (n_out + 3) // 4 * 4), dtype=torch.int32, device="cuda")
    recs = [(wl.ndm // 2, 100, 5000), (40, 30, 12000), (150, 9, 20001)]
    cands = np.zeros(len(recs), dtype=gsp.CAND_DTYPE)
    for k, (d, w, t) in enumerate(recs):
        cands[k]["dm_idx"], cands[k]["width"], cands[k]["t"] = d, w, t
    dc = torch.from_numpy(cands.view(np.uint8).copy()).cuda()
    for beam in (0, 1):
        x, _, _, _ = synth.workload_filterbank(
            wl, lambda dm: orc.delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, [dm])[0][0], n_out,
            beam=beam)
        gsp.gsp_search(plan, torch.from_numpy(x).cuda(), wl.n_in, out=D)
        out = torch.zeros((len(cands), 64, 64), dtype=torch.float32, device="cuda")
        gsp.gsp_ranker_snippets(plan, D, dc, out)
        got = out.cpu().numpy()
        Dref = orc.dedisperse(x, wl.n_in, dl)
        rows = sorted({r for d, _, _ in recs for r in range(max(d - 32, 0), min(d + 32, wl.ndm))})
        xr = {r: orc.search_row(Dref[r], threshold=4.0, detail=True)["xnorm"] for r in rows}
        xn = np.zeros((wl.ndm, len(xr[rows[0]])))
        for r in rows:
            xn[r] = xr[r]
        for k, c in enumerate(cands):
            ref = R.snippet(xn, c["dm_idx"], c["t"], c["width"])
            tol = 1e-4 * (1.0 + np.abs(ref)) * np.sqrt(R.time_bin(c["width"]))
            assert (np.abs(got[k] - ref) <= tol).all(), (beam, recs[k])
    gsp.gsp_plan_destroy(plan)


@pytest.mark.parametrize("n", [37, 130])
def test_forward_matches_oracle(gsp, n):
    p = R.init_params(11)
    r = gsp.gsp_ranker_create(256, seed=3)
    gsp.gsp_ranker_set_params(r, _flat(p))
    x, _ = _batch(n, n)
    logits = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    gsp.gsp_ranker_forward(r, torch.from_numpy(x).cuda(), n, logits)
    gsp.gsp_ranker_finish(r)
    # three fused conv + pool layers, fc1 split-K GEMM and its ordered sum, fc2
    assert gsp.gsp_ranker_launches(r) == 6
    got = logits.cpu().numpy().astype(np.float64)
    ref, _ = R.forward(p, x.astype(np.float64))
    err = np.abs(got - ref)
    # FP32 vs FP64 accumulation; a bf16 rounding flip changes one operand by 2^-8
    assert np.median(err) < 1e-4 * max(1.0, np.abs(ref).max())
    assert err.max() < 1e-2 * max(1.0, np.abs(ref).max())


def test_inference_and_training_passes_agree(gsp):
    """The fused inference pass and the im2col training pass round at the same
    points: the cross-entropy of the inference logits equals the training
    step's loss (lr 0) up to FP32 summation order."""
    p = R.init_params(14)
    n = 200
    x, y = _batch(n, 8)
    r = gsp.gsp_ranker_create(256, seed=6)
    gsp.gsp_ranker_set_params(r, _flat(p))
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    logits = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    gsp.gsp_ranker_forward(r, xd, n, logits)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gsp.gsp_ranker_train_step(r, xd, yd, n, 0.0, loss=loss)
    gsp.gsp_ranker_finish(r)
    ce = float(torch.nn.functional.cross_entropy(logits.double().cpu(),
                                                 torch.from_numpy(y).long()))
    assert abs(ce - float(loss.item())) <= 1e-4 * max(1.0, ce), (ce, float(loss.item()))


def test_gradients_match_oracle(gsp):
    p = R.init_params(12)
    rng = np.random.default_rng(5)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.uniform(-0.05, 0.05, p[k].shape).astype(np.float32).astype(np.float64)
    n = 96
    x, y = _batch(n, 6)
    r = gsp.gsp_ranker_create(128, seed=4)
    gsp.gsp_ranker_set_params(r, _flat(p))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gsp.gsp_ranker_train_step(r, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), n, 0.0,
                              loss=loss)
    gsp.gsp_ranker_finish(r)
    params, grads = gsp.gsp_ranker_get_params(r)
    assert np.array_equal(params, _flat(p).astype(np.float32))       # lr 0: unchanged
    ref_loss, ref_g = R.loss_and_grad(p, x.astype(np.float64), y)
    assert abs(float(loss.item()) - ref_loss) < 1e-4 * max(1.0, ref_loss)
    g = _split(grads)
    for k in R.ORDER:
        num = np.linalg.norm(g[k] - ref_g[k])
        den = np.linalg.norm(ref_g[k])
        assert num <= 1e-2 * den + 1e-7, (k, num, den)


def test_adam_steps_match_oracle(gsp):
    p = R.init_params(13)
    n, lr = 64, 1e-3
    x, y = _batch(n, 7)
    r = gsp.gsp_ranker_create(64, seed=5)
    gsp.gsp_ranker_set_params(r, _flat(p))
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    m = {k: np.zeros(R.SHAPES[k]) for k in R.ORDER}
    v = {k: np.zeros(R.SHAPES[k]) for k in R.ORDER}
    for step in range(1, 4):
        gsp.gsp_ranker_train_step(r, xd, yd, n, lr)
        _, g = R.loss_and_grad(p, x.astype(np.float64), y)
        R.adam_step(p, g, m, v, step, lr=lr)
    gsp.gsp_ranker_finish(r)
    got, _ = gsp.gsp_ranker_get_params(r)
    diff = np.abs(got.astype(np.float64) - _flat(p))
    # Adam's first steps move each weight by about lr * sign(g); a gradient
    # component near 0 may take the other sign on the GPU: allow 1% of weights
    assert np.mean(diff > 0.1 * lr) < 0.01, np.mean(diff > 0.1 * lr)
    assert np.median(diff) < 1e-2 * lr


def test_ranker_learns_pulse_shape(gsp):
    r = gsp.gsp_ranker_create(256, seed=9)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    first = None
    for it in range(150):
        x, y = _batch(256, 100 + it)
        gsp.gsp_ranker_train_step(r, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), 256,
                                  2e-3, loss=loss)
        if it == 0:
            gsp.gsp_ranker_finish(r)
            first = float(loss.item())
    gsp.gsp_ranker_finish(r)
    assert float(loss.item()) < 0.5 * first
    x, y = _batch(256, 999)
    logits = torch.zeros((256, 2), dtype=torch.float32, device="cuda")
    gsp.gsp_ranker_forward(r, torch.from_numpy(x).cuda(), 256, logits)
    gsp.gsp_ranker_finish(r)
    pred = logits.argmax(dim=1).cpu().numpy()
    assert np.mean(pred == y) > 0.95


# ---------------------------------------------------------------------------
# Stage by stage, element by element.  Each stage of the GPU network is fed
# the GPU's own inputs of that stage (read back with gsp_ranker_tensor) and
# compared with the oracle's value of the same stage from those inputs.  The
# bound of every element is derived from the arithmetic: an FP32 sum of K
# products (+ bias) is within (K + 2) u sum|terms| of the exact sum (u = 2^-24,
# any summation order, tensor-core or FMA chain), max-pool and ReLU do not
# increase an error, and one rounding to bf16 moves a value by at most
# 2^-8 of its magnitude.

U32 = 2.0 ** -24
BF = 2.0 ** -8


def _nchw(t, n, side, c):
    return t.reshape(n, side, side, c).transpose(0, 3, 1, 2)


def _within(got, ref, bound, what):
    d = np.abs(got - ref)
    bad = d > bound
    assert not bad.any(), "%s: %d of %d elements out of bound, worst %.3g vs bound %.3g" % (
        what, int(bad.sum()), bad.size, float(d[bad].max()), float(bound[bad][np.argmax(d[bad])]))


def _conv_stage(p, l, a_in, got_pooled, got_z=None):
    """Layer l (1..3) from the GPU's input a_in (NCHW): returns the GPU's pooled
    output checked against the oracle (and the pre-pool ReLU output if given)."""
    w, b = p["w%d" % l], p["b%d" % l]
    K = 9 * a_in.shape[1]
    z = R.conv3x3(a_in, w, b)                                     # exact sum of bf16 products
    za = R.conv3x3(np.abs(R.bf16(a_in)), np.abs(R.bf16(w)), np.abs(b), exact=True)
    err = (K + 2) * U32 * za                                      # FP32 sum error bound
    if got_z is not None:
        _within(got_z, np.maximum(z, 0.0), err, "z%d" % (l - 1))
    v, _ = R.maxpool2(np.maximum(z, 0.0))
    e2, _ = R.maxpool2(err)                                       # the pool's error: max over window
    _within(got_pooled, v, BF * np.abs(v) + e2 * (1 + BF), "a%d" % (l - 1))


def _params_with_biases(seed):
    p = R.init_params(seed)
    rng = np.random.default_rng(seed)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.uniform(-0.05, 0.05, p[k].shape).astype(np.float32).astype(np.float64)
    return p


@pytest.mark.parametrize("train", [False, True])
def test_forward_stages_element_by_element(gsp, train):
    p = _params_with_biases(31)
    n = 40
    x, y = _batch(n, 17)
    r = gsp.gsp_ranker_create(64, seed=2)
    gsp.gsp_ranker_set_params(r, _flat(p))
    xd = torch.from_numpy(x).cuda()
    if train:
        gsp.gsp_ranker_train_step(r, xd, torch.from_numpy(y).cuda(), n, 0.0)
    else:
        gsp.gsp_ranker_forward(r, xd, n, torch.zeros((n, 2), dtype=torch.float32, device="cuda"))
    gsp.gsp_ranker_finish(r)
    a_in = x[:, None, :, :].astype(np.float64)
    for l, (side, c) in enumerate([(64, 8), (32, 16), (16, 32)]):
        got = _nchw(gsp.gsp_ranker_tensor(r, "a%d" % l), n, side // 2, c)
        gz = _nchw(gsp.gsp_ranker_tensor(r, "z%d" % l), n, side, c) if train else None
        _conv_stage(p, l + 1, a_in, got, gz)
        a_in = got
    f3 = R.flatten_hwc(a_in)
    z4 = gsp.gsp_ranker_tensor(r, "z4").reshape(n, -1)                 # after ReLU
    ref4 = np.maximum(f3 @ R.bf16(p["w4"]).T + p["b4"], 0.0)
    err4 = (f3.shape[1] + 2) * U32 * (np.abs(f3) @ np.abs(R.bf16(p["w4"])).T + np.abs(p["b4"]))
    _within(z4, ref4, err4, "z4")
    a4 = gsp.gsp_ranker_tensor(r, "a4").reshape(n, -1)
    assert (a4 == R.bf16(np.maximum(z4, 0.0))).all()             # the epilogue's own rounding
    z5 = gsp.gsp_ranker_tensor(r, "z5").reshape(n, 2)
    ref5 = a4 @ R.bf16(p["w5"]).T + p["b5"]
    err5 = (a4.shape[1] + 2) * U32 * (np.abs(a4) @ np.abs(R.bf16(p["w5"])).T + np.abs(p["b5"]))
    _within(z5, ref5, err5, "z5")
    gsp.gsp_ranker_destroy(r)


def test_backward_stages_element_by_element(gsp):
    p = _params_with_biases(32)
    n = 40
    x, y = _batch(n, 18)
    r = gsp.gsp_ranker_create(64, seed=2)
    gsp.gsp_ranker_set_params(r, _flat(p))
    gsp.gsp_ranker_train_step(r, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), n, 0.0)
    gsp.gsp_ranker_finish(r)
    T = {k: gsp.gsp_ranker_tensor(r, k) for k in
         ("a0", "a1", "a2", "z0", "z1", "z2", "idx0", "idx1", "idx2", "z4", "a4", "z5", "g5",
          "g4", "ga0", "ga1", "ga2", "gz0", "gz1", "gz2")}
    _, grads = gsp.gsp_ranker_get_params(r)
    G = _split(grads)
    # the loss gradient w.r.t. the logits, from the GPU's logits
    z5 = T["z5"].reshape(n, 2)
    e = np.exp(z5 - z5.max(1, keepdims=True))
    sm = e / e.sum(1, keepdims=True)
    g5 = sm.copy()
    g5[np.arange(n), y] -= 1.0
    g5 /= n
    got5 = T["g5"].reshape(n, 2)
    _within(got5, g5, 16 * U32 * (sm + 1.0) / n, "g5")
    # fc 96 -> 2 backward from the GPU's g5 and a4
    a4 = T["a4"].reshape(n, -1)
    gb5 = R.bf16(got5)
    _within(G["w5"], gb5.T @ a4, (n + 2) * U32 * (np.abs(gb5).T @ np.abs(a4)), "dw5")
    _within(G["b5"], got5.sum(0), (n + 2) * U32 * np.abs(got5).sum(0), "db5")
    w5 = R.bf16(p["w5"])
    z4 = T["z4"].reshape(n, -1)
    u4 = (gb5 @ w5) * (z4 > 0)
    t4 = (np.abs(gb5) @ np.abs(w5)) * (z4 > 0)
    g4 = T["g4"].reshape(n, -1)
    _within(g4, u4, BF * np.abs(u4) + 4 * U32 * t4 * (1 + BF), "g4")
    # fc 2048 -> 96 backward from the GPU's g4 and pooled layer-3 output
    f3 = R.flatten_hwc(_nchw(T["a2"], n, 8, 32))
    _within(G["w4"], g4.T @ f3, (n + 2) * U32 * (np.abs(g4).T @ np.abs(f3)), "dw4")
    _within(G["b4"], u4.sum(0), (n + 2) * U32 * np.abs(u4).sum(0) + 4 * U32 * t4.sum(0), "db4")
    w4 = R.bf16(p["w4"])
    ga = g4 @ w4
    _within(T["ga2"].reshape(n, -1), ga, (w4.shape[0] + 2) * U32 * (np.abs(g4) @ np.abs(w4)),
            "ga2")
    # the conv layers, from the GPU's ga, argmax, pre-pool output and inputs
    ins = [x[:, None, :, :].astype(np.float64), _nchw(T["a0"], n, 32, 8),
           _nchw(T["a1"], n, 16, 16)]
    for l, (side, c) in reversed(list(enumerate([(64, 8), (32, 16), (16, 32)]))):
        gpool = _nchw(T["ga%d" % l], n, side // 2, c)
        idx = _nchw(T["idx%d" % l].astype(np.int64), n, side // 2, c)
        zl = _nchw(T["z%d" % l], n, side, c)
        v = R.maxpool2_backward(gpool, idx) * (zl > 0)            # routed, exact in FP32
        gz = _nchw(T["gz%d" % l], n, side, c)
        assert (gz == R.bf16(v)).all(), "gz%d" % l
        w = p["w%d" % (l + 1)]
        da, dw = R.conv3x3_backward(gz, ins[l], w)
        da_abs, dw_abs = R.conv3x3_backward(np.abs(gz), np.abs(R.bf16(ins[l])), np.abs(R.bf16(w)),
                                            exact=True)
        P = n * side * side
        _within(G["w%d" % (l + 1)], dw, (P + 2) * U32 * dw_abs, "dw%d" % (l + 1))
        _within(G["b%d" % (l + 1)], v.sum(axis=(0, 2, 3)),
                (P + 2) * U32 * np.abs(v).sum(axis=(0, 2, 3)), "db%d" % (l + 1))
        if l > 0:
            _within(_nchw(T["ga%d" % (l - 1)], n, side, ins[l].shape[1]), da,
                    (c + 9 + 2) * U32 * da_abs, "ga%d" % (l - 1))
    gsp.gsp_ranker_destroy(r)
