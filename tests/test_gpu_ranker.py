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


@pytest.mark.parametrize("n", [37, 130])
def test_forward_matches_oracle(gsp, n):
    p = R.init_params(11)
    r = gsp.gsp_ranker_create(256, seed=3)
    gsp.gsp_ranker_set_params(r, _flat(p))
    x, _ = _batch(n, n)
    logits = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    gsp.gsp_ranker_forward(r, torch.from_numpy(x).cuda(), n, logits)
    gsp.gsp_ranker_finish(r)
    # three fused conv + pool layers, fc1 GEMM, fc2
    assert gsp.gsp_ranker_launches(r) == 5
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
