"""Batched multi-beam search (gsp_batch_*): beams with different lengths and DM
grids dedispersed in one launch (one CTA per item, or persistent CTAs), with
and without CUDA-graph replay and autotuning.  Every beam's candidates and
block statistics must equal a separate gsp_search of that beam."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gsp():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_12749_gb300 import build, gsp as g
    build.build()
    g.lib()
    return g


BEAMS = [  # (n_in, dm_lo, dm_step, ndm)
    (40000, 0.0, 1.0, 151),
    (33008, 5.0, 0.7, 80),
    (50016, 0.0, 0.5, 200),
]


def _make(gsp, seed):
    rng = np.random.default_rng(seed)
    nchan = 256
    plans, refs, xs, n_ins = [], [], [], []
    for n_in, lo, step, ndm in BEAMS:
        d, k = gsp.make_desc(nchan, 1200.0, 1500.0, 1e-4, n_in, ndm=ndm, dm_lo=lo, dm_step=step,
                             threshold=5.0)
        plans.append(gsp.gsp_plan_create(d, k))
        d2, k2 = gsp.make_desc(nchan, 1200.0, 1500.0, 1e-4, n_in, ndm=ndm, dm_lo=lo, dm_step=step,
                               threshold=5.0)
        refs.append(gsp.gsp_plan_create(d2, k2))
        stride = (n_in + 15) // 16 * 16
        x = np.round(rng.normal(128, 16, (nchan, stride))).clip(0, 255).astype(np.uint8)
        xs.append(torch.from_numpy(x).cuda())
        n_ins.append(n_in)
    return plans, refs, xs, n_ins


@pytest.mark.parametrize("flags", [0, 1, 7])
def test_batch_equals_single_beam_searches(gsp, flags):
    plans, refs, xs, n_ins = _make(gsp, 5 + flags)
    s = torch.cuda.Stream()
    b = gsp.gsp_batch_create(plans, flags)
    want = []
    for ref, x, n in zip(refs, xs, n_ins):
        gsp.gsp_search(ref, x, n, stream=s)
        c, _, st = gsp.gsp_candidates(ref)
        assert st == gsp.GSP_OK
        want.append(c)
    for rep in range(2):                      # the second call replays the graph
        gsp.gsp_batch_search(b, xs, n_ins, stream=s)
        got, n, st = gsp.gsp_batch_candidates(b)
        assert st == gsp.GSP_OK
        assert n == sum(len(w) for w in want)
        off = 0
        for i, w in enumerate(want):
            g = got[off:off + len(w)]
            off += len(w)
            assert (g["beam"] == i).all()
            for f in ("dm_idx", "t", "width", "snr"):
                assert (g[f] == w[f]).all(), (i, f)
        for p, ref, n_in in zip(plans, refs, n_ins):
            n_out = gsp.gsp_plan_nout(p, n_in)
            a, r = gsp.gsp_search_stats(p, n_out), gsp.gsp_search_stats(ref, n_out)
            assert (a["sigma_b"] == r["sigma_b"]).all()
    v, tuned, nl = gsp.gsp_batch_info(b)
    assert nl > 0
    if flags & 4:
        assert tuned > 0
    gsp.gsp_batch_destroy(b)


def test_batch_rejects_mixed_channels_and_shared_plans(gsp):
    d1, k1 = gsp.make_desc(64, 1200.0, 1500.0, 1e-4, 8192, ndm=8)
    d2, k2 = gsp.make_desc(128, 1200.0, 1500.0, 1e-4, 8192, ndm=8)
    p1, p2 = gsp.gsp_plan_create(d1, k1), gsp.gsp_plan_create(d2, k2)
    with pytest.raises(gsp.GspError):
        gsp.gsp_batch_create([p1, p2])
    with pytest.raises(gsp.GspError):
        gsp.gsp_batch_create([p1, p1])
