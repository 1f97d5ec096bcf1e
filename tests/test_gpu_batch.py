"""Batched multi-beam search (gsp_batch_*): beams with different lengths and DM
grids dedispersed in one launch (one CTA per item, or persistent CTAs), with
and without CUDA-graph replay and autotuning.

Small cases: every beam's candidates and block statistics must equal a
separate gsp_search of that beam.  Full shape: 19 beams of 4096 channels with
lengths uniform in 2^18..2^20 samples and their own DM grids (1000-2500 trials
to DM 500-1500, one beam the coarsest step, 1000 trials to DM 1500) in one
persistent, graph-captured, autotuned batch, checked against the CPU oracle:
every row of every beam through the exact prefix-sum identities, sampled rows
bit-exact, and the candidates of the sampled rows against the oracle search.
"""
import numpy as np
import pytest

from helpers import compare_candidates, window_contenders

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


def test_batch_full_shape_against_oracle(gsp, orc):
    import dataclasses
    from paper_2110_12749_gb300 import synth
    wl = synth.WORKLOADS["crafts"]
    rng = np.random.default_rng(synth.BASE_SEED + 31)
    nbeams = 19
    beams = []
    for b in range(nbeams):
        n_in = int(rng.integers(1 << 18, (1 << 20) + 1)) // 16 * 16
        if b == 7:
            ntr, dmax = 1000, 1500.0        # the coarsest grid of the recipe (step 1.5)
        else:
            ntr, dmax = int(rng.integers(1000, 2501)), float(rng.uniform(500.0, 1500.0))
        beams.append((n_in, ntr, dmax / ntr))
    plans, xs, expect = [], [], []
    for b, (n_in, ntr, step) in enumerate(beams):
        dms = np.arange(ntr) * step
        dl, _ = orc.delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, dms)
        n_out = n_in - orc.max_delay(dl)
        wlb = dataclasses.replace(wl, n_in=n_in, ndm=ntr, dm_step=step, n_pulses=10,
                                  pulse_dm=(10.0, ntr * step), pulse_w=(1, 150),
                                  pulse_snr=(5.0, 40.0))
        x, _, _, pulses = synth.workload_filterbank(
            wlb, lambda dm: orc.delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, [dm])[0][0],
            n_out, beam=b)
        # expected values, computed now so that the host copy can go
        s0, s1 = orc.row_sums(x, n_in, dl, n_out)
        rows = {0, ntr - 1, int(rng.integers(0, ntr))}
        p = pulses[int(rng.integers(0, len(pulses)))]
        rows.add(min(max(int(round(p.dm / step)), 0), ntr - 1))
        rows = np.array(sorted(rows))
        Dref = orc.dedisperse(x, n_in, dl, rows=rows, n_out=n_out)
        expect.append((n_out, s0, s1, rows, Dref))
        desc, keep = gsp.make_desc(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, n_in, ndm=ntr,
                                   dm_step=step, max_cands=ntr * (n_out // 1024 + 2))
        plans.append(gsp.gsp_plan_create(desc, keep))
        assert (gsp.gsp_plan_delays(plans[-1]) == dl).all()
        xs.append(torch.from_numpy(x).cuda())
        del x
    s = torch.cuda.Stream()
    flags = gsp.GSP_BATCH_PERSISTENT | gsp.GSP_BATCH_GRAPH | gsp.GSP_BATCH_AUTOTUNE
    bt = gsp.gsp_batch_create(plans, flags)
    n_ins = [b[0] for b in beams]
    gsp.gsp_batch_search(bt, xs, n_ins, stream=s)        # autotune + capture + run
    gsp.gsp_batch_search(bt, xs, n_ins, stream=s)        # graph replay
    cands, ncand, st = gsp.gsp_batch_candidates(bt)
    assert st == gsp.GSP_OK
    variant, tuned, _ = gsp.gsp_batch_info(bt)
    assert variant >= 0 and tuned > 0
    assert len(gsp.gsp_batch_tune_results(bt)) >= 2
    del xs
    torch.cuda.empty_cache()
    for b, (plan, (n_out, s0, s1, rows, Dref)) in enumerate(zip(plans, expect)):
        D = gsp.gsp_plan_series_tensor(plan)
        assert D.shape[1] == n_out
        t = torch.arange(n_out, device="cuda", dtype=torch.int64)
        g0, g1 = [], []
        for r0 in range(0, D.shape[0], 128):
            blk = D[r0:r0 + 128].to(torch.int64)
            g0.append(blk.sum(1))
            g1.append((blk * t).sum(1))
        g0, g1 = torch.cat(g0).cpu().numpy(), torch.cat(g1).cpu().numpy()
        assert (g0 == s0).all(), (b, np.nonzero(g0 != s0)[0][:5])
        assert (g1 == s1).all(), (b, np.nonzero(g1 != s1)[0][:5])
        Dg = D[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.int64)
        assert (Dg == Dref).all(), b
        contenders, ora = {}, []
        for i, r in enumerate(rows):
            det = orc.search_row(Dref[i], dm_idx=int(r), detail=True)
            contenders[int(r)] = window_contenders(det, 1024, 0, 6.0)
            ora.append(det["cands"])
        mine = cands[cands["beam"] == b]
        ncmp, bad = compare_candidates(mine, np.concatenate(ora), 6.0, 1024, 0, contenders,
                                       rows=set(rows.tolist()))
        assert not bad, (b, bad[:5])
    gsp.gsp_batch_destroy(bt)
    for p in plans:
        gsp.gsp_plan_destroy(p)
