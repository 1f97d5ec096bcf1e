"""GPU parity at the full sizes of the CRAFTS-like beam (4096 ch, 2^20 samples,
2000 DMs) and the wide-band variant (2048 ch, 500-3300 MHz, 3000 DMs, max
delay 493269 samples), in the launch configuration the benchmark times.

The oracle cannot dedisperse 8e12 adds, so: (1) every DM row is checked
exactly through the prefix-sum identities sum_t D[t] and sum_t t*D[t]
(computed on the host from channel prefix sums, independent of any
dedispersion); (2) sampled rows (every injected pulse's nearest DM +-1 plus
random rows) are compared bit-exactly with the oracle; (3) on those rows the
S/N of every (width, t), sigma_ref and the candidates are compared with the
FP64 oracle search.
"""
import numpy as np
import pytest

from helpers import compare_candidates, snr_close, window_contenders

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


def _prefix_expect(x, dl, n_out):
    """Exact int64 sum_t D[dm][t] and sum_t t*D[dm][t] for every row from
    channel prefix sums (P_c, Q_c = prefix of u*x[c][u])."""
    ndm, nchan = dl.shape
    s0 = np.zeros(ndm, np.int64)
    s1 = np.zeros(ndm, np.int64)
    u = None
    for c in range(nchan):
        xc = x[c].astype(np.int64)
        if u is None or u.size != xc.size:
            u = np.arange(xc.size, dtype=np.int64)
        P = np.concatenate([[0], np.cumsum(xc)])
        Q = np.concatenate([[0], np.cumsum(xc * u)])
        lo = dl[:, c].astype(np.int64)
        hi = lo + n_out
        dp = P[hi] - P[lo]
        s0 += dp
        s1 += (Q[hi] - Q[lo]) - lo * dp
    return s0, s1


def _gpu_row_sums(D, n_out):
    t = torch.arange(n_out, device=D.device, dtype=torch.int64)
    s0, s1 = [], []
    for r0 in range(0, D.shape[0], 64):
        blk = D[r0:r0 + 64, :n_out].to(torch.int64)
        s0.append(blk.sum(1))
        s1.append((blk * t).sum(1))
    return torch.cat(s0).cpu().numpy(), torch.cat(s1).cpu().numpy()


@pytest.mark.parametrize("name", ["crafts", "wideband"])
def test_full_size_parity(gsp, orc, name):
    from paper_2110_12749_gb300 import synth
    wl = synth.WORKLOADS[name]
    dl, margin = orc.delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.dms)
    n_out = wl.n_in - orc.max_delay(dl)
    x, rfi, bursts, pulses = synth.workload_filterbank(
        wl, lambda dm: orc.delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, [dm])[0][0], n_out)
    nwin = (n_out + 1023) // 1024
    desc, keep = gsp.make_desc(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_in, ndm=wl.ndm,
                               dm_lo=wl.dm_lo, dm_step=wl.dm_step, max_cands=wl.ndm * nwin)
    plan = gsp.gsp_plan_create(desc, keep)
    assert (gsp.gsp_plan_delays(plan) == dl).all()
    _, used = gsp.gsp_dedisperse_variants(plan)
    assert used >= 0          # the tiled kernel, also for the wide band's long sweep
    xd = torch.from_numpy(x).cuda()
    stride = (n_out + 3) // 4 * 4
    D = torch.empty((wl.ndm, stride), dtype=torch.int32, device="cuda")
    gsp.gsp_search(plan, xd, wl.n_in, 0, D)
    cands, ncand, st = gsp.gsp_candidates(plan)
    assert st == gsp.GSP_OK
    stats = gsp.gsp_search_stats(plan, n_out)
    del xd

    # (1) every row: exact prefix-sum identities
    g0, g1 = _gpu_row_sums(D, n_out)
    e0, e1 = orc.row_sums(x, wl.n_in, dl, n_out)
    assert (g0 == e0).all(), np.nonzero(g0 != e0)[0][:10]
    assert (g1 == e1).all(), np.nonzero(g1 != e1)[0][:10]

    # (2) sampled rows, bit-exact
    rng = np.random.default_rng(123)
    rows = set(int(r) for r in rng.choice(wl.ndm, 24, replace=False)) | {0, wl.ndm - 1}
    for p in pulses:
        k = int(round((p.dm - wl.dm_lo) / wl.dm_step))
        rows |= {r for r in range(k - 1, k + 2) if 0 <= r < wl.ndm}
    rows = np.array(sorted(rows))
    Dref = orc.dedisperse(x, wl.n_in, dl, rows=rows, n_out=n_out)
    Dg = D[torch.from_numpy(rows).cuda()][:, :n_out].contiguous()
    assert (Dg.cpu().numpy().astype(np.int64) == Dref).all()

    # (3) search parity on the sampled rows
    sub_desc, sub_keep = gsp.make_desc(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_in,
                                       delays=dl[rows])
    sub = gsp.gsp_plan_create(sub_desc, sub_keep)
    W = len(gsp.DEFAULT_WIDTHS)
    Ls = (n_out // 1024) * 1024
    Dg4 = torch.zeros((len(rows), stride), dtype=torch.int32, device="cuda")
    Dg4[:, :n_out] = Dg
    snr = torch.empty((len(rows), W, Ls), dtype=torch.float32, device="cuda")
    gsp.gsp_boxcar_snr(sub, Dg4, n_out, snr)
    torch.cuda.synchronize()
    contenders, ora = {}, []
    for i, r in enumerate(rows):
        det = orc.search_row(Dref[i], dm_idx=int(r), detail=True)
        assert stats["sigma_ref"][r] == pytest.approx(det["sigma_ref"], rel=1e-12)
        assert np.allclose(stats["sigma_b"][r], det["sigma_b"], rtol=1e-12, atol=0)
        ok, msg = snr_close(snr[i].cpu().numpy(), det["snr"])
        assert ok, "row %d: %s" % (r, msg)
        contenders[int(r)] = window_contenders(det, 1024, 0, 6.0)
        ora.append(det["cands"])
    ora = np.concatenate(ora)
    ncmp, bad = compare_candidates(cands, ora, 6.0, 1024, 0, contenders, rows=set(rows.tolist()))
    assert not bad, bad[:10]
    assert ncmp > 0
    # injected pulses with S/N >= 10 whose DM-trial smearing (largest delay
    # difference to the nearest trial) is at most their width are detected near
    # their DM and time
    found, strong = 0, 0
    for p in pulses:
        k = int(round((p.dm - wl.dm_lo) / wl.dm_step))
        k = min(max(k, 0), wl.ndm - 1)
        smear = int(np.abs(np.asarray(p.delays) - dl[k]).max())
        if p.snr < 10 or smear > p.width or p.t0 + p.width > Ls:
            continue
        strong += 1
        m = cands[(np.abs(cands["dm_idx"] - k) <= 3) &
                  (np.abs(cands["t"] - p.t0) <= p.width + smear + 4)]
        found += int(len(m) > 0)
    assert strong > 0 and found >= 0.8 * strong, (found, strong)


def test_full_size_subband_parity(gsp, orc):
    # The two-stage sub-band path on the CRAFTS-like beam in the bench's
    # configuration (64 sub-bands of 64 channels, groups of 16 trials): every row
    # through the prefix-sum identities with the effective per-channel delays
    # d1[g][c] + d2[d][s(c)], and sampled rows bit-exactly against the oracle.
    from paper_2110_12749_gb300 import synth
    wl = synth.WORKLOADS["crafts"]
    nsub, group = 64, 16
    dl, _ = orc.delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.dms)
    d1, d2, si = orc.subband_delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.dms, nsub, group)
    n_out = orc.subband_nout(wl.n_in, d1, d2)
    x, _, _, pulses = synth.workload_filterbank(
        wl, lambda dm: orc.delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, [dm])[0][0],
        wl.n_in - orc.max_delay(dl))
    desc, keep = gsp.make_desc(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_in, ndm=wl.ndm,
                               dm_lo=wl.dm_lo, dm_step=wl.dm_step)
    sb = gsp.gsp_subband_create(desc, nsub, group)
    g1, g2, gsi = gsp.gsp_subband_delays(sb)
    assert (g1 == d1).all() and (g2 == d2).all() and (gsi == si).all()
    assert gsp.gsp_subband_nout(sb, wl.n_in) == n_out
    D = torch.empty((wl.ndm, (n_out + 3) // 4 * 4), dtype=torch.int32, device="cuda")
    xd = torch.from_numpy(x).cuda()
    gsp.gsp_subband_dedisperse(sb, xd, wl.n_in, D)
    gsp.gsp_subband_finish(sb)
    del xd
    gsp.gsp_subband_destroy(sb)
    torch.cuda.empty_cache()
    # (1) every row
    cs = wl.nchan // nsub
    eff = d1[np.arange(wl.ndm) // group] + np.repeat(d2, cs, axis=1)
    g0, gs1 = _gpu_row_sums(D, n_out)
    e0, e1 = _prefix_expect(x, eff, n_out)
    assert (g0 == e0).all(), np.nonzero(g0 != e0)[0][:10]
    assert (gs1 == e1).all(), np.nonzero(gs1 != e1)[0][:10]
    # (2) sampled rows: sub-band DM trials, trials next to pulses, random ones
    rng = np.random.default_rng(321)
    rows = {int(si[0]), int(si[-1]), 0, wl.ndm - 1}
    rows |= set(int(r) for r in rng.choice(wl.ndm, 3, replace=False))
    for p in pulses[:2]:
        rows.add(min(max(int(round((p.dm - wl.dm_lo) / wl.dm_step)), 0), wl.ndm - 1))
    rows = np.array(sorted(rows))
    Dref = orc.subband_dedisperse(x, wl.n_in, d1, d2, group, rows=rows)
    Dg = D[torch.from_numpy(rows).cuda()][:, :n_out].cpu().numpy().astype(np.int64)
    assert (Dg == Dref).all()
    # the sub-band DM trials equal brute force
    brute = orc.dedisperse(x, wl.n_in, dl, rows=[int(si[0]), int(si[-1])], n_out=n_out)
    assert (Dg[np.searchsorted(rows, [int(si[0]), int(si[-1])])] == brute).all()
