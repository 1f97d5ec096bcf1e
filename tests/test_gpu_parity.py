"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Dedispersion: bit-exact int32 series.  Search: per-block sigma and sigma_ref
(1e-12 relative), S/N of every (dm, width, t) within 1e-5 * max(|snr|, 1),
and candidate lists identical except within 1e-4 of the threshold or where
the oracle's own top two contenders of a window are within 1e-5.
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


def _plan(gsp, orc_dl, nsamp, flags=0, **kw):
    desc, keep = gsp.make_desc(orc_dl.shape[1], 1200.0, 1500.0, 1e-4, nsamp, delays=orc_dl,
                               flags=flags, **kw)
    return gsp.gsp_plan_create(desc, keep)


def _tiny(orc):
    from paper_2110_12749_gb300 import synth
    wl = synth.WORKLOADS["tiny"]
    dl, _ = orc.delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.dms)
    n_out = wl.n_in - orc.max_delay(dl)
    x, _, _, pulses = synth.workload_filterbank(
        wl, lambda dm: orc.delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, [dm])[0][0], n_out)
    return wl, dl, x, n_out, pulses


@pytest.fixture(scope="module")
def tiny(orc):
    wl, dl, x, n_out, pulses = _tiny(orc)
    D = orc.dedisperse(x, wl.n_in, dl)
    return wl, dl, x, n_out, pulses, D


@pytest.mark.parametrize("flags", [0, 2])
def test_tiny_dedisperse_bit_exact(gsp, orc, tiny, flags):
    wl, dl, x, n_out, pulses, Dref = tiny
    desc, keep = gsp.make_desc(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_in, ndm=wl.ndm,
                               dm_lo=wl.dm_lo, dm_step=wl.dm_step, flags=flags)
    plan = gsp.gsp_plan_create(desc, keep)
    assert (gsp.gsp_plan_delays(plan) == dl).all()
    assert gsp.gsp_plan_nout(plan, wl.n_in) == n_out
    xd = torch.from_numpy(x).cuda()
    out = torch.full((wl.ndm, n_out + 12), -7, dtype=torch.int32, device="cuda")
    gsp.gsp_dedisperse(plan, xd, wl.n_in, out)
    o = out.cpu().numpy()
    assert (o[:, :n_out].astype(np.int64) == Dref).all()
    assert (o[:, n_out:] == -7).all()          # nothing written past n_out


@pytest.mark.parametrize("thr", [6.0, 3.5])
def test_tiny_search_parity(gsp, orc, tiny, thr):
    wl, dl, x, n_out, pulses, Dref = tiny
    plan = _plan(gsp, dl, wl.n_in, threshold=thr)
    Dd = torch.from_numpy(Dref.astype(np.int32)).cuda()
    W = len(gsp.DEFAULT_WIDTHS)
    Ls = (n_out // 1024) * 1024
    snr = torch.empty((wl.ndm, W, Ls), dtype=torch.float32, device="cuda")
    gsp.gsp_boxcar_snr(plan, Dd, n_out, snr)
    st = gsp.gsp_search_stats(plan, n_out)
    snr = snr.cpu().numpy()
    cands, n, status = gsp.gsp_candidates(plan)
    assert status == gsp.GSP_OK
    contenders = {}
    ora = []
    for r in range(wl.ndm):
        det = orc.search_row(Dref[r], dm_idx=r, threshold=thr, detail=True)
        assert np.allclose(st["sigma_b"][r], det["sigma_b"], rtol=1e-12, atol=0)
        assert st["sigma_ref"][r] == pytest.approx(det["sigma_ref"], rel=1e-12)
        assert (st["bad"][r] == det["bad"]).all()
        ok, msg = snr_close(snr[r], det["snr"])
        assert ok, "row %d: %s" % (r, msg)
        contenders[r] = window_contenders(det, 1024, 0, thr)
        ora.append(det["cands"])
    ora = np.concatenate(ora)
    ncmp, bad = compare_candidates(cands, ora, thr, 1024, 0, contenders)
    assert not bad, bad[:10]
    assert ncmp >= (5 if thr == 6.0 else 1000)
    # the injected pulse (DM 50, w 5, S/N 15) is found at its DM and time
    p = pulses[0]
    hit = [c for c in cands if abs(int(c["dm_idx"]) - 50) <= 1 and abs(int(c["t"]) - p.t0) <= 5]
    assert hit and max(float(c["snr"]) for c in hit) > 10.0


def test_tiny_fused_search_equals_series_search(gsp, orc, tiny):
    wl, dl, x, n_out, pulses, Dref = tiny
    plan = _plan(gsp, dl, wl.n_in)
    xd = torch.from_numpy(x).cuda()
    gsp.gsp_search(plan, xd, wl.n_in)                  # D into plan scratch, fused block sums
    c1, n1, _ = gsp.gsp_candidates(plan)
    st1 = gsp.gsp_search_stats(plan, n_out)
    Dd = torch.from_numpy(Dref.astype(np.int32)).cuda()
    gsp.gsp_search_series(plan, Dd, n_out)              # block sums from the series
    c2, n2, _ = gsp.gsp_candidates(plan)
    st2 = gsp.gsp_search_stats(plan, n_out)
    assert n1 == n2 and (c1 == c2).all()
    assert (st1["sigma_b"] == st2["sigma_b"]).all() and (st1["sigma_ref"] == st2["sigma_ref"]).all()
    c3, n3, _ = gsp.gsp_search_host(plan, x, wl.n_in)  # host input path
    assert n3 == n1 and (c3 == c1).all()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_ragged_shapes_bit_exact(gsp, orc, seed):
    rng = np.random.default_rng(seed)
    nchan = int(rng.integers(1, 200))
    ndm = int(rng.integers(1, 70))
    n_in = int(rng.integers(3000, 9000))
    stride = (n_in + 15) // 16 * 16 + 16 * int(rng.integers(0, 3))
    dms = np.sort(rng.uniform(0, 120, ndm))
    desc_flag = bool(rng.integers(0, 2))
    dl, _ = orc.delays(nchan, 1200.0, 1500.0, 1e-4, dms, descending=desc_flag)
    n_out = n_in - orc.max_delay(dl)
    x = rng.integers(0, 256, (nchan, stride), dtype=np.uint8)
    Dref = orc.dedisperse(x, n_in, dl)
    for flags in (0, 2):
        desc, keep = gsp.make_desc(nchan, 1200.0, 1500.0, 1e-4, n_in, dms=dms,
                                   freq_descending=desc_flag, flags=flags)
        plan = gsp.gsp_plan_create(desc, keep)
        assert (gsp.gsp_plan_delays(plan) == dl).all()
        out = torch.zeros((ndm, (n_out + 3) // 4 * 4), dtype=torch.int32, device="cuda")
        gsp.gsp_dedisperse(plan, torch.from_numpy(x).cuda(), n_in, out)
        assert (out.cpu().numpy()[:, :n_out].astype(np.int64) == Dref).all(), flags


def test_explicit_unsorted_delay_table(gsp, orc):
    rng = np.random.default_rng(12)
    nchan, ndm, n_in = 77, 33, 5000
    dl = rng.integers(0, 900, (ndm, nchan)).astype(np.int32)
    x = rng.integers(0, 256, (nchan, 5008), dtype=np.uint8)
    n_out = n_in - int(dl.max())
    Dref = orc.dedisperse(x, n_in, dl)
    plan = _plan(gsp, dl, n_in)
    out = torch.zeros((ndm, (n_out + 3) // 4 * 4), dtype=torch.int32, device="cuda")
    gsp.gsp_dedisperse(plan, torch.from_numpy(x).cuda(), n_in, out)
    assert (out.cpu().numpy()[:, :n_out].astype(np.int64) == Dref).all()


def test_extreme_values_no_overflow(gsp, orc):
    nchan, n_in = 4096, 6000
    dl, _ = orc.delays(nchan, 1000.0, 1500.0, 49.152e-6, [0.0, 10.0, 20.0])
    x = np.full((nchan, n_in), 255, np.uint8)
    n_out = n_in - orc.max_delay(dl)
    plan = _plan(gsp, dl, n_in)
    out = torch.zeros((3, (n_out + 3) // 4 * 4), dtype=torch.int32, device="cuda")
    gsp.gsp_dedisperse(plan, torch.from_numpy(x).cuda(), n_in, out)
    assert (out.cpu().numpy()[:, :n_out] == 255 * nchan).all()
    # constant series: sigma_ref = 0, no candidates, no NaN
    gsp.gsp_search_series(plan, out, n_out)
    c, n, st = gsp.gsp_candidates(plan)
    assert n == 0
    s = gsp.gsp_search_stats(plan, n_out)
    assert (s["sigma_ref"] == 0).all() and s["bad"].all()


def test_custom_widths_blocks_windows_offset(gsp, orc, tiny):
    """Generic (non-default) width set, block and window lengths, and an absolute
    sample offset of the series: S/N and candidates against the oracle."""
    wl, dl, x, n_out, pulses, Dref = tiny
    widths, B, L, off, thr = (1, 3, 7, 16, 40, 90), 512, 700, 333, 3.5
    rows = np.arange(0, wl.ndm, 7)
    desc, keep = gsp.make_desc(dl.shape[1], 1200.0, 1500.0, 1e-4, wl.n_in, delays=dl[rows],
                               widths=widths, block_len=B, window_len=L, threshold=thr)
    plan = gsp.gsp_plan_create(desc, keep)
    stride = (n_out + 3) // 4 * 4
    Dd = torch.zeros((len(rows), stride), dtype=torch.int32, device="cuda")
    Dd[:, :n_out] = torch.from_numpy(Dref[rows].astype(np.int32)).cuda()
    Ls = (n_out // B) * B
    snr = torch.empty((len(rows), len(widths), Ls), dtype=torch.float32, device="cuda")
    gsp.gsp_boxcar_snr(plan, Dd, n_out, snr)
    snr = snr.cpu().numpy()
    gsp.gsp_search_series(plan, Dd, n_out, t_offset=off)
    cands, n, st = gsp.gsp_candidates(plan)
    contenders, ora = {}, []
    for i, r in enumerate(rows):
        det = orc.search_row(Dref[r], dm_idx=i, block_len=B, window_len=L, widths=widths,
                             threshold=thr, detail=True)
        ok, msg = snr_close(snr[i], det["snr"])
        assert ok, "row %d: %s" % (r, msg)
        det_off = orc.search_row(Dref[r], dm_idx=i, block_len=B, window_len=L, widths=widths,
                                 threshold=thr, t_offset=off, detail=True)
        contenders[i] = window_contenders(det_off, L, off, thr)
        ora.append(det_off["cands"])
    ora = np.concatenate(ora)
    ncmp, bad = compare_candidates(cands, ora, thr, L, off, contenders)
    assert not bad, bad[:10]
    assert ncmp >= 10


@pytest.mark.parametrize("chunks,flags,block_len",
                         [("8", 0, 1000), ("3", 0, 1000), ("1", 0, 1000), ("8", 2, 1000),
                          ("8", 0, 256), ("5", 0, 256)])
def test_host_input_in_chunks_equals_device_search(gsp, orc, monkeypatch, chunks, flags,
                                                   block_len):
    # gsp_search_host copies the input in time chunks that overlap the
    # dedispersion; block_len 1000 makes the chunk unit lcm(1000, 16) = 2000
    # (equal chunks: the series is too short for the growing ones), block_len
    # 256 a unit of 256 (chunks growing 1, 1, 2, 4, 8, ... units of weight), and
    # the host rows have a stride that is not a multiple of 16.  One chunk and
    # the simple kernel (flags 2) take the copy-first path.
    monkeypatch.setenv("GSP_HOST_CHUNKS", chunks)
    rng = np.random.default_rng(21)
    nchan, n_in = 96, 30000
    dms = np.arange(0.0, 40.0, 0.5)
    x = rng.integers(0, 256, (nchan, n_in + 7), dtype=np.uint8)
    x[:, 12000:12004] = 255
    desc, keep = gsp.make_desc(nchan, 1200.0, 1500.0, 1e-4, n_in, dms=dms, block_len=block_len,
                               threshold=4.0, flags=gsp.GSP_FLAG_TIMING | flags)
    plan = gsp.gsp_plan_create(desc, keep)
    c1, n1, _ = gsp.gsp_search_host(plan, x, n_in, t_offset=4000)
    assert n1 > 0
    launches = gsp.gsp_plan_launches(plan)
    if flags == 0:
        assert launches >= int(chunks) + 5     # one dedispersion launch per chunk + the search
    dd_ms, se_ms = gsp.gsp_plan_timing(plan)
    assert dd_ms > 0 and se_ms > 0
    xd = torch.zeros((nchan, (n_in + 15) // 16 * 16), dtype=torch.uint8)
    xd[:, :n_in] = torch.from_numpy(x[:, :n_in])
    gsp.gsp_search(plan, xd.cuda(), n_in, t_offset=4000)
    c2, n2, _ = gsp.gsp_candidates(plan)
    assert n1 == n2 and (c1 == c2).all()
    # and the oracle on the same input
    dl, _ = orc.delays(nchan, 1200.0, 1500.0, 1e-4, dms)
    D = orc.dedisperse(np.ascontiguousarray(x[:, :n_in]), n_in, dl)
    cont, ora = {}, []
    for r in range(len(dms)):
        det = orc.search_row(D[r], dm_idx=r, block_len=block_len, threshold=4.0, t_offset=4000,
                             detail=True)
        cont[r] = window_contenders(det, 1024, 4000, 4.0)
        ora.append(det["cands"])
    ncmp, bad = compare_candidates(c1, np.concatenate(ora), 4.0, 1024, 4000, cont)
    assert not bad, bad[:5]
    assert ncmp > 0
