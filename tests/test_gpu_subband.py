"""GPU parity of the DDplan ranges (time downsampling, Sec. 3.1 Tables 2-3) and of
the two-stage sub-band dedispersion (Sec. 2.3) against the CPU oracle, through
the C ABI: downsampled filterbanks and sub-band series bit-exact, candidate
lists as in the brute-force parity tests."""
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


@pytest.mark.parametrize("ds", [1, 2, 3, 4, 8, 16, 128])
def test_downsample_bit_exact(gsp, orc, ds):
    rng = np.random.default_rng(ds)
    nchan, n_in = 7, 5003                      # ragged: the trailing partial group is dropped
    x = rng.integers(0, 256, (nchan, 5008), dtype=np.uint8)
    x[2] = 255
    x[3, ::2] = 0
    n_ds = n_in // ds
    out = torch.full((nchan, (n_ds + 15) // 16 * 16 + 16), 7, dtype=torch.uint8, device="cuda")
    gsp.gsp_downsample(torch.from_numpy(x).cuda(), nchan, n_in, ds, out)
    o = out.cpu().numpy()
    assert (o[:, :n_ds] == orc.downsample(x, n_in, ds)).all()
    assert (o[:, n_ds:] == 7).all()            # nothing written past n_in // ds


def _subband_case(gsp, orc, nchan, nsub, group, ndm, n_in, descending, seed):
    rng = np.random.default_rng(seed)
    desc, keep = gsp.make_desc(nchan, 1200.0, 1500.0, 1e-4, n_in, ndm=ndm, dm_lo=0.0,
                               dm_step=0.5, freq_descending=descending, threshold=5.0)
    sb = gsp.gsp_subband_create(desc, nsub, group)
    dms = 0.5 * np.arange(ndm)
    d1, d2, si = orc.subband_delays(nchan, 1200.0, 1500.0, 1e-4, dms, nsub, group,
                                    descending=descending)
    g1, g2, gsi = gsp.gsp_subband_delays(sb)
    assert (g1 == d1).all() and (g2 == d2).all() and (gsi == si).all()
    n_out = orc.subband_nout(n_in, d1, d2)
    assert gsp.gsp_subband_nout(sb, n_in) == n_out
    stride = (n_in + 15) // 16 * 16
    x = rng.integers(0, 256, (nchan, stride), dtype=np.uint8)
    return desc, keep, sb, dms, d1, d2, si, n_out, x


@pytest.mark.parametrize("nchan,nsub,group,ndm,desc_order,seed", [
    (256, 16, 8, 70, False, 1),       # ragged last group
    (256, 32, 16, 48, True, 2),       # descending channel order
    (96, 96, 5, 23, False, 3),        # one channel per sub-band: brute force
    (128, 4, 1, 20, False, 4),        # one trial per group: brute force
])
def test_subband_dedisperse_bit_exact(gsp, orc, nchan, nsub, group, ndm, desc_order, seed):
    n_in = 12000
    _, _, sb, dms, d1, d2, si, n_out, x = _subband_case(gsp, orc, nchan, nsub, group, ndm,
                                                        n_in, desc_order, seed)
    out = torch.full((ndm, (n_out + 3) // 4 * 4 + 4), -7, dtype=torch.int32, device="cuda")
    gsp.gsp_subband_dedisperse(sb, torch.from_numpy(x).cuda(), n_in, out)
    gsp.gsp_subband_finish(sb)
    assert gsp.gsp_subband_launches(sb) >= 2
    o = out.cpu().numpy()
    ref = orc.subband_dedisperse(x, n_in, d1, d2, group)
    assert (o[:, :n_out].astype(np.int64) == ref).all()
    assert (o[:, n_out:] == -7).all()
    # the sub-band DM trials equal brute-force dedispersion
    dl, _ = orc.delays(nchan, 1200.0, 1500.0, 1e-4, dms, descending=desc_order)
    brute = orc.dedisperse(x, n_in, dl, rows=si, n_out=n_out)
    assert (o[si, :n_out] == brute).all()


def test_subband_then_search_parity(gsp, orc):
    from paper_2110_12749_gb300 import synth
    nchan, nsub, group, ndm, n_in = 256, 16, 8, 64, 40000
    desc, keep, sb, dms, d1, d2, si, n_out, _ = _subband_case(gsp, orc, nchan, nsub, group, ndm,
                                                              n_in, False, 5)
    pulses = []
    for dm, t0, w in [(12.0, 9000, 4), (20.25, 21000, 9)]:
        dl1, _ = orc.delays(nchan, 1200.0, 1500.0, 1e-4, [dm])
        pulses.append(synth.Pulse(dm, t0, w, 20.0, synth.pulse_amplitude(20.0, 16.0, nchan, w),
                                  dl1[0]))
    x = synth.filterbank(nchan, (n_in + 15) // 16 * 16, 31, 128.0, 16.0, pulses=pulses,
                         threads=4)
    D = torch.zeros((ndm, (n_out + 3) // 4 * 4), dtype=torch.int32, device="cuda")
    gsp.gsp_subband_dedisperse(sb, torch.from_numpy(x).cuda(), n_in, D)
    gsp.gsp_subband_finish(sb)
    plan = gsp.gsp_plan_create(desc, keep)
    gsp.gsp_search_series(plan, D, n_out)
    got, n, st = gsp.gsp_candidates(plan)
    assert st == gsp.GSP_OK and n > 0
    ref = orc.subband_dedisperse(x, n_in, d1, d2, group)
    cont, ora = {}, []
    for r in range(ndm):
        det = orc.search_row(ref[r], dm_idx=r, threshold=5.0, detail=True)
        cont[r] = window_contenders(det, 1024, 0, 5.0)
        ora.append(det["cands"])
    ora = np.concatenate(ora)
    ncmp, bad = compare_candidates(got, ora, 5.0, 1024, 0, cont)
    assert not bad, bad[:5]
    assert ncmp > 0
    # both injected pulses are found near their DM and time
    for dm, t0, w in [(12.0, 9000, 4), (20.25, 21000, 9)]:
        near = got[(np.abs(dms[got["dm_idx"]] - dm) <= 1.0) & (np.abs(got["t"] - t0) <= 2 * w)]
        assert near.size > 0 and near["snr"].max() > 10.0, (dm, t0)


def _ddplan_oracle(orc, x, n_in, nchan, f_lo, f_hi, ts, ranges, thr):
    """Per range: downsample, delays at ts*ds, dedisperse, search every row."""
    out = []
    dm0 = 0
    for lo, step, n, ds in ranges:
        xd = orc.downsample(x, n_in, ds)
        dms = orc.ddplan_dms(lo, step, n)
        dl, _ = orc.delays(nchan, f_lo, f_hi, ts * ds, dms)
        D = orc.dedisperse(xd, n_in // ds, dl)
        rows, cont = [], {}
        for r in range(n):
            det = orc.search_row(D[r], dm_idx=dm0 + r, threshold=thr, detail=True)
            cont[dm0 + r] = window_contenders(det, 1024, 0, thr)
            rows.append(det["cands"])
        out.append((ds, np.concatenate(rows), cont))
        dm0 += n
    return out


def test_ddplan_parity(gsp, orc):
    from paper_2110_12749_gb300 import synth
    nchan, f_lo, f_hi, ts, n_in, thr = 64, 1200.0, 1500.0, 1e-4, 65536, 5.0
    ranges = [(0.0, 0.5, 40, 1), (20.0, 1.0, 30, 2), (50.0, 2.0, 25, 4)]
    pulses = []
    for dm, t0, w in [(8.0, 20000, 3), (35.0, 40000, 8), (80.0, 30000, 16)]:
        dl1, _ = orc.delays(nchan, f_lo, f_hi, ts, [dm])
        pulses.append(synth.Pulse(dm, t0, w, 25.0, synth.pulse_amplitude(25.0, 16.0, nchan, w),
                                  dl1[0]))
    x = synth.filterbank(nchan, n_in, 17, 128.0, 16.0, pulses=pulses, threads=4)
    base, keep = gsp.make_desc(nchan, f_lo, f_hi, ts, n_in, ndm=1, threshold=thr)
    dd = gsp.gsp_ddplan_create(base, ranges)
    gsp.gsp_ddplan_search(dd, torch.from_numpy(x).cuda(), n_in)
    got, n, st = gsp.gsp_ddplan_candidates(dd)
    assert st == gsp.GSP_OK and n == got.size
    ref = _ddplan_oracle(orc, x, n_in, nchan, f_lo, f_hi, ts, ranges, thr)
    total = 0
    for r, (ds, ora, cont) in enumerate(ref):
        mine = got[got["beam"] == r].copy()
        assert (mine["t"] % ds == 0).all() and (mine["width"] % ds == 0).all()
        mine["t"] //= ds
        mine["width"] //= ds
        ncmp, bad = compare_candidates(mine, ora, thr, 1024, 0, cont)
        assert not bad, (r, bad[:5])
        total += ncmp
    assert total > 0
    # range r's trials follow range r-1's in dm_idx
    lo = 0
    for r, (_, _, nr, _) in enumerate(ranges):
        sel = got["beam"] == r
        assert ((got["dm_idx"][sel] >= lo) & (got["dm_idx"][sel] < lo + nr)).all()
        lo += nr
    with pytest.raises(gsp.GspError):
        gsp.gsp_ddplan_search(dd, torch.from_numpy(x).cuda(), n_in, t_offset=2)


def test_ddplan_paper_band1_plan_runs(gsp):
    # the eight ranges of Table 2 (Band1, 271-398 MHz, 512 channels) on a short noise input
    ranges = [(0.0, 0.01, 1134, 1), (11.34, 0.03, 362, 2), (22.2, 0.05, 337, 4),
              (39.05, 0.1, 381, 8), (77.15, 0.2, 383, 16), (153.75, 0.5, 380, 32),
              (343.75, 1.0, 344, 64), (687.75, 2.0, 141, 128)]
    n_in = 1 << 20
    base, keep = gsp.make_desc(512, 271.0, 398.0, 98.304e-6, n_in, ndm=1, threshold=7.0)
    dd = gsp.gsp_ddplan_create(base, ranges)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randint(96, 160, (512, n_in), dtype=torch.uint8, device="cuda", generator=g)
    gsp.gsp_ddplan_search(dd, x, n_in)
    got, n, st = gsp.gsp_ddplan_candidates(dd)
    assert st == gsp.GSP_OK
    assert got.size == n
    if n:
        assert got["dm_idx"].max() < sum(r[2] for r in ranges)
        assert set(np.unique(got["beam"])) <= set(range(len(ranges)))
