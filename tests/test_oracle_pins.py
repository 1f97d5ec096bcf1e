"""Pins of the CPU oracle against what the method and the mathematics fix.

Every oracle function is checked here against something other than itself:
physical invariants and an independent textbook form of the dispersion law
(delays); channel-sum, single-channel and prefix-sum identities plus pure-
Python brute force (dedispersion, Sec. 2.3 / Alg. 2-3); exact closed forms of
least-squares detrending, the lower median, the matched-filter S/N of an
injected boxcar in Gaussian noise, the Gaussian false-alarm rate, and a
pure-Python enumeration of the whole search on tiny series.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

WIDTHS = (1, 2, 3, 4, 6, 9, 14, 20, 30, 45, 70, 100, 150)


# ----------------------------------------------------------------- delays

def test_delays_top_channel_and_dm0_are_zero(orc):
    dl, _ = orc.delays(256, 1200.0, 1500.0, 1e-4, np.arange(200.0))
    assert (dl[:, -1] == 0).all()          # top channel = reference
    assert (dl[0] == 0).all()              # DM 0
    dld, _ = orc.delays(256, 1200.0, 1500.0, 1e-4, np.arange(200.0), descending=True)
    assert (dld[:, 0] == 0).all()
    assert (dld == dl[:, ::-1]).all()      # descending = mirrored channel order


def test_delays_monotone(orc):
    dl, _ = orc.delays(512, 1000.0, 1500.0, 49.152e-6, np.arange(0, 1000, 3.7))
    assert (np.diff(dl, axis=0) >= 0).all()   # more DM, more delay
    assert (np.diff(dl, axis=1) <= 0).all()   # higher frequency, less delay


def test_delays_linear_in_dm(orc):
    dms = np.array([13.25, 26.5, 53.0, 106.0])
    dl, _ = orc.delays(1024, 1000.0, 1500.0, 49.152e-6, dms)
    for k in range(1, 4):
        assert np.abs(dl[k] - 2 * dl[k - 1]).max() <= 1


def test_delays_textbook_form(orc):
    # Cold-plasma delay in the usual astronomer's units:
    # dt = 4.148808 ms * DM * (nu_GHz^-2 - nu_top_GHz^-2).  Evaluated here in
    # ms/GHz with exact rational arithmetic, rounded to the nearest sample.
    nchan, f_lo, f_hi, ts = 4096, 1000.0, 1500.0, 49.152e-6
    dms = [0.5, 77.0, 999.5]
    dl, margin = orc.delays(nchan, f_lo, f_hi, ts, dms)
    assert margin > 1e-9
    df = Fraction(f_hi - f_lo) / nchan
    ftop = (Fraction(f_lo) + (nchan - 1 + Fraction(1, 2)) * df) / 1000
    rng = np.random.default_rng(1)
    for i, dm in enumerate(dms):
        for c in list(rng.integers(0, nchan, 40)) + [0, nchan - 1]:
            f = (Fraction(f_lo) + (int(c) + Fraction(1, 2)) * df) / 1000
            ms = Fraction("4.148808") * Fraction(dm) * (1 / (f * f) - 1 / (ftop * ftop))
            x = ms / 1000 / Fraction(ts)
            want = math.floor(x + Fraction(1, 2))
            assert dl[i, c] == want, (dm, c)
    # whole-band sweep of DM 1000 between the band edges is 2.3049 s
    x_edges = 4.148808e-3 * 1000 * (1.0 / 1.0**2 - 1.0 / 1.5**2) / ts
    d1000, _ = orc.delays(nchan, f_lo, f_hi, ts, [1000.0])
    assert abs(d1000[0, 0] - x_edges) < 0.01 * x_edges   # centres sit df/2 inside the edges


def test_delay_table_of_the_three_workloads(orc):
    # max delay, samples per unit DM at the lowest channel and tie margins
    cases = [
        (256, 1200.0, 1500.0, 100e-6, np.arange(200.0), 2056),
        (4096, 1000.0, 1500.0, 49.152e-6, 0.5 * np.arange(2000), 46856),
        (2048, 500.0, 3300.0, 98.304e-6, np.arange(3000.0), 493269),
    ]
    for nchan, lo, hi, ts, dms, dmax in cases:
        dl, margin = orc.delays(nchan, lo, hi, ts, dms)
        assert orc.max_delay(dl) == dmax
        assert margin > 1e-9


# ------------------------------------------------------------ dedispersion

def _brute_dedisperse(x, dl, n_out):
    ndm, nchan = dl.shape
    out = [[0] * n_out for _ in range(ndm)]
    for d in range(ndm):
        for t in range(n_out):
            s = 0
            for c in range(nchan):
                s += int(x[c][t + int(dl[d][c])])
            out[d][t] = s
    return np.array(out, dtype=np.int64)


def test_dedisperse_dm0_is_channel_sum(orc):
    rng = np.random.default_rng(2)
    x = rng.integers(0, 256, (64, 3000), dtype=np.uint8)
    dl, _ = orc.delays(64, 1200.0, 1500.0, 1e-4, [0.0, 30.0])
    D = orc.dedisperse(x, 3000, dl)
    n_out = 3000 - orc.max_delay(dl)
    assert D.shape == (2, n_out)
    assert (D[0] == x[:, :n_out].astype(np.int64).sum(0)).all()


def test_dedisperse_single_channel_identity(orc):
    rng = np.random.default_rng(3)
    x = rng.integers(0, 256, (1, 500), dtype=np.uint8)
    dl, _ = orc.delays(1, 1200.0, 1500.0, 1e-4, np.arange(0, 500, 7.0))
    assert (dl == 0).all()
    D = orc.dedisperse(x, 500, dl)
    assert (D == x[0].astype(np.int64)[None, :]).all()


def test_dedisperse_brute_force_tiny(orc):
    rng = np.random.default_rng(4)
    for trial in range(6):
        nchan = int(rng.integers(1, 9))
        n_in = int(rng.integers(20, 65))
        ndm = int(rng.integers(1, 6))
        dl = rng.integers(0, n_in // 2, (ndm, nchan)).astype(np.int32)
        stride = n_in + int(rng.integers(0, 5))
        x = rng.integers(0, 256, (nchan, stride), dtype=np.uint8)
        n_out = n_in - int(dl.max())
        D = orc.dedisperse(x, n_in, dl)
        assert (D == _brute_dedisperse(x, dl, n_out)).all()
        rows = rng.permutation(ndm)[: max(1, ndm // 2)]
        Dr = orc.dedisperse(x, n_in, dl, rows=rows)
        assert (Dr == D[rows]).all()


def test_dedisperse_noiseless_pulse(orc):
    nchan, n_in, ts = 128, 8192, 1e-4
    dms = np.arange(0, 100, 2.0)
    dl, _ = orc.delays(nchan, 1200.0, 1500.0, ts, dms)
    n_out = n_in - orc.max_delay(dl)
    x = np.zeros((nchan, n_in), np.uint8)
    dstar, t0, w, a = 21, 1000, 7, 3
    for c in range(nchan):
        x[c, t0 + dl[dstar, c]: t0 + dl[dstar, c] + w] = a
    D = orc.dedisperse(x, n_in, dl)
    want = np.zeros(n_out, np.int64)
    want[t0:t0 + w] = a * nchan
    assert (D[dstar] == want).all()
    # every row collects the same total (each sample lies in range)
    assert (D.sum(1) == a * nchan * w).all()
    # the pulse is smeared at the wrong DM: the peak is lower
    assert D[0].max() < a * nchan and D[-1].max() < a * nchan


def test_dedisperse_prefix_sum_invariants(orc):
    rng = np.random.default_rng(5)
    nchan, n_in = 96, 4000
    x = rng.integers(0, 256, (nchan, n_in), dtype=np.uint8)
    dl, _ = orc.delays(nchan, 1200.0, 1500.0, 1e-4, np.arange(0, 150, 1.5))
    n_out = n_in - orc.max_delay(dl)
    D = orc.dedisperse(x, n_in, dl)
    xi = x.astype(np.int64)
    P = np.concatenate([np.zeros((nchan, 1), np.int64), np.cumsum(xi, 1)], 1)
    tt = np.arange(n_in, dtype=np.int64)
    Q = np.concatenate([np.zeros((nchan, 1), np.int64), np.cumsum(xi * tt, 1)], 1)
    for d in range(dl.shape[0]):
        s0 = sum(P[c, dl[d, c] + n_out] - P[c, dl[d, c]] for c in range(nchan))
        s1 = sum((Q[c, dl[d, c] + n_out] - Q[c, dl[d, c]]) - dl[d, c] * (P[c, dl[d, c] + n_out] - P[c, dl[d, c]])
                 for c in range(nchan))
        assert D[d].sum() == s0
        assert (D[d] * np.arange(n_out)).sum() == s1


def test_row_sums_equal_brute_force_and_dedispersed_sums(orc):
    """oracle.row_sums (the prefix-sum identities, used to check every row of
    full-size series) against pure-Python brute force on tiny inputs and the
    sums of the oracle's dedispersed rows on a larger one."""
    rng = np.random.default_rng(51)
    for trial in range(5):
        nchan = int(rng.integers(1, 9))
        n_in = int(rng.integers(20, 65))
        ndm = int(rng.integers(1, 6))
        dl = rng.integers(0, n_in // 2, (ndm, nchan)).astype(np.int32)
        x = rng.integers(0, 256, (nchan, n_in + int(rng.integers(0, 5))), dtype=np.uint8)
        n_out = n_in - int(dl.max())
        Db = _brute_dedisperse(x, dl, n_out)
        s0, s1 = orc.row_sums(x, n_in, dl)
        assert (s0 == Db.sum(1)).all()
        assert (s1 == (Db * np.arange(n_out)).sum(1)).all()
    nchan, n_in = 77, 6007
    x = np.full((nchan, 6016), 255, np.uint8)
    x[:, ::3] = rng.integers(0, 256, (nchan, 2006), dtype=np.uint8)
    dl, _ = orc.delays(nchan, 1000.0, 1500.0, 1e-4, np.arange(0, 60, 0.7))
    D = orc.dedisperse(x, n_in, dl)
    s0, s1 = orc.row_sums(x, n_in, dl)
    assert (s0 == D.sum(1)).all()
    assert (s1 == (D * np.arange(D.shape[1])).sum(1)).all()


# ------------------------------------------------------------------ search

def _pattern(n):
    # e = [1, -1, -1, 1] repeated: zero sum and zero correlation with j
    return np.tile(np.array([1, -1, -1, 1], np.int64), n // 4)


def test_search_ramp_has_zero_residual(orc):
    B, nb = 256, 6
    j = np.arange(B)
    D = np.concatenate([1000 + 37 * b + (3 * b - 7) * j for b in range(nb)]).astype(np.int64)
    r = orc.search_row(D, block_len=B, window_len=B, detail=True)
    assert np.allclose(r["sigma_b"], 0.0, atol=1e-9)
    assert r["sigma_ref"] < 1e-9 and r["ncand"] == 0


def test_search_detrend_closed_form_and_lower_median(orc):
    B = 256
    scales = [4, 9, 3, 5, 1, 40, 7, 6, 2]        # sigma_b of each block, exactly
    e = _pattern(B)
    j = np.arange(B)
    D = np.concatenate([50000 + 11 * b + (b - 4) * j + s * e for b, s in enumerate(scales)])
    r = orc.search_row(D.astype(np.int64), block_len=B, window_len=B, detail=True)
    assert np.allclose(r["sigma_b"], scales, rtol=1e-12)
    med = sorted(scales)[(len(scales) - 1) // 2]
    assert r["sigma_ref"] == pytest.approx(med, rel=1e-12)
    bad = [(s < 0.5 * med) or (s > 2.5 * med) for s in scales]
    assert list(r["bad"]) == bad
    for b, s in enumerate(scales):
        xb = r["xnorm"][b * B:(b + 1) * B]
        if bad[b]:
            assert (xb == 0).all()
        else:
            assert np.allclose(xb, s * e / med, atol=1e-9)


def test_search_boxcar_matches_direct_sums(orc):
    rng = np.random.default_rng(6)
    D = rng.integers(-500, 500, 4096).astype(np.int64) + 10**6
    r = orc.search_row(D, block_len=1024, window_len=1024, detail=True)
    x = r["xnorm"]
    Ls = x.size
    c = np.concatenate([[0.0], np.cumsum(x)])
    for iw, w in enumerate(WIDTHS):
        want = (c[w:Ls + 1] - c[:Ls + 1 - w]) / math.sqrt(w)
        got = r["snr"][iw]
        assert np.allclose(got[:Ls + 1 - w], want, atol=1e-9)
        assert np.isnan(got[Ls + 1 - w:]).all()
    snr = np.where(np.isnan(r["snr"]), -np.inf, r["snr"])
    assert np.allclose(r["best"], snr.max(0))
    assert (r["best_w"] == np.array(WIDTHS)[snr.argmax(0)]).all()


def _py_search(D, B, L, thr, lo, hi, widths, t_offset=0):
    """Independent pure-Python enumeration of the search steps."""
    n = len(D)
    nb = n // B
    Ls = nb * B
    sig, fits = [], []
    for b in range(nb):
        blk = [float(v) for v in D[b * B:(b + 1) * B]]
        A = np.vstack([np.ones(B), np.arange(B, dtype=float)]).T
        coef, *_ = np.linalg.lstsq(A, np.array(blk), rcond=None)
        res = [blk[j] - coef[0] - coef[1] * j for j in range(B)]
        fits.append(res)
        sig.append(math.sqrt(sum(v * v for v in res) / B))
    sref = sorted(sig)[(nb - 1) // 2] if nb else 0.0
    x = []
    for b in range(nb):
        badb = sref == 0 or sig[b] < lo * sref or sig[b] > hi * sref
        x += [0.0] * B if badb else [v / sref for v in fits[b]]
    cands = {}
    if sref == 0:
        return [], x
    for t in range(Ls):
        best, bw = -math.inf, 0
        for w in widths:
            if t + w > Ls:
                continue
            s = sum(x[t:t + w]) / math.sqrt(w)
            if s > best:
                best, bw = s, w
        if bw and best >= thr:
            win = (t + t_offset) // L
            if win not in cands or best > cands[win][2]:
                cands[win] = (t, bw, best)
    return [cands[k] for k in sorted(cands)], x


def test_search_pure_python_enumeration(orc):
    rng = np.random.default_rng(7)
    B, L, widths = 256, 128, (1, 2, 3, 5, 8, 13)
    for trial in range(3):
        n = 2048 + int(rng.integers(0, 200))
        D = (rng.normal(0, 30, n) + 4000).round().astype(np.int64)
        for _ in range(4):   # a few pulses so that candidates exist
            t0, w = int(rng.integers(0, n - 20)), int(rng.integers(1, 14))
            D[t0:t0 + w] += int(rng.integers(60, 200))
        off = int(rng.integers(0, 300))
        r = orc.search_row(D, block_len=B, window_len=L, threshold=3.0, widths=widths,
                           t_offset=off, detail=True)
        want, x = _py_search(D, B, L, 3.0, 0.5, 2.5, widths, off)
        assert np.allclose(r["xnorm"], x, atol=1e-9)
        got = [(int(c["t"]), int(c["width"]), float(c["snr"])) for c in r["cands"]]
        assert len(got) == len(want) and len(got) > 0
        for g, w_ in zip(got, want):
            assert g[0] == w_[0] and g[1] == w_[1] and g[2] == pytest.approx(w_[2], rel=1e-9)


def test_search_window_tie_keeps_earliest(orc):
    B = 256
    rng = np.random.default_rng(8)
    blk = (rng.normal(0, 10, B) + 900).round().astype(np.int64)
    blk[100:104] += 200
    D = np.concatenate([blk, blk, blk, blk])       # identical blocks: equal maxima
    r = orc.search_row(D, block_len=B, window_len=2 * B, threshold=5.0)
    ts = [int(c["t"]) for c in r["cands"]]
    assert ts == [100, 2 * B + 100]


def test_search_closed_form_snr_of_injected_boxcar(orc):
    # Gaussian noise (sigma s) + boxcar of amplitude a*s and width w.  The
    # expected matched S/N is a*sqrt(w) times the part of the boxcar that the
    # per-block line fit leaves (exact, from the hat matrix), divided by the
    # expected lower-median block sigma, s*sqrt(nu/B)*(1 - 2/(9 nu))^(3/2) with
    # nu = B - 2 degrees of freedom.
    B, nb, s, a, w, t0 = 1024, 15, 1000.0, 2.0, 20, 7 * 1024 + 300
    j = np.arange(B, dtype=float)
    A = np.vstack([np.ones(B), j]).T
    H = A @ np.linalg.inv(A.T @ A) @ A.T
    p = np.zeros(B)
    p[300:300 + w] = a * s
    kept = ((p - H @ p)[300:300 + w]).sum() / (a * s * w)
    nu = B - 2
    expect = a * math.sqrt(w) * kept / (math.sqrt(nu / B) * (1 - 2 / (9 * nu)) ** 1.5)
    rng = np.random.default_rng(9)
    vals, widths_hit = [], 0
    nseed = 200
    for _ in range(nseed):
        D = rng.normal(0.0, s, nb * B)
        D[t0:t0 + w] += a * s
        r = orc.search_row(np.round(D + 5e6).astype(np.int64), block_len=B, window_len=B,
                           threshold=-1e9, detail=True)
        iw = WIDTHS.index(w)
        vals.append(r["snr"][iw][t0])
        widths_hit += int(r["best_w"][t0] in (14, 20, 30))
    m = float(np.mean(vals))
    assert abs(m - expect) < 3.0 / math.sqrt(nseed), (m, expect)
    assert abs(np.std(vals) - 1.0) < 0.15
    assert widths_hit > 0.8 * nseed


def test_search_white_noise_false_alarm_rate(orc):
    B, nb = 1024, 12000
    rng = np.random.default_rng(10)
    D = np.round(rng.normal(0, 500.0, nb * B) + 1e6).astype(np.int64)
    r = orc.search_row(D, block_len=B, window_len=B, widths=(1,), threshold=1e9, detail=True)
    x = r["snr"][0]
    n = x.size
    for thr in (3.0, 4.0):
        p = 0.5 * math.erfc(thr / math.sqrt(2))
        k = int((x > thr).sum())
        assert abs(k - n * p) < 4.5 * math.sqrt(n * p), (thr, k, n * p)


def test_search_short_series_and_flat_rows(orc):
    r = orc.search_row(np.full(1000, 7, np.int64), block_len=1024)
    assert r["ncand"] == 0 and r["sigma_ref"] == 0.0
    r = orc.search_row(np.full(4096, 7, np.int64), block_len=1024)
    assert r["ncand"] == 0 and r["sigma_ref"] == 0.0


def test_search_rows_matches_search_row(orc):
    rng = np.random.default_rng(11)
    D = (rng.normal(0, 50, (5, 3000)) + 10000).round().astype(np.int64)
    D[2, 1500:1510] += 400
    c, sref = orc.search_rows(D, block_len=512, window_len=512, threshold=4.0)
    want = []
    for rr in range(5):
        one = orc.search_row(D[rr], dm_idx=rr, block_len=512, window_len=512, threshold=4.0)
        assert sref[rr] == one["sigma_ref"]
        want.extend([(int(q["dm_idx"]), int(q["t"]), int(q["width"])) for q in one["cands"]])
    assert [(int(q["dm_idx"]), int(q["t"]), int(q["width"])) for q in c] == want
