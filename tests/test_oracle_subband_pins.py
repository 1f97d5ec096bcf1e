"""Pins of the oracle's DDplan ranges, time downsampling and two-stage
sub-band dedispersion (Sec. 2.3: GSP accelerates the sub-band algorithm of
PRESTO's prepsubband; Sec. 3.1, Tables 2-3: the DDplan ranges, with a DM step
and a downsampling factor per range).

Each function is checked against something other than itself: the paper's
printed tables (tests/golden), exact rational arithmetic, pure-Python
enumeration on tiny inputs, and the special cases where the two-stage sum
reduces to plain brute-force dedispersion (one channel per sub-band, one DM
per group, the sub-band DM trials themselves).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _ddplan(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        no, lo, hi, ddm, ds, n = line.split()
        rows.append((int(no), lo, hi, ddm, int(ds), int(n)))
    return rows


# ------------------------------------------------------------ DDplan tables

@pytest.mark.parametrize("name,total", [("ddplan_band1.txt", 3462), ("ddplan_band2.txt", 10730)])
def test_ddplan_tables_are_consistent(name, total):
    rows = _ddplan(name)
    assert [r[0] for r in rows] == list(range(1, len(rows) + 1))
    for i, (_, lo, hi, ddm, ds, n) in enumerate(rows):
        # Number of DMs = (High DM - Low DM) / dDM exactly (decimal arithmetic)
        assert (Fraction(hi) - Fraction(lo)) / Fraction(ddm) == n
        assert ds >= 1 and ds & (ds - 1) == 0          # powers of two
        if i + 1 < len(rows):
            assert hi == rows[i + 1][1]                    # ranges are contiguous
            assert Fraction(rows[i + 1][3]) >= Fraction(ddm)
            assert rows[i + 1][4] >= ds
    assert rows[0][1] == "0"
    assert sum(r[5] for r in rows) == total


@pytest.mark.parametrize("name", ["ddplan_band1.txt", "ddplan_band2.txt"])
def test_ddplan_dms_cover_each_range(orc, name):
    for _, lo, hi, ddm, ds, n in _ddplan(name):
        dms = orc.ddplan_dms(float(lo), float(ddm), n)
        assert dms.size == n and dms[0] == float(lo)
        assert abs((dms[-1] + float(ddm)) - float(hi)) < 1e-9
        assert np.all(np.diff(dms) > 0)


# ------------------------------------------------------------- downsampling

def test_downsample_identity_and_constant(orc):
    rng = np.random.default_rng(3)
    x = rng.integers(0, 256, (5, 97), dtype=np.uint8)
    assert (orc.downsample(x, 97, 1) == x).all()
    for k in (0, 1, 128, 255):
        c = np.full((3, 64), k, np.uint8)
        for ds in (2, 3, 7, 16):
            assert (orc.downsample(c, 64, ds) == k).all()


def test_downsample_rounds_half_up(orc):
    x = np.array([[1, 2, 0, 1, 254, 255, 3, 3]], np.uint8)
    assert orc.downsample(x, 8, 2).tolist() == [[2, 1, 255, 3]]
    y = np.array([[0, 0, 1, 0, 1, 1, 2, 2, 2]], np.uint8)    # means 1/3, 2/3, 2
    assert orc.downsample(y, 9, 3).tolist() == [[0, 1, 2]]


@pytest.mark.parametrize("ds", [2, 3, 5, 8, 16])
def test_downsample_brute_force(orc, ds):
    rng = np.random.default_rng(ds)
    n_in = 203                                   # ragged: trailing partial group dropped
    x = rng.integers(0, 256, (4, n_in + 9), dtype=np.uint8)
    got = orc.downsample(x, n_in, ds)
    assert got.shape == (4, n_in // ds)
    for c in range(4):
        for t in range(n_in // ds):
            mean = Fraction(sum(int(v) for v in x[c, t * ds:(t + 1) * ds]), ds)
            assert got[c, t] == math.floor(mean + Fraction(1, 2))


# ------------------------------------------------------- sub-band delay tables

def _ref_channel(s, cs, descending):
    return s * cs if descending else s * cs + cs - 1


@pytest.mark.parametrize("descending", [False, True])
def test_subband_delays_compose_to_brute_force_at_subband_dms(orc, descending):
    nchan, nsub, group = 512, 16, 7
    dms = np.arange(0.0, 300.0, 2.5)
    dl, _ = orc.delays(nchan, 1000.0, 1500.0, 64e-6, dms, descending=descending)
    d1, d2, si = orc.subband_delays(nchan, 1000.0, 1500.0, 64e-6, dms, nsub, group,
                                    descending=descending)
    cs = nchan // nsub
    assert si.tolist() == [min(g * group + group // 2, len(dms) - 1)
                           for g in range((len(dms) + group - 1) // group)]
    assert (d1 >= 0).all()
    for s in range(nsub):
        ref = _ref_channel(s, cs, descending)
        assert (d1[:, ref] == 0).all()                  # the reference channel
        assert (d2[:, s] == dl[:, ref]).all()           # stage 2 = the reference's delay
    for g, i in enumerate(si):
        total = d1[g] + np.repeat(d2[i], cs)
        assert (total == dl[i]).all()                   # exact at the sub-band DM


def test_subband_delays_textbook_form(orc):
    # the reference-channel delays, from the ms/GHz form in exact rationals
    nchan, nsub, f_lo, f_hi, ts = 256, 8, 300.0, 800.0, 98.304e-6
    dms = [3.0, 41.5, 200.0]
    _, d2, _ = orc.subband_delays(nchan, f_lo, f_hi, ts, dms, nsub, 1)
    df = Fraction(f_hi - f_lo) / nchan
    ftop = (Fraction(f_lo) + (nchan - 1 + Fraction(1, 2)) * df) / 1000
    cs = nchan // nsub
    for i, dm in enumerate(dms):
        for s in range(nsub):
            f = (Fraction(f_lo) + (s * cs + cs - 1 + Fraction(1, 2)) * df) / 1000
            ms = Fraction("4.148808") * Fraction(dm) * (1 / (f * f) - 1 / (ftop * ftop))
            assert d2[i, s] == math.floor(ms / 1000 / Fraction(ts) + Fraction(1, 2))


# --------------------------------------------------- two-stage dedispersion

def _subband_python(x, n_in, d1, d2, group, n_out):
    nsdm, nchan = d1.shape
    ndm, nsub = d2.shape
    cs = nchan // nsub
    n1 = n_in - int(d1.max())
    S = [[[sum(int(x[c, t + d1[g, c]]) for c in range(s * cs, (s + 1) * cs))
           for t in range(n1)] for s in range(nsub)] for g in range(nsdm)]
    return np.array([[sum(S[d // group][s][t + d2[d, s]] for s in range(nsub))
                      for t in range(n_out)] for d in range(ndm)], np.int64)


@pytest.mark.parametrize("nsub,group", [(2, 2), (4, 3), (8, 1), (1, 4)])
def test_subband_dedisperse_brute_force_tiny(orc, nsub, group):
    rng = np.random.default_rng(nsub * 10 + group)
    nchan, n_in = 8, 90
    dms = np.sort(rng.uniform(0.0, 5.0, 7))
    d1, d2, _ = orc.subband_delays(nchan, 1200.0, 1500.0, 1e-4, dms, nsub, group)
    x = rng.integers(0, 256, (nchan, n_in + 5), dtype=np.uint8)
    n_out = orc.subband_nout(n_in, d1, d2)
    assert n_out > 10
    got = orc.subband_dedisperse(x, n_in, d1, d2, group)
    assert (got == _subband_python(x, n_in, d1, d2, group, n_out)).all()


def test_subband_reduces_to_brute_force(orc):
    rng = np.random.default_rng(9)
    nchan, n_in = 64, 3000
    dms = np.arange(0.0, 40.0, 1.0)
    x = rng.integers(0, 256, (nchan, n_in), dtype=np.uint8)
    dl, _ = orc.delays(nchan, 1200.0, 1500.0, 1e-4, dms)
    brute = orc.dedisperse(x, n_in, dl)
    # one channel per sub-band, or one DM per group: exact for every trial
    for nsub, group in ((nchan, 5), (8, 1)):
        d1, d2, _ = orc.subband_delays(nchan, 1200.0, 1500.0, 1e-4, dms, nsub, group)
        D = orc.subband_dedisperse(x, n_in, d1, d2, group)
        assert (D == brute[:, :D.shape[1]]).all(), (nsub, group)
    # otherwise exact at the sub-band DM trials
    d1, d2, si = orc.subband_delays(nchan, 1200.0, 1500.0, 1e-4, dms, 8, 6)
    D = orc.subband_dedisperse(x, n_in, d1, d2, 6)
    assert (D[si] == brute[si, :D.shape[1]]).all()
    other = np.setdiff1d(np.arange(len(dms)), si)
    assert (D[other] != brute[other, :D.shape[1]]).any()    # and an approximation elsewhere


def test_subband_pulse_smearing_bound(orc):
    # A noiseless dispersed pulse of width w at a trial DM: the sub-band
    # series keeps the full pulse sum a * C * w (every channel's contribution
    # lands in the row), displaced by at most the stage-1 rounding per channel.
    nchan, nsub, group, n_in, a, w = 128, 16, 8, 4000, 3, 6
    dms = np.arange(0.0, 64.0, 0.5)
    d1, d2, si = orc.subband_delays(nchan, 1200.0, 1500.0, 1e-4, dms, nsub, group)
    dl, _ = orc.delays(nchan, 1200.0, 1500.0, 1e-4, dms)
    i = 37
    t0 = 500
    x = np.zeros((nchan, n_in), np.uint8)
    for c in range(nchan):
        x[c, t0 + dl[i, c]:t0 + dl[i, c] + w] = a
    D = orc.subband_dedisperse(x, n_in, d1, d2, group)
    assert D[i].sum() == a * nchan * w
    assert D[i].max() <= a * nchan
    lo, hi = np.nonzero(D[i])[0][[0, -1]]
    spread = int(np.abs(d1[i // group] + np.repeat(d2[i], nchan // nsub) - dl[i]).max())
    assert t0 - spread <= lo and hi <= t0 + w - 1 + spread


def test_subband_row_selection(orc):
    rng = np.random.default_rng(13)
    nchan, n_in = 64, 2500
    dms = np.arange(0.0, 30.0, 1.0)
    d1, d2, _ = orc.subband_delays(nchan, 1200.0, 1500.0, 1e-4, dms, 8, 4)
    x = rng.integers(0, 256, (nchan, n_in), dtype=np.uint8)
    full = orc.subband_dedisperse(x, n_in, d1, d2, 4)
    rows = [29, 3, 3, 17, 0]
    assert (orc.subband_dedisperse(x, n_in, d1, d2, 4, rows=rows) == full[rows]).all()


def test_ingest_transpose_definition(orc):
    x = np.random.default_rng(2).integers(0, 256, (13, 5), dtype=np.uint8)
    out = orc.ingest_transpose(x)
    for t in range(13):
        for c in range(5):
            assert out[c, t] == x[t, c]
