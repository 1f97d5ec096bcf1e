"""CPU oracle for the GSP hot path (arXiv 2110.12749): TEST INFRASTRUCTURE.

Plain C (oracle.c) loaded through ctypes: int64 dedispersion and an FP64
single-pulse search, written from the definitions (Sec. 2.3, Alg. 2/3 for
dedispersion; the search steps are the project's readings of a step the paper
names but does not define).  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library.
"""
import ctypes
import os

import numpy as np

from . import build as _build

DEFAULT_WIDTHS = (1, 2, 3, 4, 6, 9, 14, 20, 30, 45, 70, 100, 150)

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
        L.oracle_delays.argtypes = [i64, dbl, dbl, ctypes.c_int, dbl, i64, vp, vp, vp]
        L.oracle_delays.restype = ctypes.c_int
        L.oracle_max_delay.argtypes = [vp, i64, i64]
        L.oracle_max_delay.restype = i64
        L.oracle_dedisperse.argtypes = [vp, i64, i64, i64, vp, i64, vp, i64, i64, vp]
        L.oracle_dedisperse.restype = ctypes.c_int
        L.oracle_row_sums.argtypes = [vp, i64, i64, i64, vp, i64, i64, vp, vp]
        L.oracle_row_sums.restype = ctypes.c_int
        L.oracle_lower_median.argtypes = [vp, i64]
        L.oracle_lower_median.restype = dbl
        L.oracle_search_row.argtypes = [vp, i64, i32, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_search_row.restype = ctypes.c_int
        L.oracle_search_rows.argtypes = [vp, i64, i64, i64, vp, vp, vp, i64, vp, vp]
        L.oracle_search_rows.restype = ctypes.c_int
        L.oracle_downsample.argtypes = [vp, i64, i64, i64, i64, vp, i64]
        L.oracle_downsample.restype = ctypes.c_int
        L.oracle_subband_delays.argtypes = [i64, dbl, dbl, ctypes.c_int, dbl, i64, vp, i64, i64,
                                            vp, vp, vp]
        L.oracle_subband_delays.restype = ctypes.c_int
        L.oracle_subband_dedisperse.argtypes = [vp, i64, i64, i64, i64, i64, vp, vp, i64, vp, i64,
                                                i64, vp]
        L.oracle_subband_dedisperse.restype = ctypes.c_int
        L.oracle_num_threads.argtypes = []
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


class _Params(ctypes.Structure):
    _fields_ = [("block_len", ctypes.c_int64), ("window_len", ctypes.c_int64),
                ("t_offset", ctypes.c_int64), ("threshold", ctypes.c_double),
                ("bad_lo", ctypes.c_double), ("bad_hi", ctypes.c_double),
                ("widths", ctypes.c_void_p), ("nwidths", ctypes.c_int64)]


CAND_DTYPE = np.dtype([("dm_idx", np.int32), ("width", np.int32),
                       ("t", np.int64), ("snr", np.float64)], align=True)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def num_threads():
    return int(lib().oracle_num_threads())


def delays(nchan, f_lo, f_hi, t_samp, dms, descending=False):
    """Delay matrix int32 [ndm][nchan] and the minimum distance of any entry
    from a rounding tie (Sec. 2.3 delay matrix; cold-plasma law)."""
    dms = np.ascontiguousarray(np.asarray(dms, dtype=np.float64).reshape(-1))
    out = np.empty((dms.size, nchan), dtype=np.int32)
    margin = ctypes.c_double(0.0)
    rc = lib().oracle_delays(nchan, float(f_lo), float(f_hi), int(bool(descending)),
                             float(t_samp), dms.size, _ptr(dms), _ptr(out),
                             ctypes.byref(margin))
    if rc != 0:
        raise ValueError("oracle_delays failed (%d)" % rc)
    return out, margin.value


def max_delay(dl):
    dl = np.ascontiguousarray(dl, dtype=np.int32)
    return int(lib().oracle_max_delay(_ptr(dl), dl.shape[0], dl.shape[1]))


def dedisperse(x, n_in, dl, rows=None, n_out=None):
    """int64 D[r][t] = sum_c x[c][t + dl[rows[r]][c]], t < n_out (Alg. 2/3)."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    dl = np.ascontiguousarray(dl, dtype=np.int32)
    nchan, stride = x.shape
    ndm = dl.shape[0]
    if n_out is None:
        n_out = n_in - max_delay(dl)
    if rows is None:
        r = None
        nrows = ndm
    else:
        r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64).reshape(-1))
        nrows = r.size
    out = np.empty((nrows, max(n_out, 0)), dtype=np.int64)
    rc = lib().oracle_dedisperse(_ptr(x), nchan, n_in, stride, _ptr(dl), ndm,
                                 _ptr(r), nrows, n_out, _ptr(out))
    if rc != 0:
        raise ValueError("oracle_dedisperse failed (%d)" % rc)
    return out


def row_sums(x, n_in, dl, n_out=None):
    """Exact int64 (sum_t D[d][t], sum_t t*D[d][t]) of every DM row from channel
    prefix sums, without dedispersing (the full-coverage identities of the
    plain sum of Alg. 2/3)."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    dl = np.ascontiguousarray(dl, dtype=np.int32)
    nchan, stride = x.shape
    ndm = dl.shape[0]
    if n_out is None:
        n_out = n_in - max_delay(dl)
    s0 = np.empty(ndm, np.int64)
    s1 = np.empty(ndm, np.int64)
    rc = lib().oracle_row_sums(_ptr(x), nchan, n_in, stride, _ptr(dl), ndm, n_out, _ptr(s0),
                               _ptr(s1))
    if rc != 0:
        raise ValueError("oracle_row_sums failed (%d)" % rc)
    return s0, s1


def _params(block_len, window_len, t_offset, threshold, bad_lo, bad_hi, widths):
    w = np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
    p = _Params(block_len, window_len, t_offset, threshold, bad_lo, bad_hi,
                w.ctypes.data, w.size)
    return p, w


def lower_median(v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    return float(lib().oracle_lower_median(_ptr(v), v.size))


def search_row(D, dm_idx=0, block_len=1024, window_len=1024, t_offset=0,
               threshold=6.0, bad_lo=0.5, bad_hi=2.5, widths=DEFAULT_WIDTHS,
               detail=False, cap=None):
    """FP64 single-pulse search of one series.  Returns a dict with the
    candidates (CAND_DTYPE array, ascending t) and, with detail=True, the
    per-block sigma, bad flags, sigma_ref, normalised series, snr[nw][Ls],
    best snr and best width per sample."""
    D = np.ascontiguousarray(D, dtype=np.int64).reshape(-1)
    p, w = _params(block_len, window_len, t_offset, threshold, bad_lo, bad_hi, widths)
    n_out = D.size
    nb = n_out // block_len
    Ls = nb * block_len
    if cap is None:
        cap = Ls // window_len + 2
    cands = np.zeros(max(cap, 1), dtype=CAND_DTYPE)
    n = ctypes.c_int64(0)
    sref = ctypes.c_double(0.0)
    res = {}
    if detail:
        sig = np.zeros(max(nb, 1)); bad = np.zeros(max(nb, 1), np.uint8)
        xn = np.zeros(max(Ls, 1)); snr = np.zeros((w.size, max(Ls, 1)))
        best = np.zeros(max(Ls, 1)); bw = np.zeros(max(Ls, 1), np.int32)
        ptrs = [_ptr(sig), _ptr(bad), ctypes.byref(sref), _ptr(xn), _ptr(snr), _ptr(best), _ptr(bw)]
    else:
        ptrs = [None, None, ctypes.byref(sref), None, None, None, None]
    rc = lib().oracle_search_row(_ptr(D), n_out, int(dm_idx), ctypes.byref(p),
                                 _ptr(cands), cap, ctypes.byref(n), *ptrs)
    if rc != 0:
        raise ValueError("oracle_search_row failed (%d)" % rc)
    res["cands"] = cands[:min(n.value, cap)].copy()
    res["ncand"] = n.value
    res["sigma_ref"] = sref.value
    if detail:
        res.update(sigma_b=sig[:nb], bad=bad[:nb].astype(bool), xnorm=xn[:Ls],
                   snr=snr[:, :Ls], best=best[:Ls], best_w=bw[:Ls])
    return res


def search_rows(D, dm_idx=None, block_len=1024, window_len=1024, t_offset=0,
                threshold=6.0, bad_lo=0.5, bad_hi=2.5, widths=DEFAULT_WIDTHS):
    """Search every row of D (int64 [nrows][n_out]); returns (candidates
    sorted by (dm_idx, t), sigma_ref per row)."""
    D = np.ascontiguousarray(D, dtype=np.int64)
    nrows, n_out = D.shape
    if dm_idx is None:
        dm_idx = np.arange(nrows, dtype=np.int32)
    dm_idx = np.ascontiguousarray(dm_idx, dtype=np.int32)
    p, w = _params(block_len, window_len, t_offset, threshold, bad_lo, bad_hi, widths)
    cap = (n_out // block_len) * block_len // window_len + 2
    cands = np.zeros((nrows, cap), dtype=CAND_DTYPE)
    ncand = np.zeros(nrows, dtype=np.int64)
    sref = np.zeros(nrows, dtype=np.float64)
    rc = lib().oracle_search_rows(_ptr(D), nrows, n_out, n_out, _ptr(dm_idx),
                                  ctypes.byref(p), _ptr(cands), cap, _ptr(ncand), _ptr(sref))
    if rc != 0:
        raise ValueError("oracle_search_rows failed (%d)" % rc)
    out = np.concatenate([cands[r, :min(ncand[r], cap)] for r in range(nrows)]) \
        if nrows else np.zeros(0, CAND_DTYPE)
    return out, sref


def downsample(x, n_in, ds):
    """uint8 [nchan][n_in // ds]: rounded-half-up mean of ds consecutive
    samples (the DownSamp column of the DDplan ranges, Sec. 3.1 Tables 2-3)."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    nchan, stride = x.shape
    n_ds = n_in // ds
    out = np.zeros((nchan, max(n_ds, 1)), dtype=np.uint8)
    rc = lib().oracle_downsample(_ptr(x), nchan, n_in, stride, int(ds), _ptr(out), out.shape[1])
    if rc != 0:
        raise ValueError("oracle_downsample failed (%d)" % rc)
    return out[:, :n_ds]


def ddplan_dms(lo, ddm, n):
    """Trial DMs of one DDplan range: lo + i * ddm, i < n, in FP64 (Sec. 3.1,
    Tables 2-3: Low DM, dDM, Number of DMs)."""
    return float(lo) + np.arange(int(n), dtype=np.float64) * float(ddm)


def subband_delays(nchan, f_lo, f_hi, t_samp, dms, nsub, group, descending=False):
    """Two-stage delay tables (d1 int32 [nsdm][nchan], d2 int32 [ndm][nsub],
    sub-band DM trial indices int32 [nsdm]) of the sub-band algorithm."""
    dms = np.ascontiguousarray(np.asarray(dms, dtype=np.float64).reshape(-1))
    ndm = dms.size
    nsdm = (ndm + group - 1) // group
    d1 = np.empty((nsdm, nchan), np.int32)
    d2 = np.empty((ndm, nsub), np.int32)
    si = np.empty(nsdm, np.int32)
    rc = lib().oracle_subband_delays(nchan, float(f_lo), float(f_hi), int(bool(descending)),
                                     float(t_samp), ndm, _ptr(dms), int(nsub), int(group),
                                     _ptr(d1), _ptr(d2), _ptr(si))
    if rc != 0:
        raise ValueError("oracle_subband_delays failed (%d)" % rc)
    return d1, d2, si


def subband_nout(n_in, d1, d2):
    return n_in - max_delay(d1) - max_delay(d2)


def subband_dedisperse(x, n_in, d1, d2, group, n_out=None, rows=None):
    """int64 D [nrows][n_out] of the two-stage sub-band dedispersion (rows: the
    trial indices to compute, default all)."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    d1 = np.ascontiguousarray(d1, dtype=np.int32)
    d2 = np.ascontiguousarray(d2, dtype=np.int32)
    nchan, stride = x.shape
    ndm, nsub = d2.shape
    if n_out is None:
        n_out = subband_nout(n_in, d1, d2)
    if rows is None:
        r, nrows = None, ndm
    else:
        r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64).reshape(-1))
        nrows = r.size
    out = np.empty((nrows, max(n_out, 0)), dtype=np.int64)
    rc = lib().oracle_subband_dedisperse(_ptr(x), nchan, n_in, stride, nsub, int(group),
                                         _ptr(d1), _ptr(d2), ndm, _ptr(r), nrows, n_out, _ptr(out))
    if rc != 0:
        raise ValueError("oracle_subband_dedisperse failed (%d)" % rc)
    return out


def ingest_transpose(x_tc):
    """Channel-major copy x[c][t] of time-major samples x_tc[t][c] (the input
    layout of Alg. 2, numpts x numchan, Sec. 2.3)."""
    x_tc = np.asarray(x_tc, dtype=np.uint8)
    n, c = x_tc.shape
    out = np.empty((c, n), np.uint8)
    for ch in range(c):
        out[ch, :] = x_tc[:, ch]
    return out
