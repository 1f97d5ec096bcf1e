"""Shared test helpers: workload set-up through the oracle, and the
candidate-list comparison rule (identical except near the threshold or where
the oracle's own top two contenders of a window are too close to order)."""
import math

import numpy as np

SNR_RTOL = 1e-5      # |snr_gpu - snr_oracle| <= SNR_RTOL * max(|snr_oracle|, 1)
THR_BAND = 1e-4      # candidates within this of the threshold are not compared
TIE_RTOL = 1e-5      # windows whose top-two oracle contenders are this close are skipped


def snr_close(g, o):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    nan_g, nan_o = np.isnan(g), np.isnan(o)
    if not (nan_g == nan_o).all():
        return False, "NaN pattern differs"
    ok = np.abs(g - o) <= SNR_RTOL * np.maximum(np.abs(o), 1.0)
    ok |= nan_o
    if not ok.all():
        i = np.unravel_index(np.argmax(~ok), ok.shape)
        return False, "worst at %s: gpu %r oracle %r" % (i, g[i], o[i])
    return True, ""


def window_contenders(detail, L, t_offset, thr):
    """Per window: (top S/N, second S/N) over all (t, w) pairs >= thr - THR_BAND."""
    snr = detail["snr"]
    Ls = snr.shape[1]
    out = {}
    if detail["sigma_ref"] == 0 or Ls == 0:
        return out
    s = np.where(np.isnan(snr), -np.inf, snr)
    k_first = (0 + t_offset) // L
    k_last = (Ls - 1 + t_offset) // L
    for k in range(k_first, k_last + 1):
        a = max(k * L - t_offset, 0)
        b = min((k + 1) * L - t_offset, Ls)
        v = s[:, a:b].ravel()
        v = v[v >= thr - THR_BAND]
        if v.size == 0:
            continue
        if v.size > 1:
            top = np.partition(v, v.size - 2)[-2:]
            out[int(k)] = (float(top[1]), float(top[0]))
        else:
            out[int(k)] = (float(v[0]), -math.inf)
    return out


def compare_candidates(gpu, ora, thr, L, t_offset=0, contenders=None, rows=None):
    """gpu / ora: structured arrays with dm_idx, t, width, snr.  contenders:
    {dm_idx: window_contenders(...)} for the rows whose windows are checked for
    ambiguous maxima (None = no tie screening).  rows: restrict to these DMs.
    Returns (n_compared, list of mismatch strings)."""
    def keyed(c):
        d = {}
        for r in c:
            dm = int(r["dm_idx"])
            if rows is not None and dm not in rows:
                continue
            d[(dm, (int(r["t"]) + t_offset) // L)] = (int(r["t"]), int(r["width"]), float(r["snr"]))
        return d

    g, o = keyed(gpu), keyed(ora)
    bad, n = [], 0
    for key in sorted(set(g) | set(o)):
        dm, k = key
        if contenders is not None and dm in contenders:
            c = contenders[dm].get(k)
            if c is not None and c[1] > -math.inf and (c[0] - c[1]) <= TIE_RTOL * max(abs(c[0]), 1.0):
                continue
        ref = o.get(key, g.get(key))
        if abs(ref[2] - thr) < THR_BAND:
            continue
        if key not in g or key not in o:
            bad.append("%s only in %s: %s" % (key, "gpu" if key in g else "oracle", ref))
            continue
        n += 1
        a, b = g[key], o[key]
        if a[0] != b[0] or a[1] != b[1] or abs(a[2] - b[2]) > SNR_RTOL * max(abs(b[2]), 1.0):
            bad.append("%s gpu %s oracle %s" % (key, a, b))
    return n, bad
