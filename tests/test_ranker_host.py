"""Host logic of the ranker's training and evaluation (paper_2110_12749_gb300/
ranker.py), on CPU: candidate labels against injected pulses."""
import numpy as np

from paper_2110_12749_gb300 import ranker, synth
from paper_2110_12749_gb300.gsp import CAND_DTYPE


def _cands(rows):
    c = np.zeros(len(rows), dtype=CAND_DTYPE)
    for i, (d, t, w, snr) in enumerate(rows):
        c[i]["dm_idx"], c[i]["t"], c[i]["width"], c[i]["snr"] = d, t, w, snr
    return c


def _table(ndm=200, nchan=64):
    # delays growing linearly with DM and towards the bottom channel (channel 0)
    dm = np.arange(ndm)[:, None]
    ch = (nchan - 1 - np.arange(nchan))[None, :]
    return (dm * ch // 8).astype(np.int32)


def test_labels_core_track_and_background():
    dl = _table()
    k = 100
    pulse = synth.Pulse(dm=float(k), t0=5000, width=4, snr=20.0, delays=dl[k].astype(np.int64))
    rows = [
        (k, 5000, 4, 20.0),          # the pulse itself: positive
        (k + 2, 5003, 4, 15.0),      # core, strong: positive
        (k + 3, 5001, 2, 9.0),       # core but weak (< 0.6 of the best): ignored
        (k + 20, 5000 + (dl[k, 0] - dl[k + 20, 0]), 8, 7.0),   # on the dispersion track: ignored
        (k + 80, 5000, 4, 7.0),      # far in DM: background
        (k, 90000, 4, 7.0),          # far in time: background
    ]
    lab, pid = ranker.label_candidates(_cands(rows), [pulse], dl, dl.shape[0])
    assert lab.tolist() == [1, 1, -1, -1, 0, 0]
    assert pid.tolist() == [0, 0, 0, -1, -1, -1]


def test_labels_without_pulses_are_background():
    dl = _table()
    lab, pid = ranker.label_candidates(_cands([(5, 10, 1, 6.5), (150, 99, 30, 8.0)]), [], dl, 200)
    assert lab.tolist() == [0, 0] and pid.tolist() == [-1, -1]


def test_short_crafts_recipe():
    wl = ranker.short_crafts(1 << 18, n_pulses=100)
    base = synth.WORKLOADS["crafts"]
    assert wl.n_in == 1 << 18 and wl.n_pulses == 100
    assert (wl.nchan, wl.ndm, wl.dm_step, wl.t_samp) == (base.nchan, base.ndm, base.dm_step,
                                                         base.t_samp)
