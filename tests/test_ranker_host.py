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


def _ps():
    # five pulses: detected S/N 9, 15, 25 (>= 8); 7.5 (below 8, nominal 10); one undetected
    return {"nominal": np.array([9.0, 16.0, 30.0, 10.0, 12.0]),
            "width": np.array([2, 20, 80, 1, 3]),
            "detected": np.array([9.0, 15.0, 25.0, 7.5, -1.0]),
            "best": np.array([0.9, 0.2, 0.6, 0.05, -1.0]),
            "neg": np.array([0.01, 0.3, 0.7, 0.02]),
            "pos": np.array([0.9, 0.6, 0.2]),
            "n_scored": 12, "rank_s": 0.5}


def test_summarise_counts():
    out = ranker.summarise(_ps(), thresholds=(0.5, 0.1))
    assert out["pulses_detected_snr_ge_min"] == 3
    assert out["pulses_nominal_snr_ge_min"] == 5
    assert out["nominal_snr_ge_min_detected"] == 4
    assert abs(out["recall"] - 2 / 3) < 1e-12                 # 0.9 and 0.6 pass 0.5
    assert abs(out["recall_nominal"] - 2 / 4) < 1e-12
    assert abs(out["precision"] - 2 / 3) < 1e-12              # pos 0.9, 0.6; neg 0.7
    assert abs(out["negatives_rejected"] - 3 / 4) < 1e-12
    assert out["recalled_by_width"] == {"1-9": [1, 1], "10-49": [0, 1], "50-150": [1, 1]}
    assert out["recalled_by_snr"] == {"8-12": [1, 1], "12-20": [0, 1], ">=20": [1, 1]}
    assert out["missed"] == [[16.0, 20, 15.0, 0.2]]
    at = out["at"]["0.1"]
    assert at["recall"] == 1.0 and abs(at["recall_nominal"] - 3 / 4) < 1e-12
    assert abs(out["candidates_per_s"] - 24.0) < 1e-12


def test_threshold_for_keeps_the_share():
    ps = _ps()
    assert ranker.threshold_for(ps, keep=1.0) == 0.2          # the weakest detected >= 8
    assert ranker.threshold_for(ps, keep=0.5) == 0.5          # capped at 0.5
    ps["best"] = np.linspace(0.0, 0.45, 201)
    ps["detected"] = np.full(201, 9.0)
    # keep 99% of 201 pulses: floor(0.01 * 201) = 2 may fall below the threshold
    t = ranker.threshold_for(ps, keep=0.99)
    assert t == ps["best"][2] and (ps["best"] >= t).mean() >= 0.99
    ps["detected"][:] = 7.0
    assert ranker.threshold_for(ps) == 0.5                    # none detected at >= 8


def test_bench_entry_points_wrap_the_host_summary(monkeypatch):
    # the GPU scoring pass replaced by fixed per-pulse arrays
    monkeypatch.setattr(ranker, "pulse_scores", lambda r, src, beams, seed: _ps())
    thr = ranker.choose_threshold(None, None, 8, 0)
    assert thr == ranker.threshold_for(_ps())
    ev = ranker.evaluate(None, None, 4, 0, thresholds=(thr, 0.05, 0.5))
    assert ev == ranker.summarise(_ps(), 8.0, (thr, 0.05, 0.5))
    assert set(ev["at"]) == {"0.05", "0.5"}
    import json
    json.dumps(ev)      # the bench line must serialise


def test_two_tier_operating_point():
    # three pulses detected at S/N >= 8; candidates at S/N >= 8 pass at the
    # validation threshold, weaker ones only at a score >= 0.5
    ps = {"nominal": np.array([9.0, 12.0, 8.5]), "width": np.array([3, 40, 90]),
          "detected": np.array([9.1, 11.0, 8.2]),
          "best": np.array([0.9, 0.02, 0.6]),      # best score over all core candidates
          "best8": np.array([0.9, 0.02, 0.001]),   # best over core candidates at S/N >= 8
          "pos": np.array([0.9, 0.02, 0.6, 0.001]), "pos_snr": np.array([9.1, 11.0, 7.0, 8.2]),
          "neg": np.array([0.03, 0.4, 0.7, 0.0]), "neg_snr": np.array([9.0, 6.5, 6.1, 8.0]),
          "n_scored": 8, "rank_s": 1.0}
    out = ranker.summarise(ps, 8.0, (0.01,))
    # pulse 0 (0.9 at S/N >= 8), pulse 1 (0.02 >= 0.01 at S/N 11), pulse 2 (0.6 >= 0.5 below 8)
    assert out["recall"] == 1.0
    # kept positives: 0.9, 0.02, 0.6 (< 8 but >= 0.5); kept negatives: 0.03 (S/N 9), 0.7
    assert out["precision"] == 3 / 5
    assert out["negatives_rejected"] == 0.5
    assert ranker.threshold_for(ps, 8.0, keep=1.0) == 0.001
