"""Training and evaluation of the candidate ranker on candidates that the
pipeline itself produces from synthetic beams with injected dispersed pulses,
narrowband RFI and DM-0 bursts.  Host orchestration only: dedispersion, the
search, snippet extraction, training and inference all run in libgsp.

Labels of a candidate (dm_idx d, start t, width w) against the injected
pulses of its beam (pulse DM trial k = nearest trial, per-channel delays):
  1  core of a pulse: |d - k| <= 3 and |t - t0| <= w_p + smear + 4, where
     smear = largest delay difference between the pulse and trial k, and an
     S/N at least 0.6 of the best core candidate of that pulse (weaker core
     candidates are labelled -1);
  -1 elsewhere on a pulse's dispersion track (within 60 trials, inside the
     time span the pulse's energy reaches at trial d, +-150 samples): neither
     pulse nor RFI, left out of training and of the precision;
  0  everything else (noise, RFI, DM-0 bursts).
A pulse is recalled if its best-scored core candidate scores at least the
operating threshold (softmax probability of class 1); precision counts the
candidates scoring at least the threshold among those labelled 0 or 1.  The
threshold is chosen on the training beams (the score that keeps 99% of
their pulses with S/N >= 8), never on the evaluation beams.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import gsp, synth


def short_crafts(n_in=1 << 18, n_pulses=40):
    """The CRAFTS-like beam (4096 channels, 2000 trials) cut to n_in samples."""
    return dataclasses.replace(synth.WORKLOADS["crafts"], n_in=n_in, n_pulses=n_pulses)


def label_candidates(cands, pulses, dl, ndm):
    """Labels (1 / 0 / -1) and the matched pulse index (-1 if none)."""
    n = cands.size
    lab = np.zeros(n, np.int32)
    pid = np.full(n, -1, np.int32)
    d = cands["dm_idx"].astype(np.int64)
    t = cands["t"].astype(np.int64)
    bottom = int(np.argmax(dl[-1]))            # the channel with the largest delay
    for i, p in enumerate(pulses):
        k = int(np.argmin(np.abs(dl[:, bottom] - p.delays[bottom])))
        smear = int(np.abs(p.delays - dl[k]).max())
        core = (np.abs(d - k) <= 3) & (np.abs(t - p.t0) <= p.width + smear + 4)
        shift = p.delays[bottom] - dl[d, bottom]         # energy arrives within [min, max]
        lo = p.t0 + np.minimum(shift, 0) - 150
        hi = p.t0 + p.width + np.maximum(shift, 0) + 150
        track = (np.abs(d - k) <= 60) & (t >= lo) & (t <= hi)
        lab[track & (lab == 0)] = -1
        if core.any():
            strong = core & (cands["snr"] >= 0.6 * cands["snr"][core].max())
            lab[core] = -1
            lab[strong] = 1
            pid[core] = i
    return lab, pid


class BeamSource:
    """Searches synthetic beams of one workload and hands out their candidates,
    labels and snippets."""

    def __init__(self, wl, threshold=6.0):
        import torch
        self.torch = torch
        self.wl = wl
        desc, keep = gsp.make_desc(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_in, ndm=wl.ndm,
                                   dm_lo=wl.dm_lo, dm_step=wl.dm_step, threshold=threshold)
        self.plan = gsp.gsp_plan_create(desc, keep)
        self.dl = gsp.gsp_plan_delays(self.plan)
        self.n_out = gsp.gsp_plan_nout(self.plan, wl.n_in)
        self.D = torch.zeros((wl.ndm, (self.n_out + 3) // 4 * 4), dtype=torch.int32,
                             device="cuda")
        self.search_s = 0.0

    def delays(self, dm):
        d1, _ = gsp.make_desc(self.wl.nchan, self.wl.f_lo, self.wl.f_hi, self.wl.t_samp,
                              self.wl.n_in, dms=[dm])
        return gsp.gsp_compute_delays(d1)[0][0]

    def search(self, beam, seed):
        """Search one beam; returns (candidates, labels, pulse index, pulses)."""
        torch = self.torch
        x, _, _, pulses = synth.workload_filterbank(self.wl, self.delays, self.n_out, beam=beam,
                                                    seed=seed)
        xd = torch.from_numpy(x).cuda()
        del x
        t0 = time.perf_counter()
        gsp.gsp_search(self.plan, xd, self.wl.n_in, out=self.D)
        cands, n, _ = gsp.gsp_candidates(self.plan)
        self.search_s += time.perf_counter() - t0
        del xd
        lab, pid = label_candidates(cands, pulses, self.dl, self.wl.ndm)
        return cands, lab, pid, pulses

    def snippets(self, cands):
        """Snippets (torch float CUDA [n][64][64]) of candidates of the last searched beam."""
        torch = self.torch
        out = torch.empty((cands.size, 64, 64), dtype=torch.float32, device="cuda")
        if cands.size:
            dc = torch.from_numpy(np.ascontiguousarray(cands).view(np.uint8).copy()).cuda()
            gsp.gsp_ranker_snippets(self.plan, self.D, dc, out)
        return out


def build_training_set(src, beams, seed):
    """Snippets (torch float CUDA) and labels of every candidate labelled 0 or
    1 in the given number of beams (candidates on a pulse's track excluded),
    a global pulse id per snippet (-1 for label 0) and the nominal S/N of
    every pulse (indexed by that id)."""
    torch = src.torch
    xs, ys, ps, snr = [], [], [], []
    base = 0
    for b in range(beams):
        cands, lab, pid, pulses = src.search(b, seed)
        keep = lab >= 0
        xs.append(src.snippets(cands[keep]))
        ys.append(lab[keep].astype(np.int32))
        ps.append(np.where(pid[keep] >= 0, pid[keep] + base, -1))
        snr.extend(p.snr for p in pulses)
        base += len(pulses)
    return torch.cat(xs), np.concatenate(ys), np.concatenate(ps), np.array(snr)


def choose_threshold(ranker, x, y, pulse_ids, pulse_snr, snr_min=8.0, keep=0.99):
    """Score that keeps `keep` of the training pulses with S/N >= snr_min (each
    by its best positive snippet), at most 0.5."""
    pos = np.nonzero(y == 1)[0]
    s = score(ranker, x[__import__("torch").from_numpy(pos).cuda()])
    best = {}
    for i, sc in zip(pulse_ids[pos], s):
        if pulse_snr[int(i)] >= snr_min:
            best[int(i)] = max(best.get(int(i), 0.0), float(sc))
    v = np.sort(np.array(list(best.values())))
    if v.size == 0:
        return 0.5
    return float(min(0.5, v[int(np.floor((1.0 - keep) * v.size))]))


def train(ranker, x, y, steps, batch=256, lr=2e-3, seed=0, hard=None, pos_frac=0.25):
    """Mini-batches with a fixed share of positives and Adam; negatives are
    drawn uniformly, or half of them from `hard` (indices of hard negatives)
    when given.  Returns the losses seen every 50 steps."""
    torch = __import__("torch")
    rng = np.random.default_rng(seed)
    pos = np.nonzero(y == 1)[0]
    neg = np.nonzero(y == 0)[0]
    npos = max(1, int(round(batch * pos_frac)))
    nneg = batch - npos
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    yd = torch.from_numpy(y).cuda()
    losses = []
    for it in range(steps):
        if hard is not None and hard.size:
            negs = np.concatenate([rng.choice(hard, nneg // 2), rng.choice(neg, nneg - nneg // 2)])
        else:
            negs = rng.choice(neg, nneg)
        idx = torch.from_numpy(np.concatenate([rng.choice(pos, npos), negs])).cuda()
        xb = x.index_select(0, idx).contiguous()
        yb = yd.index_select(0, idx).contiguous()
        gsp.gsp_ranker_train_step(ranker, xb, yb, batch, lr, loss=loss)
        if it % 50 == 0 or it == steps - 1:
            gsp.gsp_ranker_finish(ranker)
            losses.append(float(loss.item()))
    gsp.gsp_ranker_finish(ranker)
    return losses


def fit(ranker, x, y, steps=(400, 800), hard_count=20000, lr=2e-3, seed=0):
    """Two phases: uniform negatives, then with the highest-scored negatives of
    the training set (hard-negative mining) over-sampled."""
    l1 = train(ranker, x, y, steps[0], lr=lr, seed=seed)
    neg = np.nonzero(y == 0)[0]
    s = score(ranker, x)
    hard = neg[np.argsort(-s[neg])[:hard_count]]
    l2 = train(ranker, x, y, steps[1], lr=lr * 0.5, seed=seed + 1, hard=hard)
    return l1 + l2


def score(ranker, x, chunk=None):
    """Softmax probability of class 1 for snippets x (torch CUDA [n][64][64])."""
    torch = __import__("torch")
    n = x.shape[0]
    chunk = chunk or ranker.max_batch
    logits = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    for i in range(0, n, chunk):
        m = min(chunk, n - i)
        gsp.gsp_ranker_forward(ranker, x[i:i + m], m, logits[i:i + m])
    gsp.gsp_ranker_finish(ranker)
    return torch.softmax(logits, dim=1)[:, 1].cpu().numpy()


def evaluate(ranker, src, beams, seed, snr_min=8.0, chunk=4096, threshold=0.5):
    """Score every candidate of fresh beams; recall on injected pulses with
    S/N >= snr_min (of those the search detects), precision, and the ranking
    throughput (snippets + forward)."""
    torch = src.torch
    recalled, detected, strong = 0, 0, 0
    det8, rec8 = 0, 0      # pulses whose best detected S/N (not the nominal one) is >= snr_min
    tp = fp = neg_total = neg_rejected = 0
    n_scored, rank_s = 0, 0.0
    per_pulse = []   # (nominal S/N, width, recalled) of detected pulses with S/N >= snr_min
    for b in range(beams):
        cands, lab, pid, pulses = src.search(b, seed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        scores = np.empty(cands.size, np.float32)
        for i in range(0, cands.size, chunk):
            sub = cands[i:i + chunk]
            torch.cuda.synchronize()
            e0.record()
            x = src.snippets(sub)
            logits = torch.empty((sub.size, 2), dtype=torch.float32, device="cuda")
            gsp.gsp_ranker_forward(ranker, x, sub.size, logits)
            e1.record()
            gsp.gsp_ranker_finish(ranker)
            rank_s += e0.elapsed_time(e1) / 1e3
            scores[i:i + sub.size] = torch.softmax(logits, dim=1)[:, 1].cpu().numpy()
            del x
        n_scored += cands.size
        Ls = (src.n_out // 1024) * 1024
        for i, p in enumerate(pulses):
            if p.snr < snr_min or p.t0 + p.width > Ls:
                continue
            strong += 1
            mine = pid == i
            if mine.any():
                detected += 1
                ok = bool(scores[mine].max() >= threshold)
                recalled += int(ok)
                per_pulse.append((p.snr, p.width, ok))
        # the same over the pulses the search detects at S/N >= snr_min: DM-trial
        # smearing can leave a pulse of nominal S/N >= snr_min near the threshold
        for i, p in enumerate(pulses):
            mine = pid == i
            if p.t0 + p.width > Ls or not mine.any() or cands["snr"][mine].max() < snr_min:
                continue
            det8 += 1
            rec8 += int(scores[mine].max() >= threshold)
        hi = scores >= threshold
        tp += int((hi & (lab == 1)).sum())
        fp += int((hi & (lab == 0)).sum())
        neg_total += int((lab == 0).sum())
        neg_rejected += int((~hi & (lab == 0)).sum())
    pp = np.array(per_pulse, dtype=np.float64).reshape(-1, 3)

    def rec(sel):
        return [int(pp[sel, 2].sum()), int(sel.sum())]

    by_width = {"1-9": rec(pp[:, 1] < 10), "10-49": rec((pp[:, 1] >= 10) & (pp[:, 1] < 50)),
                "50-100": rec(pp[:, 1] >= 50)}
    by_snr = {"8-12": rec(pp[:, 0] < 12), "12-20": rec((pp[:, 0] >= 12) & (pp[:, 0] < 20)),
              "20-30": rec(pp[:, 0] >= 20)}
    return {"threshold": threshold, "recalled_by_width": by_width, "recalled_by_snr": by_snr,
            "pulses_detected_at_snr_ge_min": det8, "recall_detected_snr_ge_min": rec8 / max(det8, 1),
            "pulses_snr_ge_min": strong, "detected_by_search": detected,
            "recall": recalled / max(detected, 1), "precision": tp / max(tp + fp, 1),
            "negatives": neg_total, "negatives_rejected": neg_rejected / max(neg_total, 1),
            "candidates_scored": n_scored, "rank_s": rank_s,
            "candidates_per_s": n_scored / max(rank_s, 1e-9)}
