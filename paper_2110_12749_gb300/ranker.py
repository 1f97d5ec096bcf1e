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
threshold is chosen on held-out validation beams (the score that keeps 99%
of their pulses the search detects at S/N >= 8), never on the training or
the evaluation beams.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import gsp, synth


def short_crafts(n_in=1 << 18, n_pulses=40):
    """The CRAFTS-like beam (4096 channels, 2000 trials) cut to n_in samples."""
    return dataclasses.replace(synth.WORKLOADS["crafts"], n_in=n_in, n_pulses=n_pulses)


def learned_crafts(n_in=1 << 18, n_pulses=40):
    """The learned + streaming workload's beams: CRAFTS-shaped chunks (4096
    channels, 1000-1500 MHz, 49.152 us, 2^18 samples) with pulses injected at DM
    10-1500, width 1-150 samples and S/N 5-40, searched over 2000 trials 0-1499.25
    (step 0.75) so that every injected DM lies inside the grid."""
    return dataclasses.replace(synth.WORKLOADS["crafts"], name="learned", n_in=n_in,
                               dm_step=0.75, n_pulses=n_pulses, pulse_dm=(10.0, 1500.0),
                               pulse_w=(1, 150), pulse_snr=(5.0, 40.0))


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


def subsample(x, y, pid, total, seed, width=None):
    """Keep every positive and a seeded random subset of the negatives so that
    `total` snippets remain (all of them if there are fewer).  `width` (per
    snippet, optional) is subset alike and returned last."""
    torch = __import__("torch")
    pos = np.nonzero(y == 1)[0]
    neg = np.nonzero(y == 0)[0]
    if pos.size + neg.size <= total:
        return (x, y, pid) if width is None else (x, y, pid, width)
    rng = np.random.default_rng(seed)
    keep = np.sort(np.concatenate([pos, rng.choice(neg, max(total - pos.size, 0),
                                                   replace=False)]))
    idx = torch.from_numpy(keep).cuda()
    out = (x.index_select(0, idx), y[keep], pid[keep])
    return out if width is None else out + (width[keep],)


class ScoredBeams:
    """Searched beams whose candidates, labels, pulses and snippets are kept, so
    that several rankers can be scored on the same beams (validation and
    evaluation sets)."""

    def __init__(self, src, beams, seed):
        torch = __import__("torch")
        self.items = []
        self.snip_s = 0.0   # device time of the snippet extraction (CUDA events)
        for b in range(beams):
            cands, lab, pid, pulses = src.search(b, seed)
            Ls = (src.n_out // 1024) * 1024
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            x = src.snippets(cands)
            e1.record()
            torch.cuda.synchronize()
            self.snip_s += e0.elapsed_time(e1) / 1e3
            self.items.append((cands, lab, pid, pulses, x, Ls))

    def scores(self, ranker, chunk=4096):
        """pulse_scores() of this set for one ranker."""
        torch = __import__("torch")
        nominal, width, det, best, best8 = [], [], [], [], []
        neg, pos, neg_snr, pos_snr = [], [], [], []
        n_scored, rank_s = 0, self.snip_s
        for cands, lab, pid, pulses, x, Ls in self.items:
            scores = np.empty(cands.size, np.float32)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for i in range(0, cands.size, chunk):
                m = min(chunk, cands.size - i)
                logits = torch.empty((m, 2), dtype=torch.float32, device="cuda")
                torch.cuda.synchronize()
                e0.record()
                gsp.gsp_ranker_forward(ranker, x[i:i + m], m, logits)
                e1.record()
                gsp.gsp_ranker_finish(ranker)
                rank_s += e0.elapsed_time(e1) / 1e3
                scores[i:i + m] = torch.softmax(logits, dim=1)[:, 1].cpu().numpy()
            n_scored += cands.size
            for i, p in enumerate(pulses):
                if p.t0 + p.width > Ls:
                    continue
                mine = pid == i
                nominal.append(p.snr)
                width.append(p.width)
                det.append(float(cands["snr"][mine].max()) if mine.any() else -1.0)
                best.append(float(scores[mine].max()) if mine.any() else -1.0)
                m8 = mine & (cands["snr"] >= 8.0)
                best8.append(float(scores[m8].max()) if m8.any() else -1.0)
            neg.append(scores[lab == 0])
            pos.append(scores[lab == 1])
            neg_snr.append(cands["snr"][lab == 0])
            pos_snr.append(cands["snr"][lab == 1])
        return {"nominal": np.array(nominal), "width": np.array(width),
                "detected": np.array(det), "best": np.array(best), "best8": np.array(best8),
                "neg": np.concatenate(neg), "pos": np.concatenate(pos),
                "neg_snr": np.concatenate(neg_snr), "pos_snr": np.concatenate(pos_snr),
                "n_scored": n_scored, "rank_s": rank_s, "snip_s": self.snip_s}


def build_training_set(src, beams, seed, with_width=False):
    """Snippets (torch float CUDA) and labels of every candidate labelled 0 or
    1 in the given number of beams (candidates on a pulse's track excluded),
    a global pulse id per snippet (-1 for label 0) and the nominal S/N of
    every pulse (indexed by that id); with_width also the candidate widths."""
    torch = src.torch
    xs, ys, ps, snr, ws = [], [], [], [], []
    base = 0
    for b in range(beams):
        cands, lab, pid, pulses = src.search(b, seed)
        keep = lab >= 0
        xs.append(src.snippets(cands[keep]))
        ys.append(lab[keep].astype(np.int32))
        ps.append(np.where(pid[keep] >= 0, pid[keep] + base, -1))
        ws.append(cands["width"][keep].astype(np.int32))
        snr.extend(p.snr for p in pulses)
        base += len(pulses)
    out = (torch.cat(xs), np.concatenate(ys), np.concatenate(ps), np.array(snr))
    return out + (np.concatenate(ws),) if with_width else out


def pulse_scores(ranker, src, beams, seed, chunk=4096):
    """Score every candidate of the given beams.  Returns a dict with, per
    injected pulse that ends inside the searched blocks, its nominal S/N and
    width, its best detected S/N and its best score (both -1 if the search finds none of
    its core candidates); the scores of the candidates labelled 0 and 1; the
    candidates scored and the seconds spent on snippets + forward passes."""
    torch = src.torch
    nominal, width, det, best, neg, pos = [], [], [], [], [], []
    n_scored, rank_s = 0, 0.0
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
            if p.t0 + p.width > Ls:
                continue
            mine = pid == i
            nominal.append(p.snr)
            width.append(p.width)
            det.append(float(cands["snr"][mine].max()) if mine.any() else -1.0)
            best.append(float(scores[mine].max()) if mine.any() else -1.0)
        neg.append(scores[lab == 0])
        pos.append(scores[lab == 1])
    return {"nominal": np.array(nominal), "width": np.array(width), "detected": np.array(det),
            "best": np.array(best),
            "neg": np.concatenate(neg), "pos": np.concatenate(pos), "n_scored": n_scored,
            "rank_s": rank_s}


def threshold_for(ps, snr_min=8.0, keep=0.99):
    """The score that keeps `keep` of the pulses in pulse_scores output `ps`
    that the search detects at S/N >= snr_min (each by its best core
    candidate; with per-candidate S/N, its best core candidate detected at
    S/N >= snr_min), at most 0.5; 0.5 if there are none."""
    v = np.sort((ps["best8"] if "best8" in ps else ps["best"])[ps["detected"] >= snr_min])
    if v.size == 0:
        return 0.5
    return float(min(0.5, v[int(np.floor((1.0 - keep) * v.size))]))


def choose_threshold(ranker, src, beams, seed, snr_min=8.0, keep=0.99):
    """Operating threshold from validation beams (threshold_for over them)."""
    return threshold_for(pulse_scores(ranker, src, beams, seed), snr_min, keep)


def train(ranker, x, y, steps, batch=256, lr=2e-3, seed=0, hard=None, pos_frac=0.25,
          wide=None):
    """Mini-batches with a fixed share of positives and Adam; negatives are
    drawn uniformly, or half of them from `hard` (indices of hard negatives)
    when given; positives uniformly, or half of them from `wide` (indices of
    wide positives, the rare hard class) when given.  Returns the losses seen
    every 50 steps."""
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
        if wide is not None and wide.size:
            poss = np.concatenate([rng.choice(wide, npos // 2), rng.choice(pos, npos - npos // 2)])
        else:
            poss = rng.choice(pos, npos)
        idx = torch.from_numpy(np.concatenate([poss, negs])).cuda()
        xb = x.index_select(0, idx).contiguous()
        yb = yd.index_select(0, idx).contiguous()
        gsp.gsp_ranker_train_step(ranker, xb, yb, batch, lr, loss=loss)
        if it % 50 == 0 or it == steps - 1:
            gsp.gsp_ranker_finish(ranker)
            losses.append(float(loss.item()))
    gsp.gsp_ranker_finish(ranker)
    return losses


def fit(ranker, x, y, steps=(400, 800), hard_count=20000, lr=2e-3, seed=0, wide=None):
    """Two phases: uniform negatives, then with the highest-scored negatives of
    the training set (hard-negative mining) over-sampled; `wide` (indices of
    wide positives) are over-sampled in both."""
    l1 = train(ranker, x, y, steps[0], lr=lr, seed=seed, wide=wide)
    neg = np.nonzero(y == 0)[0]
    s = score(ranker, x)
    hard = neg[np.argsort(-s[neg])[:hard_count]]
    l2 = train(ranker, x, y, steps[1], lr=lr * 0.5, seed=seed + 1, hard=hard, wide=wide)
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


def evaluate(ranker, src, beams, seed, snr_min=8.0, thresholds=(0.5,)):
    """Score every candidate of fresh beams and summarise (see summarise)."""
    return summarise(pulse_scores(ranker, src, beams, seed), snr_min, thresholds)


def summarise(ps, snr_min=8.0, thresholds=(0.5,)):
    """Quality of the scores in pulse_scores output `ps`.  At each threshold
    (the first one as a two-tier operating point when `ps` has per-candidate
    S/N: score >= threshold at detected S/N >= snr_min, score >= 0.5 below):
    recall on the injected pulses the search detects at S/N >= snr_min,
    recall on those of nominal S/N >= snr_min that it detects at all,
    precision and the share of negatives rejected; for the first threshold
    also [recalled, pulses] by width and by detected S/N, and the missed
    pulses detected at S/N >= snr_min ([nominal S/N, width, detected S/N,
    score], at most 10).  Plus the ranking throughput (snippets + forward)."""
    nom, wid, det, best = ps["nominal"], ps["width"], ps["detected"], ps["best"]
    d8 = det >= snr_min                       # detected at S/N >= snr_min
    n8 = (nom >= snr_min) & (det >= 0)        # nominal S/N >= snr_min, detected
    at = {}
    for t in thresholds:
        tp, fp = int((ps["pos"] >= t).sum()), int((ps["neg"] >= t).sum())
        at[t] = {"recall": float((best[d8] >= t).mean()) if d8.any() else 0.0,
                 "recall_nominal": float((best[n8] >= t).mean()) if n8.any() else 0.0,
                 "precision": tp / max(tp + fp, 1),
                 "negatives_rejected": 1.0 - fp / max(ps["neg"].size, 1)}
        if "pos_snr" in ps:
            # the same over the candidates the search reports at S/N >= snr_min
            tp8 = int(((ps["pos"] >= t) & (ps["pos_snr"] >= snr_min)).sum())
            fp8 = int(((ps["neg"] >= t) & (ps["neg_snr"] >= snr_min)).sum())
            at[t]["precision_snr_ge_min"] = tp8 / max(tp8 + fp8, 1)
    t0 = thresholds[0]
    ok = best >= t0
    if "best8" in ps:
        # two-tier operating point: candidates detected at S/N >= snr_min are kept
        # at score >= t0, weaker ones at score >= 0.5 (the recall target is set at
        # S/N >= snr_min; the many faint noise candidates below it need a confident score)
        lo = max(t0, 0.5)
        ok = (ps["best8"] >= t0) | (best >= lo)
        kp = ((ps["pos"] >= t0) & (ps["pos_snr"] >= snr_min)) | (ps["pos"] >= lo)
        kn = ((ps["neg"] >= t0) & (ps["neg_snr"] >= snr_min)) | (ps["neg"] >= lo)
        tp, fp = int(kp.sum()), int(kn.sum())
        at[t0] = {"recall": float(ok[d8].mean()) if d8.any() else 0.0,
                  "recall_nominal": float(ok[n8].mean()) if n8.any() else 0.0,
                  "precision": tp / max(tp + fp, 1),
                  "negatives_rejected": 1.0 - fp / max(ps["neg"].size, 1),
                  "precision_snr_ge_min": at[t0].get("precision_snr_ge_min")}

    def rec(sel):
        sel = sel & d8
        return [int((ok & sel).sum()), int(sel.sum())]

    out = dict(at[t0])
    out.update({
        "threshold": t0,
        "pulses_detected_snr_ge_min": int(d8.sum()),
        "pulses_nominal_snr_ge_min": int((nom >= snr_min).sum()),
        "nominal_snr_ge_min_detected": int(n8.sum()),
        "recalled_by_width": {"1-9": rec(wid < 10), "10-49": rec((wid >= 10) & (wid < 50)),
                              "50-150": rec(wid >= 50)},
        "recalled_by_snr": {"8-12": rec(det < 12), "12-20": rec((det >= 12) & (det < 20)),
                            ">=20": rec(det >= 20)},
        "negatives": int(ps["neg"].size), "candidates_scored": ps["n_scored"],
        "rank_s": ps["rank_s"], "candidates_per_s": ps["n_scored"] / max(ps["rank_s"], 1e-9),
        "snippets_per_s": (ps["n_scored"] / ps["snip_s"]) if ps.get("snip_s") else None,
        "forward_per_s": (ps["n_scored"] / (ps["rank_s"] - ps["snip_s"]))
                         if ps.get("snip_s") and ps["rank_s"] > ps["snip_s"] else None,
        "missed": [[round(float(nom[i]), 2), int(wid[i]), round(float(det[i]), 2),
                    round(float(best[i]), 4)] for i in np.nonzero(d8 & ~ok)[0][:10]],
        "at": {"%.4g" % t: at[t] for t in thresholds[1:]}})
    return out
