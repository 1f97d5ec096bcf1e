"""Streaming search (gsp_stream_*): chunks admitted one after another with the
dispersion-overlap tail kept on the device.  Every chunk's candidates must
equal a one-shot gsp_search of the same input span (with the same absolute
offset), and match the CPU oracle on that span."""
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


def test_stream_chunks_equal_one_shot_spans(gsp, orc):
    from paper_2110_12749_gb300 import synth
    nchan, ts, chunk, nchunks = 128, 1e-4, 4096, 4
    dms = np.arange(0.0, 64.0, 1.0)
    dl, _ = orc.delays(nchan, 1200.0, 1500.0, ts, dms)
    md = orc.max_delay(dl)
    n_total = md + nchunks * chunk
    pulses = []
    for k, (dm, t0, w) in enumerate([(20.0, 4090, 3), (41.0, 9000, 8), (12.5, 12287, 2)]):
        d1, _ = orc.delays(nchan, 1200.0, 1500.0, ts, [dm])
        pulses.append(synth.Pulse(dm, t0, w, 18.0, synth.pulse_amplitude(18.0, 16.0, nchan, w),
                                  d1[0]))
    x = synth.filterbank(nchan, n_total, 77, 128.0, 16.0, pulses=pulses, threads=4)
    desc, keep = gsp.make_desc(nchan, 1200.0, 1500.0, ts, chunk + md, dms=dms, threshold=5.0)
    plan = gsp.gsp_plan_create(desc, keep)
    s = gsp.gsp_stream_create(plan, chunk, beam=3)
    ref_desc, ref_keep = gsp.make_desc(nchan, 1200.0, 1500.0, ts, chunk + md, dms=dms, threshold=5.0)
    ref = gsp.gsp_plan_create(ref_desc, ref_keep)
    total = 0
    for k in range(nchunks):
        need = gsp.gsp_stream_need(s)
        assert need == (chunk + md if k == 0 else chunk)
        lo = 0 if k == 0 else md + k * chunk
        part = np.ascontiguousarray(x[:, lo:lo + need])
        gsp.gsp_stream_push(s, part, need)
        got, n, st, t_abs0 = gsp.gsp_stream_results(s)
        assert st == gsp.GSP_OK and t_abs0 == k * chunk
        assert (got["beam"] == 3).all()
        # the same span searched in one shot
        span = np.zeros((nchan, (chunk + md + 15) // 16 * 16), np.uint8)
        span[:, :chunk + md] = x[:, k * chunk:k * chunk + chunk + md]
        gsp.gsp_search(ref, torch.from_numpy(span).cuda(), chunk + md, t_offset=k * chunk)
        want, nw, _ = gsp.gsp_candidates(ref)
        assert n == nw
        assert (got["t"] == want["t"] + k * chunk).all()
        assert (got["dm_idx"] == want["dm_idx"]).all() and (got["width"] == want["width"]).all()
        assert (got["snr"] == want["snr"]).all()
        # and the oracle on that span
        D = orc.dedisperse(span, chunk + md, dl)
        cont, ora = {}, []
        for r in range(len(dms)):
            det = orc.search_row(D[r], dm_idx=r, threshold=5.0, t_offset=k * chunk, detail=True)
            cont[r] = window_contenders(det, 1024, k * chunk, 5.0)
            ora.append(det["cands"])
        ora = np.concatenate(ora)
        rel = got.copy()
        rel["t"] -= k * chunk
        ncmp, bad = compare_candidates(rel, ora, 5.0, 1024, k * chunk, cont)
        assert not bad, bad[:5]
        total += ncmp
    assert total > 0
    # wrong chunk size is refused
    with pytest.raises(gsp.GspError):
        gsp.gsp_stream_push(s, np.zeros((nchan, chunk + 16), np.uint8), chunk + 16)
    gsp.gsp_stream_destroy(s)


def test_stream_bytes_for_admission(gsp, orc):
    nchan, chunk = 64, 4096
    desc, keep = gsp.make_desc(nchan, 1200.0, 1500.0, 1e-4, 1 << 16, ndm=32, dm_lo=0.0,
                               dm_step=1.0)
    plan = gsp.gsp_plan_create(desc, keep)
    md = gsp.gsp_plan_max_delay(plan)
    bufs = 2 * ((chunk + md + 15) // 16 * 16) * nchan
    scratch = 32 * (((1 << 16) - md + 3) // 4 * 4) * 4
    assert gsp.gsp_stream_bytes(plan, chunk) == bufs + scratch   # plan not searched yet
    s = gsp.gsp_stream_create(plan, chunk)
    x = np.zeros((nchan, chunk + md), np.uint8)
    gsp.gsp_stream_push(s, x, gsp.gsp_stream_need(s))
    gsp.gsp_stream_results(s)
    assert gsp.gsp_stream_bytes(plan, chunk) == bufs               # scratch now exists
    assert gsp.gsp_stream_bytes(plan, 0) == -1
    gsp.gsp_stream_destroy(s)


def test_pooled_streams_share_buffers_and_refuse_when_full(gsp, orc):
    # two beams with their own DM grids (different overlap tails) draw their input
    # buffers from one pool of a single buffer: a chunk is admitted only when the
    # buffer's previous chunk has run, and every chunk equals a one-shot search
    from paper_2110_12749_gb300 import synth
    nchan, ts, chunk, nchunks = 96, 1e-4, 4096, 3
    grids = [np.arange(0.0, 64.0, 1.0), np.arange(0.0, 60.0, 1.5)]
    beams = []
    for b, dms in enumerate(grids):
        dl, _ = orc.delays(nchan, 1200.0, 1500.0, ts, dms)
        md = orc.max_delay(dl)
        x = synth.filterbank(nchan, md + nchunks * chunk, 300 + b, 128.0, 16.0, threads=4)
        desc, keep = gsp.make_desc(nchan, 1200.0, 1500.0, ts, chunk + md, dms=dms, threshold=5.0)
        rdesc, rkeep = gsp.make_desc(nchan, 1200.0, 1500.0, ts, chunk + md, dms=dms, threshold=5.0)
        beams.append(dict(dms=dms, md=md, x=x, plan=gsp.gsp_plan_create(desc, keep),
                          ref=gsp.gsp_plan_create(rdesc, rkeep)))
    max_tail = max(b["md"] for b in beams)
    pool = gsp.gsp_chunkpool_create(nchan, chunk, max_tail, 1)
    assert gsp.gsp_chunkpool_bytes(nchan, chunk, max_tail, 1) == nchan * ((chunk + max_tail + 15) // 16 * 16)
    for b, bm in enumerate(beams):
        before = gsp.gsp_stream_pooled_bytes(bm["plan"], chunk)
        assert before == ((bm["md"] + 15) // 16 * 16) * nchan + \
            len(bm["dms"]) * ((chunk + 3) // 4 * 4) * 4
        bm["s"] = gsp.gsp_stream_create_pooled(bm["plan"], pool, beam=10 + b)
    cs = torch.cuda.Stream()
    refused = 0
    for k in range(nchunks):
        for b, bm in enumerate(beams):
            s, md, x = bm["s"], bm["md"], bm["x"]
            need = gsp.gsp_stream_need(s)
            lo = 0 if k == 0 else md + k * chunk
            part = np.ascontiguousarray(x[:, lo:lo + need])
            if k == 1 and b == 1:
                # the other beam's chunk holds the only buffer while its stream sleeps
                # (pinned host memory: the push returns while its copy waits behind the sleep)
                other = beams[0]
                ahead = torch.from_numpy(np.ascontiguousarray(
                    other["x"][:, other["md"] + 2 * chunk:other["md"] + 3 * chunk])).pin_memory()
                with torch.cuda.stream(cs):
                    torch.cuda._sleep(20_000_000)
                    assert gsp.gsp_stream_push(other["s"], ahead, chunk, stream=cs, busy_ok=True)
                assert not gsp.gsp_stream_push(s, part, need, busy_ok=True)  # not admitted
                refused += 1
                assert gsp.gsp_chunkpool_free(pool) == 0
                g, n, st, t0 = gsp.gsp_stream_results(other["s"])          # waits for it
                assert st == gsp.GSP_OK and t0 == 2 * chunk
                other["pushed_ahead"] = True
            if b == 0 and beams[0].get("pushed_ahead") and k == 2:
                continue                                  # beam 0's chunk 2 went in early
            assert gsp.gsp_stream_push(s, part, need, busy_ok=True)
            got, n, st, t_abs0 = gsp.gsp_stream_results(s)
            assert st == gsp.GSP_OK and t_abs0 == k * chunk
            assert (got["beam"] == 10 + b).all()
            span = np.zeros((nchan, (chunk + md + 15) // 16 * 16), np.uint8)
            span[:, :chunk + md] = x[:, k * chunk:k * chunk + chunk + md]
            gsp.gsp_search(bm["ref"], torch.from_numpy(span).cuda(), chunk + md, t_offset=k * chunk)
            want, nw, _ = gsp.gsp_candidates(bm["ref"])
            assert n == nw, (k, b)
            assert (got["t"] == want["t"] + k * chunk).all()
            assert (got["dm_idx"] == want["dm_idx"]).all() and (got["snr"] == want["snr"]).all()
    assert refused == 1
    torch.cuda.synchronize()
    assert gsp.gsp_chunkpool_free(pool) == 1
    for bm in beams:
        gsp.gsp_stream_destroy(bm["s"])
    gsp.gsp_chunkpool_destroy(pool)
