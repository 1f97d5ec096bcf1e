"""Long dispersion sweeps on the tiled dedispersion kernel (Sec. 2.3, Alg. 3
with the merged buffer spanning the whole sweep).

A plan whose largest delay spread inside a block of DM trials does not fit
two 64-channel shared-memory stages must still run on a tiled variant (32-
channel stages or 7-DM blocks), never silently on the simple kernel.  The
cases are the wide-band workload (2048 channels, 500-3300 MHz, 3000 DMs
0-2999, largest delay 493269 samples) and the worst beam of the batched
workload (4096 channels, 1000-1500 MHz, 1000 trials to DM 1500, step 1.5).
Each runs on an input a little longer than its largest delay, so that the
oracle can dedisperse every row: every row bit-exact, the fused block sums
through the candidates of every row (oracle search, comparison rule of the
other parity tests), for the automatic choice and for each variant that fits.
"""
import numpy as np
import pytest

from helpers import compare_candidates, window_contenders

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# name: (nchan, f_lo, f_hi, t_samp, ndm, dm_step, variants that must fit)
CASES = {
    "wideband": (2048, 500.0, 3300.0, 98.304e-6, 3000, 1.0, (42, 43, 34, 44)),
    "batch_worst_beam": (4096, 1000.0, 1500.0, 49.152e-6, 1000, 1.5, (42, 43, 34)),
}
N_EXTRA = 20480     # output samples beyond the largest delay


@pytest.fixture(scope="module")
def gsp():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_12749_gb300 import build, gsp as g
    build.build()
    g.lib()
    return g


@pytest.fixture(scope="module")
def sweeps(orc):
    from paper_2110_12749_gb300 import synth
    out = {}
    for name, (nchan, f_lo, f_hi, ts, ndm, step, _) in CASES.items():
        dms = np.arange(ndm) * step
        dl, _ = orc.delays(nchan, f_lo, f_hi, ts, dms)
        md = orc.max_delay(dl)
        n_in = md + N_EXTRA + 1000
        n_out = n_in - md
        # Gaussian noise with three dispersed pulses (delays from the oracle)
        pulses = []
        for k, (frac, w) in enumerate([(0.2, 3), (0.55, 12), (0.9, 40)]):
            d = int(frac * (ndm - 1))
            pulses.append(synth.Pulse(dm=float(dms[d]), t0=3000 + 6000 * k, width=w, snr=25.0,
                                      amp=synth.pulse_amplitude(25.0, 20.0, nchan, w),
                                      delays=dl[d]))
        x = synth.filterbank(nchan, n_in, 4242 + len(name), 128.0, 20.0, pulses=pulses)
        D = orc.dedisperse(x, n_in, dl)
        out[name] = (x, n_in, dl, D)
    return out


def test_long_sweep_plans_report_a_tiled_variant(gsp):
    # full-size plans (2^20 samples) of both workloads and a still coarser grid
    for nchan, f_lo, f_hi, ts, ndm, step in [
            (2048, 500.0, 3300.0, 98.304e-6, 3000, 1.0),
            (4096, 1000.0, 1500.0, 49.152e-6, 1000, 1.5),
            (2048, 500.0, 3300.0, 98.304e-6, 1500, 2.0)]:
        desc, keep = gsp.make_desc(nchan, f_lo, f_hi, ts, 1 << 20, ndm=ndm, dm_step=step)
        plan = gsp.gsp_plan_create(desc, keep)
        _, used = gsp.gsp_dedisperse_variants(plan)
        assert used >= 0, (nchan, ndm, step)
        gsp.gsp_plan_destroy(plan)


@pytest.mark.parametrize("name", sorted(CASES))
def test_long_sweep_every_row_bit_exact(gsp, orc, sweeps, monkeypatch, name):
    nchan, f_lo, f_hi, ts, ndm, step, fitting = CASES[name]
    x, n_in, dl, Dref = sweeps[name]
    n_out = Dref.shape[1]
    xd = torch.from_numpy(x).cuda()
    stride = (n_out + 3) // 4 * 4
    ora, _ = orc.search_rows(Dref)
    contenders = {}
    for v in (None,) + tuple(fitting):
        if v is None:
            monkeypatch.delenv("GSP_DD_VARIANT", raising=False)
        else:
            monkeypatch.setenv("GSP_DD_VARIANT", str(v))
        desc, keep = gsp.make_desc(nchan, f_lo, f_hi, ts, n_in, ndm=ndm, dm_step=step,
                                   max_cands=ndm * (n_out // 1024 + 2))
        plan = gsp.gsp_plan_create(desc, keep)
        _, used = gsp.gsp_dedisperse_variants(plan)
        assert used >= 0 and (v is None or used == v), (v, used)
        D = torch.full((ndm, stride), -7, dtype=torch.int32, device="cuda")
        gsp.gsp_search(plan, xd, n_in, 0, D)
        cands, n, st = gsp.gsp_candidates(plan)
        assert st == gsp.GSP_OK
        got = D[:, :n_out].cpu().numpy().astype(np.int64)
        assert (got == Dref).all(), (v, np.argwhere(got != Dref)[:5])
        assert (D[:, n_out:] == -7).all()
        ncmp, bad = compare_candidates(cands, ora, 6.0, 1024, 0, contenders)
        if bad:
            # screen the windows of the rows that differ for ambiguous maxima
            for b in bad:
                r = int(b.split(",")[0].strip("("))
                if r not in contenders:
                    contenders[r] = window_contenders(
                        orc.search_row(Dref[r], dm_idx=r, detail=True), 1024, 0, 6.0)
            ncmp, bad = compare_candidates(cands, ora, 6.0, 1024, 0, contenders)
        assert not bad, (v, bad[:5])
        assert ncmp > 0
        gsp.gsp_plan_destroy(plan)
