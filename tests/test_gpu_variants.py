"""Every tile variant of the tiled dedispersion kernel against the CPU oracle,
bit-exact.  The cases cover a ragged channel count (the last channel stage is
partly filled), a partial DM block, several time tiles with a ragged tail,
and saturated input (every byte 255: the worst case for the 16-bit SWAR
lanes, 256 channels x 255 per lane between flushes).  Each variant's fused
block sums are checked too: a fused gsp_search must give the same candidates
and block statistics as the search of the oracle's series."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (nchan, ndm, n_in, highest DM, saturated input, seed)
CASES = [
    (300, 37, 6000, 60.0, False, 11),
    (517, 20, 4500, 30.0, True, 12),
]


@pytest.fixture(scope="module")
def gsp():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_12749_gb300 import build, gsp as g
    build.build()
    g.lib()
    return g


@pytest.fixture(scope="module")
def cases(orc):
    out = []
    for nchan, ndm, n_in, dm_hi, sat, seed in CASES:
        rng = np.random.default_rng(seed)
        dms = np.sort(rng.uniform(0.0, dm_hi, ndm))
        dl, _ = orc.delays(nchan, 1200.0, 1500.0, 1e-4, dms)
        stride = (n_in + 15) // 16 * 16
        if sat:
            x = np.full((nchan, stride), 255, np.uint8)
        else:
            x = rng.integers(0, 256, (nchan, stride), dtype=np.uint8)
        out.append((nchan, dms, n_in, x, orc.dedisperse(x, n_in, dl)))
    return out


def test_every_variant_bit_exact(gsp, cases, monkeypatch):
    nvar, _ = gsp.gsp_dedisperse_variants()
    assert nvar >= 1
    bad = []
    for v in range(nvar):
        monkeypatch.setenv("GSP_DD_VARIANT", str(v))
        for ci, (nchan, dms, n_in, x, Dref) in enumerate(cases):
            desc, keep = gsp.make_desc(nchan, 1200.0, 1500.0, 1e-4, n_in, dms=dms, threshold=4.0)
            plan = gsp.gsp_plan_create(desc, keep)
            _, used = gsp.gsp_dedisperse_variants(plan)
            assert used == v, (v, used)
            n_out = Dref.shape[1]
            xd = torch.from_numpy(x).cuda()
            out = torch.full((len(dms), (n_out + 3) // 4 * 4 + 4), -7, dtype=torch.int32,
                             device="cuda")
            gsp.gsp_dedisperse(plan, xd, n_in, out)
            o = out.cpu().numpy()
            if not (o[:, :n_out].astype(np.int64) == Dref).all():
                r, t = np.argwhere(o[:, :n_out] != Dref)[0]
                bad.append("variant %d case %d: D[%d][%d] = %d, oracle %d"
                           % (v, ci, r, t, o[r, t], Dref[r, t]))
                continue
            if (o[:, n_out:] != -7).any():
                bad.append("variant %d case %d: wrote past the row" % (v, ci))
            # fused block sums of this variant == block sums of the series
            gsp.gsp_search(plan, xd, n_in)
            c1, n1, _ = gsp.gsp_candidates(plan)
            s1 = gsp.gsp_search_stats(plan, n_out)
            gsp.gsp_search_series(plan, torch.from_numpy(Dref.astype(np.int32)).cuda(), n_out)
            c2, n2, _ = gsp.gsp_candidates(plan)
            s2 = gsp.gsp_search_stats(plan, n_out)
            if n1 != n2 or not (c1 == c2).all() or not (s1["sigma_b"] == s2["sigma_b"]).all():
                bad.append("variant %d case %d: fused search differs" % (v, ci))
    assert not bad, bad
