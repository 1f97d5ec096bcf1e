"""Boundary behaviour of the C ABI on a GPU: every bad call returns a status
(nothing traps), candidate overflow reports the true count, the
host-side fault hooks make allocation and launch failures observable
without any GPU fault, and a bounded wait of the dedispersion pipeline that
runs out (on a barrier nothing completes, with no copy in flight) comes back
as GSP_ERR_TIMEOUT with the plan still usable."""
import os

import numpy as np
import pytest

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


@pytest.fixture
def small(gsp, orc):
    nchan, n_in = 64, 8192
    dms = np.arange(0, 40, 1.0)
    dl, _ = orc.delays(nchan, 1200.0, 1500.0, 1e-4, dms)
    desc, keep = gsp.make_desc(nchan, 1200.0, 1500.0, 1e-4, n_in, dms=dms, max_cands=5,
                               threshold=2.0)
    plan = gsp.gsp_plan_create(desc, keep)
    rng = np.random.default_rng(0)
    x = torch.from_numpy(rng.integers(0, 256, (nchan, n_in), dtype=np.uint8)).cuda()
    return plan, x, dl, n_in


def _status(fn):
    from paper_2110_12749_gb300.gsp import GspError
    try:
        fn()
    except GspError as e:
        return e.status
    return 0


def test_too_short_and_too_long(gsp, small):
    plan, x, dl, n_in = small
    md = gsp.gsp_plan_max_delay(plan)
    out = torch.zeros((40, n_in), dtype=torch.int32, device="cuda")
    assert _status(lambda: gsp.gsp_dedisperse(plan, x, md, out)) == gsp.GSP_ERR_TOO_SHORT
    big = torch.zeros((64, n_in + 64), dtype=torch.uint8, device="cuda")
    assert _status(lambda: gsp.gsp_dedisperse(plan, big, n_in + 16, out)) == gsp.GSP_ERR_INVALID_ARG


def test_misaligned_pointers_and_strides(gsp, small):
    plan, x, dl, n_in = small
    out = torch.zeros((40, n_in), dtype=torch.int32, device="cuda")
    xm = torch.zeros(64 * (n_in + 16) + 1, dtype=torch.uint8, device="cuda")[1:].view(64, n_in + 16)
    assert _status(lambda: gsp.gsp_dedisperse(plan, xm, n_in, out)) == gsp.GSP_ERR_ALIGN
    xs = torch.zeros((64, n_in + 8), dtype=torch.uint8, device="cuda")
    assert _status(lambda: gsp.gsp_dedisperse(plan, xs, n_in, out)) == gsp.GSP_ERR_ALIGN
    om = torch.zeros((40, n_in + 2), dtype=torch.int32, device="cuda")
    assert _status(lambda: gsp.gsp_dedisperse(plan, x, n_in, om)) == gsp.GSP_ERR_ALIGN


def test_candidate_capacity(gsp, small):
    plan, x, dl, n_in = small
    gsp.gsp_search(plan, x, n_in)
    c, n, st = gsp.gsp_candidates(plan)
    assert n > 5 and st == gsp.GSP_ERR_CAPACITY and len(c) == 5
    c2, n2, st2 = gsp.gsp_candidates(plan, cap=2)
    assert n2 == n and st2 == gsp.GSP_ERR_CAPACITY and len(c2) == 2
    assert (c2 == c[:2]).all()


def test_candidates_before_search(gsp, small):
    plan, x, dl, n_in = small
    c, n, st = None, None, None
    assert _status(lambda: gsp.gsp_candidates(plan)) == gsp.GSP_ERR_STATE


def test_series_shorter_than_a_block(gsp, small):
    plan, x, dl, n_in = small
    D = torch.randint(0, 1000, (40, 1000), dtype=torch.int32, device="cuda")
    gsp.gsp_search_series(plan, D, 1000)
    c, n, st = gsp.gsp_candidates(plan)
    assert n == 0 and st == gsp.GSP_OK


def test_fault_hooks(gsp, orc):
    desc, keep = gsp.make_desc(32, 1200.0, 1500.0, 1e-4, 4096, ndm=4)
    os.environ["GSP_FAULT"] = "alloc"
    try:
        assert _status(lambda: gsp.gsp_plan_create(desc, keep)) == gsp.GSP_ERR_OOM
    finally:
        del os.environ["GSP_FAULT"]
    plan = gsp.gsp_plan_create(desc, keep)
    x = torch.zeros((32, 4096), dtype=torch.uint8, device="cuda")
    out = torch.zeros((4, 4096), dtype=torch.int32, device="cuda")
    os.environ["GSP_FAULT"] = "launch"
    try:
        assert _status(lambda: gsp.gsp_dedisperse(plan, x, 4096, out)) == gsp.GSP_ERR_CUDA
        assert _status(lambda: gsp.gsp_search(plan, x, 4096)) == gsp.GSP_ERR_CUDA
    finally:
        del os.environ["GSP_FAULT"]
    gsp.gsp_dedisperse(plan, x, 4096, out)          # the plan still works afterwards
    torch.cuda.synchronize()


def test_tie_margin_rejected(gsp):
    # t_samp chosen so that some delay lands on an exact half sample:
    # DM 1 between the channel centres 1000.5 and 1001.5 of a 2-channel band
    f1, f2 = 1000.5, 1001.5
    x = 4.148808e3 * 1.0 * (1.0 / (f1 * f1) - 1.0 / (f2 * f2))
    desc, keep = gsp.make_desc(2, 1000.0, 1002.0, x / 0.5, 4096, dms=[1.0])
    dl, m = gsp.gsp_compute_delays(desc)
    if m < 1e-9:
        assert _status(lambda: gsp.gsp_plan_create(desc, keep)) == gsp.GSP_ERR_TIE
    else:
        pytest.skip("FP64 did not land within 1e-9 of the tie (margin %g)" % m)


def test_wait_that_runs_out_reports_timeout_and_plan_recovers(gsp, orc, small):
    plan, x, dl, n_in = small
    _, used = gsp.gsp_dedisperse_variants(plan)
    assert used >= 0
    # the producer issues nothing, so each consumer's first stage wait runs out
    # after about 1 ms (2e6 SM cycles); nothing is in flight when the warps leave
    gsp.gsp_plan_set_wait_limit(plan, 2_000_000, 1)
    gsp.gsp_search(plan, x, n_in)
    with pytest.raises(gsp.GspError) as e:
        gsp.gsp_candidates(plan)
    assert e.value.status == gsp.GSP_ERR_TIMEOUT
    # normal limits again: the same plan searches correctly
    gsp.gsp_plan_set_wait_limit(plan, 4_000_000_000, 0)
    n_out = n_in - orc.max_delay(dl)
    D = torch.zeros((dl.shape[0], (n_out + 3) // 4 * 4), dtype=torch.int32, device="cuda")
    gsp.gsp_search(plan, x, n_in, 0, D)
    _, n, st = gsp.gsp_candidates(plan)
    assert st in (gsp.GSP_OK, gsp.GSP_ERR_CAPACITY) and n > 0
    ref = orc.dedisperse(x.cpu().numpy(), n_in, dl)
    assert (D[:, :n_out].cpu().numpy().astype(np.int64) == ref).all()
    for bad in [(0, 0), (5_000_000_000, 0), (100, 2)]:
        with pytest.raises(gsp.GspError):
            gsp.gsp_plan_set_wait_limit(plan, *bad)
