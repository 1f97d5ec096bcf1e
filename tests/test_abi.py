"""CPU-only checks of the C ABI: the library loads, exports every entry point
that include/gsp.h declares, computes the same delay table as the oracle
(bit-exact, the parity basis of the dedispersion), and rejects bad input
without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gsp():
    from paper_2110_12749_gb300 import build, gsp as g
    build.build()
    g.lib()
    return g


def _declared():
    src = open(os.path.join(ROOT, "include", "gsp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gsp_[a-z_0-9]+)\s*\(", src)))


def test_header_symbols_exported(gsp):
    names = _declared()
    assert len(names) >= 18
    L = ctypes.CDLL(gsp.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_header(gsp):
    for n in _declared():
        assert hasattr(gsp, n), n


def test_variant_count_without_plan(gsp):
    n, used = gsp.gsp_dedisperse_variants()
    assert n >= 1 and used is None


def test_struct_layout(gsp):
    assert ctypes.sizeof(gsp.gsp_plan_desc) == 136
    assert gsp.CAND_DTYPE.itemsize == 24


@pytest.mark.parametrize("name", ["tiny", "crafts", "wideband"])
def test_host_delay_table_equals_oracle(gsp, orc, name):
    from paper_2110_12749_gb300 import synth
    wl = synth.WORKLOADS[name]
    desc, keep = gsp.make_desc(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.n_in,
                               ndm=wl.ndm, dm_lo=wl.dm_lo, dm_step=wl.dm_step)
    lib_dl, lib_m = gsp.gsp_compute_delays(desc)
    ora_dl, ora_m = orc.delays(wl.nchan, wl.f_lo, wl.f_hi, wl.t_samp, wl.dms)
    assert (lib_dl == ora_dl).all()
    assert lib_m == ora_m


def test_host_delay_table_descending_and_explicit_dms(gsp, orc):
    dms = np.array([0.0, 3.3, 17.0, 250.125])
    desc, keep = gsp.make_desc(300, 700.0, 1800.0, 64e-6, 1 << 16, dms=dms, freq_descending=True)
    lib_dl, _ = gsp.gsp_compute_delays(desc)
    ora_dl, _ = orc.delays(300, 700.0, 1800.0, 64e-6, dms, descending=True)
    assert (lib_dl == ora_dl).all()


def test_invalid_descriptors_rejected_on_host(gsp):
    for kw in [dict(f_lo=-1.0), dict(f_hi=1000.0), dict(t_samp=0.0)]:
        args = dict(nchan=64, f_lo=1200.0, f_hi=1500.0, t_samp=1e-4, nsamp_max=4096)
        args.update(kw)
        desc, keep = gsp.make_desc(ndm=4, **args)
        with pytest.raises(gsp.GspError) as e:
            gsp.gsp_compute_delays(desc)
        assert e.value.status == gsp.GSP_ERR_INVALID_ARG
    desc, keep = gsp.make_desc(64, 1200.0, 1500.0, 1e-4, 4096, dms=[1.0, -2.0])
    with pytest.raises(gsp.GspError):
        gsp.gsp_compute_delays(desc)


def test_status_strings(gsp):
    for s in range(10):
        assert gsp.gsp_status_string(s) not in ("", "unknown status")
    assert gsp.gsp_status_string(99) == "unknown status"
    assert gsp.gsp_version() >= 100


def test_null_arguments_return_status(gsp):
    L = gsp.lib()
    assert L.gsp_plan_create(None, None) == gsp.GSP_ERR_INVALID_ARG
    assert L.gsp_plan_destroy(None) == gsp.GSP_ERR_INVALID_ARG
    assert L.gsp_plan_max_delay(None) == -1
    assert L.gsp_dedisperse(None, None, 0, 0, None, 0, None) == gsp.GSP_ERR_INVALID_ARG
    assert L.gsp_candidates(None, None, 0, None) == gsp.GSP_ERR_INVALID_ARG
    assert L.gsp_plan_tune(None, None, 0, 0, None, None, None) == gsp.GSP_ERR_INVALID_ARG
    assert L.gsp_plan_series(None, None, None, None) == gsp.GSP_ERR_INVALID_ARG
    assert L.gsp_plan_set_snippet_path(None, 0) == gsp.GSP_ERR_INVALID_ARG
    assert L.gsp_batch_tune_results(None, None, None, 0) == -1


def test_static_search_argument_checks_on_host(gsp):
    # argument checks of the no-allocation search return before any CUDA call
    L = gsp.lib()
    fake = 0x1000  # never dereferenced: every case below is rejected first
    args = dict(ndm=4, n_out=8192, stride=8192, t_off=0, bl=1024, wl=1024, thr=6.0)

    def call(**kw):
        a = dict(args)
        a.update(kw)
        return L.gsp_search_series_static(fake, a["ndm"], a["n_out"], a["stride"], a["t_off"],
                                          None, 0, a["bl"], a["wl"], a["thr"], 0.5, 2.5, fake,
                                          16, fake, None)
    assert call(thr=float("inf")) == gsp.GSP_ERR_INVALID_ARG
    assert call(thr=float("-inf")) == gsp.GSP_ERR_INVALID_ARG
    assert call(thr=float("nan")) == gsp.GSP_ERR_INVALID_ARG
    assert call(ndm=4097) == gsp.GSP_ERR_TOO_LARGE
    assert call(ndm=300, n_out=1024 * 1024, stride=1024 * 1024) == gsp.GSP_ERR_TOO_LARGE
    # a long series cut into one-sample windows: more windows than a grid dimension
    big = 1 << 40
    assert call(ndm=1, n_out=big, stride=big, bl=1 << 30, wl=1) == gsp.GSP_ERR_TOO_LARGE


def test_plan_without_gpu_fails_cleanly(gsp):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    desc, keep = gsp.make_desc(64, 1200.0, 1500.0, 1e-4, 4096, ndm=8)
    with pytest.raises(gsp.GspError) as e:
        gsp.gsp_plan_create(desc, keep)
    assert e.value.status == gsp.GSP_ERR_CUDA
