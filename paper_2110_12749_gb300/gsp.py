"""Thin ctypes binding of libgsp (include/gsp.h) with the same entry-point names.

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Device buffers are torch CUDA tensors (``data_ptr()``); streams
default to torch's current stream.  There is no fallback: if libgsp.so has not
been built, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgsp.so")

GSP_OK = 0
GSP_ERR_INVALID_ARG = 1
GSP_ERR_OOM = 2
GSP_ERR_CUDA = 3
GSP_ERR_TOO_SHORT = 4
GSP_ERR_CAPACITY = 5
GSP_ERR_TIMEOUT = 6
GSP_ERR_TIE = 7
GSP_ERR_ALIGN = 8
GSP_ERR_STATE = 9
GSP_ERR_TOO_LARGE = 10
GSP_ERR_BUSY = 11

GSP_FLAG_TIMING = 1
GSP_FLAG_SIMPLE_DD = 2
GSP_BATCH_PERSISTENT = 1
GSP_BATCH_GRAPH = 2
GSP_BATCH_AUTOTUNE = 4
GSP_BATCH_TIMING = 8

DEFAULT_WIDTHS = (1, 2, 3, 4, 6, 9, 14, 20, 30, 45, 70, 100, 150)


class GspError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = "%s: %s" % (where, gsp_status_string(status))
        if status == GSP_ERR_CUDA:
            msg += " [%s]" % gsp_last_error_string()
        super().__init__(msg)


class gsp_plan_desc(ctypes.Structure):
    _fields_ = [
        ("nchan", ctypes.c_int32),
        ("f_lo_mhz", ctypes.c_double),
        ("f_hi_mhz", ctypes.c_double),
        ("freq_descending", ctypes.c_int32),
        ("t_samp_s", ctypes.c_double),
        ("ndm", ctypes.c_int32),
        ("dms", ctypes.c_void_p),
        ("dm_lo", ctypes.c_double),
        ("dm_step", ctypes.c_double),
        ("delays", ctypes.c_void_p),
        ("nsamp_max", ctypes.c_int64),
        ("widths", ctypes.c_void_p),
        ("nwidths", ctypes.c_int32),
        ("block_len", ctypes.c_int32),
        ("window_len", ctypes.c_int32),
        ("threshold", ctypes.c_float),
        ("bad_lo", ctypes.c_float),
        ("bad_hi", ctypes.c_float),
        ("max_cands", ctypes.c_int64),
        ("flags", ctypes.c_int32),
    ]


CAND_DTYPE = np.dtype([("dm_idx", np.int32), ("width", np.int32), ("t", np.int64),
                       ("snr", np.float32), ("beam", np.int32)], align=True)
assert CAND_DTYPE.itemsize == 24

_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgsp.so is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "gsp_plan_desc_init": ([_vp], ctypes.c_int),
            "gsp_compute_delays": ([_vp, _vp, _vp], ctypes.c_int),
            "gsp_plan_create": ([_vp, _vp], ctypes.c_int),
            "gsp_plan_destroy": ([_vp], ctypes.c_int),
            "gsp_plan_max_delay": ([_vp], _i64),
            "gsp_plan_nout": ([_vp, _i64], _i64),
            "gsp_plan_delays": ([_vp, _vp], ctypes.c_int),
            "gsp_dedisperse": ([_vp, _vp, _i64, _i64, _vp, _i64, _vp], ctypes.c_int),
            "gsp_search": ([_vp, _vp, _i64, _i64, _i64, _vp, _i64, _vp], ctypes.c_int),
            "gsp_search_series": ([_vp, _vp, _i64, _i64, _i64, _vp], ctypes.c_int),
            "gsp_boxcar_snr": ([_vp, _vp, _i64, _i64, _vp, _vp], ctypes.c_int),
            "gsp_search_stats": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
            "gsp_candidates": ([_vp, _vp, _i64, _vp], ctypes.c_int),
            "gsp_search_host": ([_vp, _vp, _i64, _i64, _i64, _vp, _i64, _vp, _vp], ctypes.c_int),
            "gsp_plan_timing": ([_vp, _vp, _vp], ctypes.c_int),
            "gsp_search_series_static": ([_vp, ctypes.c_int32, _i64, _i64, _i64, _vp, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                          ctypes.c_float, ctypes.c_float, _vp, _i64, _vp, _vp],
                                         ctypes.c_int),
            "gsp_plan_launches": ([_vp], ctypes.c_int32),
            "gsp_dedisperse_variants": ([_vp, _vp], ctypes.c_int32),
            "gsp_plan_tune": ([_vp, _vp, _i64, _i64, _vp, _vp, _vp], ctypes.c_int),
            "gsp_plan_set_wait_limit": ([_vp, _i64, ctypes.c_int32], ctypes.c_int),
            "gsp_plan_set_snippet_path": ([_vp, ctypes.c_int32], ctypes.c_int),
            "gsp_plan_series": ([_vp, _vp, _vp, _vp], ctypes.c_int),
            "gsp_batch_tune_results": ([_vp, _vp, _vp, ctypes.c_int32], ctypes.c_int32),
            "gsp_stream_create": ([_vp, _vp, _i64, ctypes.c_int32], ctypes.c_int),
            "gsp_stream_destroy": ([_vp], ctypes.c_int),
            "gsp_stream_need": ([_vp], _i64),
            "gsp_stream_bytes": ([_vp, _i64], _i64),
            "gsp_stream_push": ([_vp, _vp, _i64, _i64, _vp], ctypes.c_int),
            "gsp_stream_results": ([_vp, _vp, _i64, _vp, _vp], ctypes.c_int),
            "gsp_chunkpool_create": ([_vp, ctypes.c_int32, _i64, _i64, ctypes.c_int32], ctypes.c_int),
            "gsp_chunkpool_destroy": ([_vp], ctypes.c_int),
            "gsp_chunkpool_bytes": ([ctypes.c_int32, _i64, _i64, ctypes.c_int32], _i64),
            "gsp_chunkpool_free": ([_vp], ctypes.c_int32),
            "gsp_stream_create_pooled": ([_vp, _vp, _vp, ctypes.c_int32], ctypes.c_int),
            "gsp_stream_pooled_bytes": ([_vp, _i64], _i64),
            "gsp_batch_create": ([_vp, _vp, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
            "gsp_batch_destroy": ([_vp], ctypes.c_int),
            "gsp_batch_search": ([_vp, _vp, _vp], ctypes.c_int),
            "gsp_batch_candidates": ([_vp, _vp, _i64, _vp], ctypes.c_int),
            "gsp_batch_info": ([_vp, _vp, _vp, _vp], ctypes.c_int),
            "gsp_batch_timing": ([_vp, _vp, _vp], ctypes.c_int),
            "gsp_ingest_transpose": ([_vp, _i64, ctypes.c_int32, _i64, _vp, _i64, _vp], ctypes.c_int),
            "gsp_downsample": ([_vp, ctypes.c_int32, _i64, _i64, ctypes.c_int32, _vp, _i64, _vp],
                               ctypes.c_int),
            "gsp_ddplan_create": ([_vp, _vp, _vp, ctypes.c_int32], ctypes.c_int),
            "gsp_ddplan_destroy": ([_vp], ctypes.c_int),
            "gsp_ddplan_search": ([_vp, _vp, _i64, _i64, _i64, _vp], ctypes.c_int),
            "gsp_ddplan_candidates": ([_vp, _vp, _i64, _vp], ctypes.c_int),
            "gsp_subband_create": ([_vp, _vp, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
            "gsp_subband_destroy": ([_vp], ctypes.c_int),
            "gsp_subband_nout": ([_vp, _i64], _i64),
            "gsp_subband_delays": ([_vp, _vp, _vp, _vp], ctypes.c_int),
            "gsp_subband_dedisperse": ([_vp, _vp, _i64, _i64, _vp, _i64, _vp], ctypes.c_int),
            "gsp_subband_finish": ([_vp, _vp], ctypes.c_int),
            "gsp_subband_launches": ([_vp], ctypes.c_int32),
            "gsp_gemm_bf16": ([_vp, _i64, _vp, _i64, _vp, _i64, ctypes.c_int32, ctypes.c_int32,
                               ctypes.c_int32, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp],
                              ctypes.c_int),
            "gsp_ranker_num_params": ([], _i64),
            "gsp_ranker_create": ([_vp, ctypes.c_int32, ctypes.c_uint64], ctypes.c_int),
            "gsp_ranker_destroy": ([_vp], ctypes.c_int),
            "gsp_ranker_set_params": ([_vp, _vp], ctypes.c_int),
            "gsp_ranker_get_params": ([_vp, _vp, _vp], ctypes.c_int),
            "gsp_ranker_snippets": ([_vp, _vp, _i64, _vp, ctypes.c_int32, _vp, _vp], ctypes.c_int),
            "gsp_ranker_forward": ([_vp, _vp, ctypes.c_int32, _vp, _vp], ctypes.c_int),
            "gsp_ranker_train_step": ([_vp, _vp, _vp, ctypes.c_int32, ctypes.c_float, _vp, _vp],
                                      ctypes.c_int),
            "gsp_ranker_finish": ([_vp, _vp], ctypes.c_int),
            "gsp_ranker_launches": ([_vp], ctypes.c_int32),
            "gsp_ranker_tensor": ([_vp, ctypes.c_char_p, _vp, _i64, _vp], ctypes.c_int),
            "gsp_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "gsp_last_error_string": ([], ctypes.c_char_p),
            "gsp_version": ([], ctypes.c_int32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _np_ptr(a):
    return a.ctypes.data_as(_vp) if a is not None else None


def _stream(stream):
    if stream is None:
        import torch
        return _vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _vp(stream)
    return _vp(stream.cuda_stream)


def _check(st, where):
    if st != GSP_OK:
        raise GspError(st, where)


def gsp_status_string(st):
    return lib().gsp_status_string(int(st)).decode()


def gsp_last_error_string():
    return lib().gsp_last_error_string().decode()


def gsp_version():
    return int(lib().gsp_version())


class Plan:
    """Owns a gsp_plan_t and the host arrays its descriptor points to."""

    def __init__(self, handle, desc, keep):
        self.handle = handle
        self.desc = desc
        self._keep = keep

    @property
    def ndm(self):
        return int(self.desc.ndm)

    @property
    def nchan(self):
        return int(self.desc.nchan)

    @property
    def widths(self):
        return self._keep.get("widths_list", DEFAULT_WIDTHS)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            try:
                _lib.gsp_plan_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def gsp_plan_desc_init():
    d = gsp_plan_desc()
    _check(lib().gsp_plan_desc_init(ctypes.byref(d)), "gsp_plan_desc_init")
    return d


def make_desc(nchan, f_lo, f_hi, t_samp, nsamp_max, dms=None, dm_lo=0.0, dm_step=1.0,
              ndm=None, delays=None, freq_descending=False, widths=None, block_len=None,
              window_len=None, threshold=None, bad_lo=None, bad_hi=None, max_cands=None,
              flags=0):
    """Descriptor plus the arrays it points to (keep both alive together)."""
    d = gsp_plan_desc_init()
    keep = {}
    d.nchan = nchan
    d.f_lo_mhz, d.f_hi_mhz, d.t_samp_s = f_lo, f_hi, t_samp
    d.freq_descending = int(bool(freq_descending))
    d.nsamp_max = nsamp_max
    if dms is not None:
        arr = np.ascontiguousarray(np.asarray(dms, dtype=np.float64).reshape(-1))
        keep["dms"] = arr
        d.dms = arr.ctypes.data
        d.ndm = arr.size
    elif ndm is not None:
        d.ndm = ndm
        d.dm_lo, d.dm_step = dm_lo, dm_step
    if delays is not None:
        arr = np.ascontiguousarray(np.asarray(delays, dtype=np.int32))
        keep["delays"] = arr
        d.delays = arr.ctypes.data
        d.ndm = arr.shape[0]
    if widths is not None:
        arr = np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
        keep["widths"] = arr
        keep["widths_list"] = tuple(int(w) for w in widths)
        d.widths = arr.ctypes.data
        d.nwidths = arr.size
    if block_len is not None:
        d.block_len = block_len
    if window_len is not None:
        d.window_len = window_len
    if threshold is not None:
        d.threshold = threshold
    if bad_lo is not None:
        d.bad_lo = bad_lo
    if bad_hi is not None:
        d.bad_hi = bad_hi
    if max_cands is not None:
        d.max_cands = max_cands
    d.flags = flags
    return d, keep


def gsp_compute_delays(desc):
    out = np.empty((desc.ndm, desc.nchan), dtype=np.int32)
    m = ctypes.c_double(0.0)
    _check(lib().gsp_compute_delays(ctypes.byref(desc), _np_ptr(out), ctypes.byref(m)),
           "gsp_compute_delays")
    return out, m.value


def gsp_plan_create(desc, keep=None):
    h = _vp()
    _check(lib().gsp_plan_create(ctypes.byref(h), ctypes.byref(desc)), "gsp_plan_create")
    return Plan(h, desc, keep or {})


def gsp_plan_destroy(plan):
    if plan.handle:
        st = lib().gsp_plan_destroy(plan.handle)
        plan.handle = None
        _check(st, "gsp_plan_destroy")


def gsp_plan_max_delay(plan):
    return int(lib().gsp_plan_max_delay(plan.handle))


def gsp_plan_nout(plan, n_in):
    return int(lib().gsp_plan_nout(plan.handle, n_in))


def gsp_plan_delays(plan):
    out = np.empty((plan.ndm, plan.nchan), dtype=np.int32)
    _check(lib().gsp_plan_delays(plan.handle, _np_ptr(out)), "gsp_plan_delays")
    return out


def gsp_dedisperse(plan, x, n_in, out, stream=None):
    """x: torch uint8 CUDA [nchan][stride]; out: torch int32 CUDA [ndm][>= n_out]."""
    st = lib().gsp_dedisperse(plan.handle, _vp(x.data_ptr()), n_in, x.stride(0),
                              _vp(out.data_ptr()), out.stride(0), _stream(stream))
    _check(st, "gsp_dedisperse")


def gsp_search(plan, x, n_in, t_offset=0, out=None, stream=None):
    st = lib().gsp_search(plan.handle, _vp(x.data_ptr()), n_in, x.stride(0), t_offset,
                          _vp(out.data_ptr()) if out is not None else None,
                          out.stride(0) if out is not None else 0, _stream(stream))
    _check(st, "gsp_search")


def gsp_search_series(plan, D, n_out, t_offset=0, stream=None):
    st = lib().gsp_search_series(plan.handle, _vp(D.data_ptr()), n_out, D.stride(0), t_offset,
                                 _stream(stream))
    _check(st, "gsp_search_series")


def gsp_boxcar_snr(plan, D, n_out, snr_out, stream=None):
    st = lib().gsp_boxcar_snr(plan.handle, _vp(D.data_ptr()), n_out, D.stride(0),
                              _vp(snr_out.data_ptr()), _stream(stream))
    _check(st, "gsp_boxcar_snr")


def gsp_search_stats(plan, n_out):
    nb = n_out // plan.desc.block_len
    sig = np.zeros((plan.ndm, max(nb, 1)), np.float64)
    bad = np.zeros((plan.ndm, max(nb, 1)), np.uint8)
    sref = np.zeros(plan.ndm, np.float64)
    nbo = ctypes.c_int64(0)
    _check(lib().gsp_search_stats(plan.handle, _np_ptr(sig), _np_ptr(bad), _np_ptr(sref),
                                  ctypes.byref(nbo)), "gsp_search_stats")
    nb = nbo.value
    return {"sigma_b": sig[:, :nb], "bad": bad[:, :nb].astype(bool), "sigma_ref": sref}


def gsp_candidates(plan, cap=None):
    """Returns (candidates sorted by (dm_idx, t, width), true count, status)."""
    if cap is None:
        cap = int(plan.desc.max_cands)
    out = np.empty(max(cap, 1), dtype=CAND_DTYPE)   # only the first n records are read
    n = ctypes.c_int64(0)
    st = lib().gsp_candidates(plan.handle, _np_ptr(out), cap, ctypes.byref(n))
    if st not in (GSP_OK, GSP_ERR_CAPACITY):
        _check(st, "gsp_candidates")
    # a view: the pages of `out` past the first n records are never touched
    return out[:min(n.value, cap)], n.value, st


def gsp_search_host(plan, x_host, n_in, t_offset=0, cap=None, stream=None):
    """x_host: numpy uint8 [nchan][stride] or a (pinned) CPU torch tensor."""
    if cap is None:
        cap = int(plan.desc.max_cands)
    out = np.empty(max(cap, 1), dtype=CAND_DTYPE)   # only the first n records are read
    n = ctypes.c_int64(0)
    if isinstance(x_host, np.ndarray):
        ptr, stride = _np_ptr(x_host), x_host.strides[0]
    else:
        ptr, stride = _vp(x_host.data_ptr()), x_host.stride(0)
    st = lib().gsp_search_host(plan.handle, ptr, n_in, stride, t_offset, _np_ptr(out), cap,
                               ctypes.byref(n), _stream(stream))
    if st not in (GSP_OK, GSP_ERR_CAPACITY):
        _check(st, "gsp_search_host")
    return out[:min(n.value, cap)], n.value, st


def gsp_plan_timing(plan):
    a, b = ctypes.c_float(0), ctypes.c_float(0)
    _check(lib().gsp_plan_timing(plan.handle, ctypes.byref(a), ctypes.byref(b)),
           "gsp_plan_timing")
    return a.value, b.value


SNIPPET_AUTO, SNIPPET_DIRECT, SNIPPET_PREFIX = 0, 1, 2


def gsp_plan_set_snippet_path(plan, path):
    """Snippet path of gsp_ranker_snippets: SNIPPET_AUTO, SNIPPET_DIRECT or
    SNIPPET_PREFIX."""
    _check(lib().gsp_plan_set_snippet_path(plan.handle, int(path)), "gsp_plan_set_snippet_path")


def gsp_plan_set_wait_limit(plan, cycles, starve=0):
    _check(lib().gsp_plan_set_wait_limit(plan.handle, int(cycles), int(starve)),
           "gsp_plan_set_wait_limit")


def gsp_plan_launches(plan):
    return int(lib().gsp_plan_launches(plan.handle))


def gsp_dedisperse_variants(plan=None):
    """(number of tile variants, variant the plan uses or -1 for the simple
    kernel; None without a plan)."""
    used = ctypes.c_int32(-2)
    n = int(lib().gsp_dedisperse_variants(plan.handle if plan is not None else None,
                                          ctypes.byref(used)))
    return n, (int(used.value) if plan is not None else None)


def gsp_plan_tune(plan, x, n_in, stream=None):
    """Autotune the plan's tile variant on x (torch uint8 CUDA [nchan][stride]);
    returns (variant, median ms of the tuning runs)."""
    v, ms = ctypes.c_int32(-1), ctypes.c_float(0)
    _check(lib().gsp_plan_tune(plan.handle, x.data_ptr(), n_in, x.stride(0), _stream(stream),
                               ctypes.byref(v), ctypes.byref(ms)), "gsp_plan_tune")
    return v.value, ms.value


def gsp_plan_series(plan):
    """(device address, row stride, n_out) of the series of the plan's last search."""
    p, st, n = _vp(), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().gsp_plan_series(plan.handle, ctypes.byref(p), ctypes.byref(st), ctypes.byref(n)),
           "gsp_plan_series")
    return p.value, st.value, n.value


class _DeviceArray:
    """A view of device memory for torch.as_tensor (CUDA array interface)."""

    def __init__(self, addr, shape, strides, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "strides": tuple(strides),
                                         "typestr": typestr, "data": (int(addr), False),
                                         "version": 3}


def gsp_plan_series_tensor(plan):
    """torch int32 CUDA view [ndm][n_out] (row stride as stored) of the series of
    the plan's last search; valid until the plan searches again or is destroyed."""
    import torch
    addr, stride, n_out = gsp_plan_series(plan)
    ndm = plan.desc.ndm if hasattr(plan, "desc") else None
    if ndm is None:
        raise RuntimeError("plan without its descriptor")
    return torch.as_tensor(_DeviceArray(addr, (ndm, n_out), (4 * stride, 4), "<i4"),
                           device="cuda")


def gsp_search_series_static(D, n_out, d_cands, d_ncand, t_offset=0, widths=None,
                             block_len=1024, window_len=1024, threshold=6.0, bad_lo=0.5,
                             bad_hi=2.5, stream=None):
    """No-allocation search of D (torch int32 CUDA [ndm][stride]); d_cands is a
    CUDA uint8 tensor of max_cands * 24 bytes, d_ncand a CUDA int64 tensor of
    one element.  Asynchronous; read the outputs after synchronising."""
    w = None if widths is None else np.ascontiguousarray(np.asarray(widths, dtype=np.int32))
    max_cands = d_cands.numel() * d_cands.element_size() // CAND_DTYPE.itemsize
    st = lib().gsp_search_series_static(
        _vp(D.data_ptr()), D.shape[0], n_out, D.stride(0), t_offset, _np_ptr(w),
        0 if w is None else w.size, block_len, window_len, threshold, bad_lo, bad_hi,
        _vp(d_cands.data_ptr()), max_cands, _vp(d_ncand.data_ptr()), _stream(stream))
    _check(st, "gsp_search_series_static")


class Stream:
    """Owns a gsp_stream_t (and keeps its plan alive)."""

    def __init__(self, handle, plan):
        self.handle = handle
        self.plan = plan

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            try:
                _lib.gsp_stream_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def gsp_stream_create(plan, chunk_out, beam=0):
    h = _vp()
    _check(lib().gsp_stream_create(ctypes.byref(h), plan.handle, chunk_out, beam),
           "gsp_stream_create")
    return Stream(h, plan)


def gsp_stream_destroy(s):
    if s.handle:
        st = lib().gsp_stream_destroy(s.handle)
        s.handle = None
        _check(st, "gsp_stream_destroy")


def gsp_stream_bytes(plan, chunk_out):
    return int(lib().gsp_stream_bytes(plan.handle, chunk_out))


def gsp_stream_need(s):
    return int(lib().gsp_stream_need(s.handle))


def gsp_stream_push(s, x_host, n, stream=None, busy_ok=False):
    """x_host: numpy uint8 [nchan][stride] or a (pinned) CPU torch tensor.  With
    busy_ok, returns False instead of raising when a pooled stream finds no free
    pool buffer (the chunk was not admitted); True when it was pushed."""
    if isinstance(x_host, np.ndarray):
        ptr, stride = _np_ptr(x_host), x_host.strides[0]
    else:
        ptr, stride = _vp(x_host.data_ptr()), x_host.stride(0)
    st = lib().gsp_stream_push(s.handle, ptr, n, stride, _stream(stream))
    if busy_ok and st == GSP_ERR_BUSY:
        return False
    _check(st, "gsp_stream_push")
    return True


class ChunkPool:
    """Owns a gsp_chunkpool_t."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            try:
                _lib.gsp_chunkpool_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def gsp_chunkpool_create(nchan, chunk_out, max_tail, nbuf):
    h = _vp()
    _check(lib().gsp_chunkpool_create(ctypes.byref(h), nchan, chunk_out, max_tail, nbuf),
           "gsp_chunkpool_create")
    return ChunkPool(h)


def gsp_chunkpool_destroy(p):
    if p.handle:
        st = lib().gsp_chunkpool_destroy(p.handle)
        p.handle = None
        _check(st, "gsp_chunkpool_destroy")


def gsp_chunkpool_bytes(nchan, chunk_out, max_tail, nbuf):
    return int(lib().gsp_chunkpool_bytes(nchan, chunk_out, max_tail, nbuf))


def gsp_chunkpool_free(p):
    return int(lib().gsp_chunkpool_free(p.handle))


def gsp_stream_create_pooled(plan, pool, beam=0):
    h = _vp()
    _check(lib().gsp_stream_create_pooled(ctypes.byref(h), plan.handle, pool.handle, beam),
           "gsp_stream_create_pooled")
    st = Stream(h, plan)
    st.pool = pool
    return st


def gsp_stream_pooled_bytes(plan, chunk_out):
    return int(lib().gsp_stream_pooled_bytes(plan.handle, chunk_out))


def gsp_stream_results(s, cap=None):
    """(candidates with absolute t and the beam label, true count, status, t_abs0)."""
    if cap is None:
        cap = int(s.plan.desc.max_cands)
    out = np.empty(max(cap, 1), dtype=CAND_DTYPE)   # only the first n records are read
    n, t0 = ctypes.c_int64(0), ctypes.c_int64(0)
    st = lib().gsp_stream_results(s.handle, _np_ptr(out), cap, ctypes.byref(n), ctypes.byref(t0))
    if st not in (GSP_OK, GSP_ERR_CAPACITY):
        _check(st, "gsp_stream_results")
    return out[:min(n.value, cap)].copy(), n.value, st, t0.value


class gsp_beam_input(ctypes.Structure):
    _fields_ = [("d_x", ctypes.c_void_p), ("n_in", ctypes.c_int64),
                ("x_stride", ctypes.c_int64), ("t_offset", ctypes.c_int64)]


class Batch:
    """Owns a gsp_batch_t and keeps its plans alive."""

    def __init__(self, handle, plans):
        self.handle = handle
        self.plans = plans

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            try:
                _lib.gsp_batch_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def gsp_batch_create(plans, flags=0):
    arr = (ctypes.c_void_p * len(plans))(*[p.handle.value for p in plans])
    h = _vp()
    _check(lib().gsp_batch_create(ctypes.byref(h), arr, len(plans), flags), "gsp_batch_create")
    return Batch(h, list(plans))


def gsp_batch_destroy(b):
    if b.handle:
        st = lib().gsp_batch_destroy(b.handle)
        b.handle = None
        _check(st, "gsp_batch_destroy")


def gsp_batch_search(b, xs, n_ins, t_offsets=None, stream=None):
    """xs: torch uint8 CUDA tensors [nchan][stride], one per beam."""
    n = len(xs)
    arr = (gsp_beam_input * n)()
    for i, x in enumerate(xs):
        arr[i].d_x = x.data_ptr()
        arr[i].n_in = n_ins[i]
        arr[i].x_stride = x.stride(0)
        arr[i].t_offset = 0 if t_offsets is None else t_offsets[i]
    b._inputs = arr
    _check(lib().gsp_batch_search(b.handle, arr, _stream(stream)), "gsp_batch_search")


def gsp_batch_candidates(b, cap=1 << 22):
    out = np.empty(max(cap, 1), dtype=CAND_DTYPE)   # only the first n records are read
    n = ctypes.c_int64(0)
    st = lib().gsp_batch_candidates(b.handle, _np_ptr(out), cap, ctypes.byref(n))
    if st not in (GSP_OK, GSP_ERR_CAPACITY):
        _check(st, "gsp_batch_candidates")
    return out[:min(n.value, cap)].copy(), n.value, st


def gsp_batch_info(b):
    v, ms, nl = ctypes.c_int32(0), ctypes.c_float(0), ctypes.c_int32(0)
    _check(lib().gsp_batch_info(b.handle, ctypes.byref(v), ctypes.byref(ms), ctypes.byref(nl)),
           "gsp_batch_info")
    return v.value, ms.value, nl.value


def gsp_batch_tune_results(b):
    """[(variant, median ms)] of every tile variant the autotuner timed."""
    n = int(lib().gsp_batch_tune_results(b.handle, None, None, 0))
    if n <= 0:
        return []
    v = np.zeros(n, np.int32)
    ms = np.zeros(n, np.float32)
    lib().gsp_batch_tune_results(b.handle, _np_ptr(v), _np_ptr(ms), n)
    return [(int(a), float(m)) for a, m in zip(v, ms)]


def gsp_batch_timing(b):
    a, t = ctypes.c_float(0), ctypes.c_float(0)
    _check(lib().gsp_batch_timing(b.handle, ctypes.byref(a), ctypes.byref(t)), "gsp_batch_timing")
    return a.value, t.value



# ---------------------------------------------------------------------------
# DDplan ranges and sub-band dedispersion

class gsp_ddplan_range(ctypes.Structure):
    _fields_ = [("dm_lo", ctypes.c_double), ("dm_step", ctypes.c_double),
                ("ndm", ctypes.c_int32), ("downsamp", ctypes.c_int32)]


def gsp_ingest_transpose(x_tc, n_samp, nchan, out, stream=None):
    """x_tc: torch uint8 CUDA [n_samp][>= nchan] (time-major); out: torch uint8 CUDA
    [nchan][>= n_samp] (channel-major)."""
    _check(lib().gsp_ingest_transpose(_vp(x_tc.data_ptr()), n_samp, nchan, x_tc.stride(0),
                                      _vp(out.data_ptr()), out.stride(0), _stream(stream)),
           "gsp_ingest_transpose")


def gsp_downsample(x, nchan, n_in, ds, out, stream=None):
    """x: torch uint8 CUDA [nchan][stride]; out: torch uint8 CUDA [nchan][>= n_in // ds]."""
    _check(lib().gsp_downsample(_vp(x.data_ptr()), nchan, n_in, x.stride(0), ds,
                                _vp(out.data_ptr()), out.stride(0), _stream(stream)),
           "gsp_downsample")


class DDPlan:
    """Owns a gsp_ddplan_t."""

    def __init__(self, handle, ranges):
        self.handle = handle
        self.ranges = ranges

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            try:
                _lib.gsp_ddplan_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def gsp_ddplan_create(base_desc, ranges):
    """ranges: iterable of (dm_lo, dm_step, ndm, downsamp)."""
    ranges = list(ranges)
    arr = (gsp_ddplan_range * len(ranges))()
    for i, (lo, step, n, ds) in enumerate(ranges):
        arr[i].dm_lo, arr[i].dm_step, arr[i].ndm, arr[i].downsamp = lo, step, n, ds
    h = _vp()
    _check(lib().gsp_ddplan_create(ctypes.byref(h), ctypes.byref(base_desc), arr, len(ranges)),
           "gsp_ddplan_create")
    return DDPlan(h, ranges)


def gsp_ddplan_destroy(d):
    if d.handle:
        st = lib().gsp_ddplan_destroy(d.handle)
        d.handle = None
        _check(st, "gsp_ddplan_destroy")


def gsp_ddplan_search(d, x, n_in, t_offset=0, stream=None):
    _check(lib().gsp_ddplan_search(d.handle, _vp(x.data_ptr()), n_in, x.stride(0), t_offset,
                                   _stream(stream)), "gsp_ddplan_search")


def gsp_ddplan_candidates(d, cap=1 << 22):
    out = np.empty(max(cap, 1), dtype=CAND_DTYPE)   # only the first n records are read
    n = ctypes.c_int64(0)
    st = lib().gsp_ddplan_candidates(d.handle, _np_ptr(out), cap, ctypes.byref(n))
    if st not in (GSP_OK, GSP_ERR_CAPACITY):
        _check(st, "gsp_ddplan_candidates")
    return out[:min(n.value, cap)].copy(), n.value, st


class Subband:
    """Owns a gsp_subband_t."""

    def __init__(self, handle, ndm, nchan, nsub, group):
        self.handle = handle
        self.ndm, self.nchan, self.nsub, self.group = ndm, nchan, nsub, group
        self.nsdm = (ndm + group - 1) // group

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            try:
                _lib.gsp_subband_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def gsp_subband_create(desc, nsub, group):
    h = _vp()
    _check(lib().gsp_subband_create(ctypes.byref(h), ctypes.byref(desc), nsub, group),
           "gsp_subband_create")
    return Subband(h, int(desc.ndm), int(desc.nchan), nsub, group)


def gsp_subband_destroy(b):
    if b.handle:
        st = lib().gsp_subband_destroy(b.handle)
        b.handle = None
        _check(st, "gsp_subband_destroy")


def gsp_subband_nout(b, n_in):
    return int(lib().gsp_subband_nout(b.handle, n_in))


def gsp_subband_delays(b):
    d1 = np.zeros((b.nsdm, b.nchan), np.int32)
    d2 = np.zeros((b.ndm, b.nsub), np.int32)
    si = np.zeros(b.nsdm, np.int32)
    _check(lib().gsp_subband_delays(b.handle, _np_ptr(d1), _np_ptr(d2), _np_ptr(si)),
           "gsp_subband_delays")
    return d1, d2, si


def gsp_subband_dedisperse(b, x, n_in, out, stream=None):
    """x: torch uint8 CUDA [nchan][stride]; out: torch int32 CUDA [ndm][>= n_out]."""
    _check(lib().gsp_subband_dedisperse(b.handle, _vp(x.data_ptr()), n_in, x.stride(0),
                                        _vp(out.data_ptr()), out.stride(0), _stream(stream)),
           "gsp_subband_dedisperse")


def gsp_subband_finish(b, stream=None):
    _check(lib().gsp_subband_finish(b.handle, _stream(stream)), "gsp_subband_finish")


def gsp_subband_launches(b):
    return int(lib().gsp_subband_launches(b.handle))


def gsp_gemm_bf16(A, B, C, M, N, K, bias=None, relu=False, splitk=1, err=None, stream=None):
    """A: torch bf16 CUDA [M][lda], B: torch bf16 CUDA [N][ldb], C: torch float CUDA [M][ldc]."""
    _check(lib().gsp_gemm_bf16(_vp(A.data_ptr()), A.stride(0), _vp(B.data_ptr()), B.stride(0),
                               _vp(C.data_ptr()), C.stride(0), M, N, K,
                               _vp(bias.data_ptr()) if bias is not None else None, int(relu),
                               splitk, _vp(err.data_ptr()) if err is not None else None,
                               _stream(stream)), "gsp_gemm_bf16")



# ---------------------------------------------------------------------------
# Candidate ranker

class Ranker:
    """Owns a gsp_ranker_t."""

    def __init__(self, handle, max_batch):
        self.handle = handle
        self.max_batch = max_batch

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            try:
                _lib.gsp_ranker_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def gsp_ranker_num_params():
    return int(lib().gsp_ranker_num_params())


def gsp_ranker_create(max_batch, seed=0):
    h = _vp()
    _check(lib().gsp_ranker_create(ctypes.byref(h), max_batch, seed), "gsp_ranker_create")
    return Ranker(h, max_batch)


def gsp_ranker_destroy(r):
    if r.handle:
        st = lib().gsp_ranker_destroy(r.handle)
        r.handle = None
        _check(st, "gsp_ranker_destroy")


def gsp_ranker_set_params(r, params):
    p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
    assert p.size == gsp_ranker_num_params()
    _check(lib().gsp_ranker_set_params(r.handle, _np_ptr(p)), "gsp_ranker_set_params")


def gsp_ranker_get_params(r):
    """(parameters, gradients of the last training step), float32 numpy."""
    n = gsp_ranker_num_params()
    p = np.zeros(n, np.float32)
    g = np.zeros(n, np.float32)
    _check(lib().gsp_ranker_get_params(r.handle, _np_ptr(p), _np_ptr(g)), "gsp_ranker_get_params")
    return p, g


def gsp_ranker_snippets(plan, D, cands, out, stream=None):
    """D: torch int32 CUDA [ndm][stride]; cands: torch uint8 CUDA holding n
    records of CAND_DTYPE; out: torch float CUDA [n][64][64]."""
    n = cands.numel() // CAND_DTYPE.itemsize
    _check(lib().gsp_ranker_snippets(plan.handle, _vp(D.data_ptr()), D.stride(0),
                                     _vp(cands.data_ptr()), n, _vp(out.data_ptr()),
                                     _stream(stream)), "gsp_ranker_snippets")


def gsp_ranker_forward(r, x, n, logits, stream=None):
    _check(lib().gsp_ranker_forward(r.handle, _vp(x.data_ptr()), n, _vp(logits.data_ptr()),
                                    _stream(stream)), "gsp_ranker_forward")


def gsp_ranker_train_step(r, x, labels, n, lr, loss=None, stream=None):
    _check(lib().gsp_ranker_train_step(r.handle, _vp(x.data_ptr()), _vp(labels.data_ptr()), n,
                                       float(lr), _vp(loss.data_ptr()) if loss is not None else None,
                                       _stream(stream)), "gsp_ranker_train_step")


def gsp_ranker_finish(r, stream=None):
    _check(lib().gsp_ranker_finish(r.handle, _stream(stream)), "gsp_ranker_finish")


def gsp_ranker_tensor(r, name):
    """Host copy of an intermediate tensor of the last pass: numpy float64 for
    bf16 and float tensors (bf16 widened exactly), uint8 for the argmaxes; flat."""
    nb = ctypes.c_int64(0)
    st = lib().gsp_ranker_tensor(r.handle, name.encode(), None, 0, ctypes.byref(nb))
    if st != GSP_ERR_CAPACITY:
        _check(st, "gsp_ranker_tensor")
    raw = np.empty(nb.value, np.uint8)
    _check(lib().gsp_ranker_tensor(r.handle, name.encode(), _np_ptr(raw), nb.value,
                                   ctypes.byref(nb)), "gsp_ranker_tensor")
    if name.startswith("idx"):
        return raw
    if name in ("a4", "g4") or name.startswith("gz") or (name[0] == "a" and name[1:].isdigit()):
        u = raw.view(np.uint16).astype(np.uint32) << 16
        return u.view(np.float32).astype(np.float64)
    return raw.view(np.float32).astype(np.float64)


def gsp_ranker_launches(r):
    return int(lib().gsp_ranker_launches(r.handle))
