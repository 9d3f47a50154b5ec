"""GB300 (sm_103a) engine for per-event tree-level QCD matrix elements of g g -> t tbar + n gluons.

Thin Python binding over the C ABI of include/mg.h (libmg.so, built by build.py): argument
marshalling only -- every step of the random numbers -> momenta -> matrix element path (arXiv
2210.11122, Sec. 1, Fig. 1 and Sec. 2) runs in the library's CUDA kernels.  Device buffers are
torch CUDA tensors (or raw device pointers as ints); streams are torch.cuda.Stream objects, raw
cudaStream_t ints, or None for torch's current stream.  There is no CPU fallback: if libmg.so is
missing every call raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

MG_GG_TT, MG_GG_TTG, MG_GG_TTGG, MG_GG_TTGGG = 0, 1, 2, 3
PROCESSES = {"ggtt": 0, "ggttg": 1, "ggttgg": 2, "ggttggg": 3}
MG_FP64, MG_FP32_AMP, MG_FP64_TCCOLOR, MG_MIXED = 0, 1, 2, 3
LAUNCH_UNROLLED, LAUNCH_DF_REDO, LAUNCH_FUSED, LAUNCH_WARP, LAUNCH_TC_APART, LAUNCH_SHARED = 1, 2, 4, 8, 16, 32
LAUNCH_TC_SYNC = 64
SERVE_MASK_SEED = 0x4D47   # mg.h MG_SERVE_MASK_SEED
GRAPH_PERSISTENT = 1       # mg.h MG_GRAPH_PERSISTENT
PAGE = 32

STATUS = {0: "MG_OK", 1: "MG_EINVAL", 2: "MG_ENOMEM", 3: "MG_ECUDA", 4: "MG_ENOCONV", 5: "MG_EAGAIN",
          6: "MG_ETIMEOUT", 7: "MG_EBUSY", 8: "MG_ENOTSUP", 9: "MG_ECANCELED"}


class MGError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s: %s (%s)" % (what, STATUS.get(status, status), _strerror(status)))


class Params(ctypes.Structure):
    _fields_ = [("mt", ctypes.c_double), ("wt", ctypes.c_double), ("alphas", ctypes.c_double),
                ("hel_warmup", ctypes.c_int), ("hel_tau", ctypes.c_double)]


class Job(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("e0", ctypes.c_int64), ("nevt", ctypes.c_int64),
                ("sqrts", ctypes.c_double), ("mom_dev", ctypes.c_void_p), ("me_dev", ctypes.c_void_p),
                ("precision", ctypes.c_int)]


class BatchJob(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("mom_dev", ctypes.c_void_p), ("nevt", ctypes.c_int64), ("me_dev", ctypes.c_void_p)]


class ServeCfg(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("max_nevt", ctypes.c_int64), ("hbm_cap_bytes", ctypes.c_int64),
                ("precision", ctypes.c_int), ("sqrts", ctypes.c_double), ("params", Params)]


_lib = None


def library_path():
    return _build.LIB


def lib():
    """Load libmg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libmg.so is not built (run paper_2210_11122_gb300.build.build(); needs nvcc)")
    L = ctypes.CDLL(_build.LIB)
    vp, i64, u64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
    P = ctypes.POINTER
    L.mg_strerror.argtypes = [i32]
    L.mg_strerror.restype = ctypes.c_char_p
    L.mg_default_params.argtypes = [P(Params)]
    L.mg_default_params.restype = None
    L.mg_process_info.argtypes = [i32, P(i32), P(i32), P(i32), P(i32)]
    L.mg_mom_count.argtypes = [i32, i64]
    L.mg_mom_count.restype = i64
    L.mg_colour_matrix.argtypes = [i32, P(ctypes.c_int64), P(ctypes.c_int64)]
    L.mg_create.argtypes = [i32, P(Params), P(vp)]
    L.mg_destroy.argtypes = [vp]
    L.mg_destroy.restype = None
    L.mg_philox.argtypes = [u64, i64, i32, vp, vp]
    L.mg_rambo.argtypes = [vp, u64, i64, dbl, vp, vp, vp]
    L.mg_rambo_range.argtypes = [vp, u64, i64, i64, dbl, vp, vp, vp]
    L.mg_measure_fma_peak.argtypes = [i32, i32, P(dbl)]
    L.mg_measure_mma_peak.argtypes = [i32, P(dbl)]
    L.mg_kernel_launches.argtypes = []
    L.mg_diag_fail_alloc.argtypes = [ctypes.c_int64]
    L.mg_diag_fail_alloc.restype = i32
    L.mg_diag_live_allocs.argtypes = []
    L.mg_diag_live_allocs.restype = ctypes.c_int64
    L.mg_diag_tc_stall.argtypes = [vp, i32]
    L.mg_set_fp32_tau.argtypes = [vp, dbl]
    L.mg_diag_tc_stall.restype = i32
    L.mg_kernel_launches.restype = i64
    L.mg_hel_filter.argtypes = [vp, vp, i64, vp]
    L.mg_sigmakin.argtypes = [vp, vp, i64, i32, vp, vp]
    L.mg_sigmakin_host.argtypes = [vp, vp, i64, i32, vp, vp]
    L.mg_sigmakin_noalloc.argtypes = [vp, vp, i64, vp, vp]
    L.mg_sigmakin_lhe.argtypes = [vp, vp, i64, vp, vp, i32, vp, vp, vp, vp, vp]
    L.mg_alphas_running.argtypes = [vp, vp, i64, vp, vp, vp]
    L.mg_colour_flow.argtypes = [i32, i32, P(i32)]
    L.mg_sde_weights.argtypes = [vp, vp, i64, vp, vp]
    L.mg_sde_channels.argtypes = [i32, P(i32)]
    L.mg_sde_channel_key.argtypes = [i32, i32, ctypes.c_char_p, i32]
    L.mg_hel_mask.argtypes = [vp, P(ctypes.c_uint32), P(i32)]
    L.mg_check.argtypes = [vp, vp, P(ctypes.c_int64)]
    L.mg_flops_per_event.argtypes = [i32, i32, P(ctypes.c_uint32), P(dbl), P(dbl)]
    L.mg_flops_per_event_shape.argtypes = [i32, i32, P(ctypes.c_uint32), i32, P(dbl), P(dbl)]
    L.mg_autotune.argtypes = [vp, i32, i64, ctypes.c_char_p, P(dbl)]
    L.mg_get_launch_shape.argtypes = [vp, i32, P(i32), P(i32), P(i32)]
    L.mg_set_launch_shape.argtypes = [vp, i32, i32, i32, i32]
    L.mg_graph_create.argtypes = [P(Job), i32, P(vp)]
    L.mg_graph_create_ex.argtypes = [P(Job), i32, i32, P(vp)]
    L.mg_sigmakin_batch.argtypes = [P(BatchJob), i32, vp]
    L.mg_graph_update.argtypes = [vp, P(Job), i32]
    L.mg_graph_launch.argtypes = [vp, vp]
    L.mg_graph_nodes.argtypes = [vp, P(i32)]
    L.mg_graph_destroy.argtypes = [vp]
    L.mg_graph_destroy.restype = None
    for name in ("mg_autotune", "mg_get_launch_shape", "mg_set_launch_shape", "mg_graph_create", "mg_graph_create_ex",
                 "mg_graph_update", "mg_graph_launch", "mg_graph_nodes", "mg_sigmakin_batch"):
        getattr(L, name).restype = i32
    L.mg_serve_default_cfg.argtypes = [P(ServeCfg)]
    L.mg_serve_default_cfg.restype = None
    L.mg_serve_footprint.argtypes = [i32, i64, i32]
    L.mg_serve_footprint.restype = i64
    L.mg_serve_create.argtypes = [P(ServeCfg), P(vp)]
    L.mg_serve_submit.argtypes = [vp, i32, u64, i64, P(ctypes.c_uint64)]
    L.mg_serve_poll.argtypes = [vp, ctypes.c_uint64, vp, P(i32), P(dbl)]
    L.mg_serve_wait.argtypes = [vp, ctypes.c_uint64, vp, i64, P(dbl)]
    L.mg_serve_stats.argtypes = [vp, P(ctypes.c_int64), P(ctypes.c_int64), P(ctypes.c_int64), P(i32)]
    L.mg_serve_cancel.argtypes = [vp, ctypes.c_uint64]
    L.mg_serve_destroy.argtypes = [vp]
    L.mg_serve_destroy.restype = None
    for name in ("mg_serve_create", "mg_serve_submit", "mg_serve_poll", "mg_serve_wait", "mg_serve_stats"):
        getattr(L, name).restype = i32
    for name in ("mg_process_info", "mg_colour_matrix", "mg_create", "mg_philox", "mg_rambo", "mg_rambo_range",
                 "mg_measure_fma_peak", "mg_hel_filter",
                 "mg_sigmakin", "mg_sigmakin_host", "mg_sigmakin_noalloc", "mg_sigmakin_lhe", "mg_alphas_running",
                 "mg_colour_flow", "mg_sde_weights", "mg_sde_channels", "mg_sde_channel_key", "mg_hel_mask", "mg_check", "mg_flops_per_event",
                 "mg_flops_per_event_shape"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def _strerror(s):
    try:
        return lib().mg_strerror(s).decode()
    except Exception:
        return "?"


def _check(status, what):
    if status != 0:
        raise MGError(status, what)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("expected a tensor, ndarray or raw pointer, got %r" % type(x))


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _proc(p):
    return PROCESSES[p] if isinstance(p, str) else int(p)


# ------------------------------------------------------------------------------------------
# host-only queries
# ------------------------------------------------------------------------------------------
def default_params():
    p = Params()
    lib().mg_default_params(ctypes.byref(p))
    return p


def process_info(process):
    a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().mg_process_info(_proc(process), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)),
           "mg_process_info")
    return {"npar": a.value, "nhel": b.value, "ncol": c.value, "ndiagrams": d.value}


def mom_count(process, nevt):
    return int(lib().mg_mom_count(_proc(process), nevt))


def colour_matrix(process):
    """Exact colour matrix as (int64 numerators [ncol, ncol], common denominator)."""
    n = process_info(process)["ncol"]
    num = np.zeros((n, n), dtype=np.int64)
    den = ctypes.c_int64()
    _check(lib().mg_colour_matrix(_proc(process), num.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  ctypes.byref(den)), "mg_colour_matrix")
    return num, den.value


def sde_channels(process):
    """Keys of the single-diagram-enhancement channels of a process, in channel order (mg_sde_channel_key)."""
    n = ctypes.c_int()
    _check(lib().mg_sde_channels(_proc(process), ctypes.byref(n)), "mg_sde_channels")
    buf = ctypes.create_string_buffer(256)
    out = []
    for c in range(n.value):
        _check(lib().mg_sde_channel_key(_proc(process), c, buf, 256), "mg_sde_channel_key")
        out.append(buf.value.decode())
    return out


def colour_flow(process, flow):
    """Gluon labels along the quark line of colour flow `flow` (mg_colour_flow)."""
    n = process_info(process)["npar"] - 2
    out = (ctypes.c_int * n)()
    _check(lib().mg_colour_flow(_proc(process), flow, out), "mg_colour_flow")
    return list(out)


def flops_per_event(process, mask=None, precision=MG_FP64, flags=None):
    """(amplitude flops, colour-sum flops) of one event's ME in the given precision mode for the given
    helicity mask, for the algorithm the launch flags select (None: the defaults of a new Context)."""
    a, c = ctypes.c_double(), ctypes.c_double()
    m = None
    if mask is not None:
        m = (ctypes.c_uint32 * len(mask))(*[int(x) for x in mask])
    _check(lib().mg_flops_per_event_shape(_proc(process), precision, m, -1 if flags is None else int(flags),
                                          ctypes.byref(a), ctypes.byref(c)), "mg_flops_per_event_shape")
    return a.value, c.value


# ------------------------------------------------------------------------------------------
# layout helpers (pure index permutations of the AoSoA layout in mg.h)
# ------------------------------------------------------------------------------------------
def to_aosoa(mom):
    """[nevt, npar, 4] -> flat AoSoA array of mom_count doubles (zero padded to 32 events)."""
    mom = np.asarray(mom, dtype=np.float64)
    nevt, npar, _ = mom.shape
    npage = (nevt + PAGE - 1) // PAGE
    buf = np.zeros((npage * PAGE, npar, 4))
    buf[:nevt] = mom
    return np.ascontiguousarray(buf.reshape(npage, PAGE, npar, 4).transpose(0, 2, 3, 1)).reshape(-1)


def from_aosoa(buf, nevt, npar):
    buf = np.asarray(buf, dtype=np.float64)
    npage = (nevt + PAGE - 1) // PAGE
    a = buf[: npage * npar * 4 * PAGE].reshape(npage, npar, 4, PAGE).transpose(0, 3, 1, 2).reshape(-1, npar, 4)
    return a[:nevt]


def measure_fma_peak(fp32=False, iters=4096):
    """Measured FMA throughput of the current device in flop/s (FMA = 2 flops)."""
    r = ctypes.c_double()
    _check(lib().mg_measure_fma_peak(1 if fp32 else 0, iters, ctypes.byref(r)), "mg_measure_fma_peak")
    return r.value


def measure_mma_peak(iters=16384):
    """Measured dense FP16 tensor-core throughput (tcgen05.mma kind::f16) in flop/s; the accumulated
    integer result is checked exactly."""
    r = ctypes.c_double()
    _check(lib().mg_measure_mma_peak(iters, ctypes.byref(r)), "mg_measure_mma_peak")
    return r.value


def kernel_launches():
    """CUDA kernels this library has launched in this process so far (all contexts and streams)."""
    return int(lib().mg_kernel_launches())


def diag_fail_alloc(nth):
    """Fault injection on the host: the nth next allocation of the library fails (0 disarms)."""
    _check(lib().mg_diag_fail_alloc(int(nth)), "mg_diag_fail_alloc")


def live_allocs():
    """Device and pinned-host allocations of the library alive now."""
    return int(lib().mg_diag_live_allocs())


def philox(seed, nevt, nfinal, words, stream=None):
    _check(lib().mg_philox(seed, nevt, nfinal, _ptr(words), _stream(stream)), "mg_philox")


# ------------------------------------------------------------------------------------------
# contexts
# ------------------------------------------------------------------------------------------
class Context:
    """One process on the current CUDA device (mg_create / mg_destroy)."""

    def __init__(self, process, mt=173.0, wt=0.0, alphas=0.118, hel_warmup=1024, hel_tau=1e-9):
        self.process = _proc(process)
        info = process_info(self.process)
        self.npar, self.nhel, self.ncol = info["npar"], info["nhel"], info["ncol"]
        self.ng = self.npar - 4
        p = Params(mt, wt, alphas, hel_warmup, hel_tau)
        h = ctypes.c_void_p()
        _check(lib().mg_create(self.process, ctypes.byref(p), ctypes.byref(h)), "mg_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().mg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def mom_count(self, nevt):
        return mom_count(self.process, nevt)

    def rambo(self, seed, nevt, sqrts, mom, wgt=None, stream=None):
        _check(lib().mg_rambo(self._h, seed, nevt, sqrts, _ptr(mom), _ptr(wgt), _stream(stream)), "mg_rambo")

    def rambo_range(self, seed, e0, nevt, sqrts, mom, wgt=None, stream=None):
        _check(lib().mg_rambo_range(self._h, seed, e0, nevt, sqrts, _ptr(mom), _ptr(wgt), _stream(stream)),
               "mg_rambo_range")

    def hel_filter(self, mom, nevt, stream=None):
        _check(lib().mg_hel_filter(self._h, _ptr(mom), nevt, _stream(stream)), "mg_hel_filter")

    def sigmakin(self, mom, nevt, me, precision=MG_FP64, stream=None):
        _check(lib().mg_sigmakin(self._h, _ptr(mom), nevt, precision, _ptr(me), _stream(stream)), "mg_sigmakin")

    def sigmakin_host(self, mom_host, nevt, me_host, precision=MG_FP64, stream=None):
        _check(lib().mg_sigmakin_host(self._h, _ptr(mom_host), nevt, precision, _ptr(me_host), _stream(stream)),
               "mg_sigmakin_host")

    def sigmakin_noalloc(self, mom, nevt, me, stream=None):
        """FP64 MEs without any device allocation (fixed 16 MiB library scratch; see mg.h)."""
        _check(lib().mg_sigmakin_noalloc(self._h, _ptr(mom), nevt, _ptr(me), _stream(stream)), "mg_sigmakin_noalloc")

    def sigmakin_lhe(self, mom, nevt, me, rnd_hel=None, rnd_col=None, hel=None, col=None, running_alphas=False,
                     alphas=None, stream=None):
        """FP64 MEs with the per-event helicity and leading-colour choices (int32 outputs, from the
        caller's uniforms) and optionally the one-loop running coupling at mu = H_T/2 (see mg.h)."""
        _check(lib().mg_sigmakin_lhe(self._h, _ptr(mom), nevt, _ptr(rnd_hel), _ptr(rnd_col), 1 if running_alphas else 0,
                                     _ptr(me), _ptr(hel), _ptr(col), _ptr(alphas), _stream(stream)), "mg_sigmakin_lhe")

    def sde_weights(self, mom, nevt, w, stream=None):
        """Single-diagram-enhancement weights w[channel * nevt + e] (mg_sde_weights)."""
        _check(lib().mg_sde_weights(self._h, _ptr(mom), nevt, _ptr(w), _stream(stream)), "mg_sde_weights")

    def alphas_running(self, mom, nevt, me, alphas=None, stream=None):
        """In place: me[e] *= (alpha_s(H_T/2)/alpha_s)^(n_g+2), one-loop running (see mg.h)."""
        _check(lib().mg_alphas_running(self._h, _ptr(mom), nevt, _ptr(me), _ptr(alphas), _stream(stream)),
               "mg_alphas_running")

    def autotune(self, precision=MG_FP64, nevt=65536, cache_path=None):
        """Pick the fastest launch shape of the ME kernel for this context; returns (tile_ev, slot_major, ms)."""
        ms = ctypes.c_double()
        _check(lib().mg_autotune(self._h, precision, nevt, cache_path.encode() if cache_path else None,
                                 ctypes.byref(ms)), "mg_autotune")
        t, s, _ = self.launch_shape(precision)
        return t, s, ms.value

    def launch_shape(self, precision=MG_FP64):
        """(tile_ev, slot_major, flags) of the ME kernel launch for this precision (flags: LAUNCH_UNROLLED,
        LAUNCH_DF_REDO, LAUNCH_FUSED, LAUNCH_WARP, LAUNCH_TC_APART, LAUNCH_SHARED bits: mg.h MG_LAUNCH_*)."""
        t, s, u = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().mg_get_launch_shape(self._h, precision, ctypes.byref(t), ctypes.byref(s), ctypes.byref(u)),
               "mg_get_launch_shape")
        return t.value, s.value, u.value

    def set_launch_shape(self, precision, tile_ev=128, slot_major=0, flags=39):
        _check(lib().mg_set_launch_shape(self._h, precision, tile_ev, slot_major, flags), "mg_set_launch_shape")

    def hel_mask(self):
        nw = (self.nhel + 31) // 32
        m = (ctypes.c_uint32 * nw)()
        n = ctypes.c_int()
        _check(lib().mg_hel_mask(self._h, m, ctypes.byref(n)), "mg_hel_mask")
        return np.array(list(m), dtype=np.uint32), n.value

    def set_fp32_tau(self, tau):
        """FP32 modes: recompute the events whose smallest internal invariant is below tau * s."""
        _check(lib().mg_set_fp32_tau(self._h, tau), "mg_set_fp32_tau")

    def diag_tc_stall(self, on):
        """Diagnostics: the tensor-memory colour pass issues no MMAs, so its bounded waits run out."""
        _check(lib().mg_diag_tc_stall(self._h, 1 if on else 0), "mg_diag_tc_stall")

    def check(self, stream=None):
        """Returns the number of RAMBO events that failed to converge since the last check."""
        n = ctypes.c_int64()
        s = lib().mg_check(self._h, _stream(stream), ctypes.byref(n))
        if s not in (0, 4):
            _check(s, "mg_check")
        return n.value


# ------------------------------------------------------------------------------------------
# serving
# ------------------------------------------------------------------------------------------
def serve_footprint(process, nevt, precision=MG_FP64):
    return int(lib().mg_serve_footprint(_proc(process), nevt, precision))


class Server:
    """Continuous-batching request server (mg_serve_*)."""

    def __init__(self, slots=8, max_nevt=65536, hbm_cap_bytes=64 << 30, precision=MG_FP64, sqrts=1500.0,
                 mt=173.0, wt=0.0, alphas=0.118, hel_warmup=1024, hel_tau=1e-9):
        c = ServeCfg()
        lib().mg_serve_default_cfg(ctypes.byref(c))
        c.slots, c.max_nevt, c.hbm_cap_bytes, c.precision, c.sqrts = slots, max_nevt, hbm_cap_bytes, precision, sqrts
        c.params = Params(mt, wt, alphas, hel_warmup, hel_tau)
        h = ctypes.c_void_p()
        _check(lib().mg_serve_create(ctypes.byref(c), ctypes.byref(h)), "mg_serve_create")
        self._h = h
        self._nevt = {}

    def submit(self, process, seed, nevt):
        t = ctypes.c_uint64()
        _check(lib().mg_serve_submit(self._h, _proc(process), seed, nevt, ctypes.byref(t)), "mg_serve_submit")
        self._nevt[t.value] = nevt
        return t.value

    def poll(self, ticket):
        """None while in flight, else (me ndarray, latency_ms)."""
        out = np.empty(self._nevt[ticket])
        done, lat = ctypes.c_int(), ctypes.c_double()
        s = lib().mg_serve_poll(self._h, ticket, out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(done), ctypes.byref(lat))
        if s == 0 and not done.value:
            return None
        del self._nevt[ticket]
        _check(s, "mg_serve_poll")
        return out, lat.value

    def wait(self, ticket, timeout_ms=600000):
        out = np.empty(self._nevt[ticket])
        lat = ctypes.c_double()
        s = lib().mg_serve_wait(self._h, ticket, out.ctypes.data_as(ctypes.c_void_p), timeout_ms, ctypes.byref(lat))
        if s == 6:
            raise MGError(s, "mg_serve_wait")
        del self._nevt[ticket]
        _check(s, "mg_serve_wait")
        return out, lat.value

    def cancel(self, ticket):
        """Cancel a queued or running request; its wait/poll then raises MGError(MG_ECANCELED)."""
        _check(lib().mg_serve_cancel(self._h, ticket), "mg_serve_cancel")

    def stats(self):
        a, b, c, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        _check(lib().mg_serve_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)),
               "mg_serve_stats")
        return {"completed": a.value, "events": b.value, "peak_bytes": c.value, "peak_inflight": d.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().mg_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------------------------------------------
# graph batches
# ------------------------------------------------------------------------------------------
def sigmakin_batch(jobs, stream=None):
    """FP64 MEs of several jobs in one persistent launch (mg_sigmakin_batch).
    jobs: list of (Context, mom_tensor, nevt, me_tensor)."""
    arr = (BatchJob * len(jobs))()
    for i, (ctx, mom, nevt, me) in enumerate(jobs):
        arr[i] = BatchJob(ctx._h, _ptr(mom), nevt, _ptr(me))
    _check(lib().mg_sigmakin_batch(arr, len(jobs), _stream(stream)), "mg_sigmakin_batch")


class GraphBatch:
    """One CUDA graph running the full step of several jobs on parallel branches (mg_graph_*), or with
    persistent=True (FP64 jobs) all their matrix elements in one persistent launch (mg_graph_create_ex).
    jobs: list of (Context, seed, e0, nevt, sqrts, mom_tensor, me_tensor, precision)."""

    def __init__(self, jobs, persistent=False):
        arr = self._jobs(jobs)
        h = ctypes.c_void_p()
        _check(lib().mg_graph_create_ex(arr, len(jobs), GRAPH_PERSISTENT if persistent else 0, ctypes.byref(h)),
               "mg_graph_create_ex")
        self._h = h

    @staticmethod
    def _jobs(jobs):
        arr = (Job * len(jobs))()
        for i, (ctx, seed, e0, nevt, sqrts, mom, me, prec) in enumerate(jobs):
            arr[i] = Job(ctx._h, seed, e0, nevt, sqrts, _ptr(mom), _ptr(me), prec)
        return arr

    def update(self, jobs):
        _check(lib().mg_graph_update(self._h, self._jobs(jobs), len(jobs)), "mg_graph_update")

    def launch(self, stream=None):
        _check(lib().mg_graph_launch(self._h, _stream(stream)), "mg_graph_launch")

    def nodes(self):
        n = ctypes.c_int()
        _check(lib().mg_graph_nodes(self._h, ctypes.byref(n)), "mg_graph_nodes")
        return n.value

    def close(self):
        if getattr(self, "_h", None):
            lib().mg_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
