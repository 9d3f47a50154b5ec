"""FP64 CPU oracle for gg -> t tbar + n gluons -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may import,
call, link or execute anything under oracle/.  The product path (paper_2210_11122_gb300)
never touches it, and nothing here imports the product package.

Contents:
  me_oracle.cpp  -- Philox4x32-10, massive RAMBO, helicity wavefunctions, colour-ordered
                    Berends-Giele recursion, colour sum, helicity filter, flop counter.
  colour.py      -- exact colour matrix by the SU(N) Fierz identity (Fractions).
  fullcolour.py  -- brute-force colour-dressed amplitudes with explicit SU(3) matrices.
  closed_form.py -- closed-form LO gg -> QQbar |M|^2 (Ellis-Stirling-Webber).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

from . import colour as _colour

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "me_oracle.cpp")
_lock = threading.Lock()
_lib = None

# physical defaults of the synthetic workloads
SQRTS = 1500.0
MT = 173.0
ALPHAS = 0.118


def build(force=False):
    """Compile me_oracle.cpp into oracle/_build/liboracle.so (plain IEEE: no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-pthread", _SRC, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.POINTER
            u32p, f64p, i32p, u64p = P(ctypes.c_uint32), P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_ulonglong)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, f64p]
            L.orc_rambo.argtypes = [ctypes.c_int, f64p, f64p, ctypes.c_double, f64p, f64p]
            L.orc_rambo.restype = ctypes.c_int
            L.orc_event.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                    f64p, f64p]
            L.orc_event.restype = ctypes.c_int
            L.orc_events.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                     ctypes.c_double, f64p, f64p, i32p]
            L.orc_events.restype = ctypes.c_int
            L.orc_me_hel.argtypes = [ctypes.c_int, f64p, f64p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, f64p, f64p]
            L.orc_me_batch.argtypes = [ctypes.c_int, ctypes.c_int64, f64p, f64p, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, u32p, f64p, ctypes.c_int]
            L.orc_flops.argtypes = [ctypes.c_int, f64p, f64p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    u32p, u64p]
            L.orc_hel_mask.argtypes = [ctypes.c_int, ctypes.c_int64, f64p, f64p, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, u32p, f64p, ctypes.c_int]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def npar(ng):
    return ng + 4


def nhel(ng):
    return 1 << (ng + 4)


def ncol(ng):
    n = 1
    for i in range(2, ng + 3):
        n *= i
    return n


def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def uniforms(seed, e, j):
    out = np.zeros(4)
    lib().orc_uniforms(seed, e, j, _p(out, ctypes.c_double))
    return out


def rambo(masses, u, sqrts):
    """Massive RAMBO from uniforms u[n][4]; returns (p[n][4], weight, status)."""
    m = _f64(masses)
    u = _f64(u)
    n = len(m)
    p = np.zeros((n, 4))
    w = np.zeros(1)
    st = lib().orc_rambo(n, _p(m, ctypes.c_double), _p(u, ctypes.c_double), sqrts, _p(p, ctypes.c_double),
                         _p(w, ctypes.c_double))
    return p, w[0], st


def events(ng, seed, nevt, e0=0, sqrts=SQRTS, mt=MT):
    """Momenta [nevt][npar][4] (particle order g1 g2 t tbar g3..), weights, per-event status."""
    mom = np.zeros((nevt, npar(ng), 4))
    wgt = np.zeros(nevt)
    st = np.zeros(nevt, dtype=np.int32)
    lib().orc_events(ng, seed, e0, nevt, sqrts, mt, _p(mom, ctypes.c_double), _p(wgt, ctypes.c_double),
                     _p(st, ctypes.c_int))
    return mom, wgt, st


def colour_matrix(ng):
    return _colour.colour_matrix(ng + 2)


def me_hel(ng, p, mt=MT, wt=0.0, alphas=ALPHAS, gauge_gluon=-1, want_jamps=False, colour=None):
    """Per-helicity colour-summed |M_h|^2 (not averaged) for one event p[npar][4]."""
    p = _f64(p)
    C = _f64(colour_matrix(ng) if colour is None else colour)
    mh = np.zeros(nhel(ng))
    jp = np.zeros((nhel(ng), ncol(ng), 2)) if want_jamps else None
    lib().orc_me_hel(ng, _p(p, ctypes.c_double), _p(C, ctypes.c_double), mt, wt, alphas, gauge_gluon,
                     _p(mh, ctypes.c_double), _p(jp, ctypes.c_double) if want_jamps else None)
    if want_jamps:
        return mh, jp[..., 0] + 1j * jp[..., 1]
    return mh


def full_mask(ng):
    nw = (nhel(ng) + 31) // 32
    m = np.zeros(nw, dtype=np.uint32)
    for h in range(nhel(ng)):
        m[h >> 5] |= np.uint32(1 << (h & 31))
    return m


def me_batch(ng, mom, mask=None, mt=MT, wt=0.0, alphas=ALPHAS, nthreads=1):
    """Averaged ME per event: (1/256)(1/ng!) sum_{h in mask} sum_colours |M_h|^2."""
    mom = _f64(mom)
    nevt = mom.shape[0]
    C = _f64(colour_matrix(ng))
    mask = np.ascontiguousarray(full_mask(ng) if mask is None else mask, dtype=np.uint32)
    me = np.zeros(nevt)
    lib().orc_me_batch(ng, nevt, _p(mom, ctypes.c_double), _p(C, ctypes.c_double), mt, wt, alphas,
                       _p(mask, ctypes.c_uint32), _p(me, ctypes.c_double), nthreads)
    return me


def hel_mask(ng, mom, tau=1e-9, mt=MT, wt=0.0, alphas=ALPHAS, nthreads=1):
    """Helicity filter: good(h) <=> max_e |M_h|^2 / sum_h' |M_h'|^2 > tau.  Returns (mask, maxratio)."""
    mom = _f64(mom)
    C = _f64(colour_matrix(ng))
    mask = np.zeros((nhel(ng) + 31) // 32, dtype=np.uint32)
    ratio = np.zeros(nhel(ng))
    lib().orc_hel_mask(ng, mom.shape[0], _p(mom, ctypes.c_double), _p(C, ctypes.c_double), mt, wt, alphas, tau,
                       _p(mask, ctypes.c_uint32), _p(ratio, ctypes.c_double), nthreads)
    return mask, ratio


def flops(ng, p, mask=None, mt=MT, wt=0.0, alphas=ALPHAS):
    """Operation counts of one event: dict with amplitude and colour-sum add/mul/div/sqrt."""
    p = _f64(p)
    C = _f64(colour_matrix(ng))
    mask = np.ascontiguousarray(full_mask(ng) if mask is None else mask, dtype=np.uint32)
    c = np.zeros(8, dtype=np.uint64)
    lib().orc_flops(ng, _p(p, ctypes.c_double), _p(C, ctypes.c_double), mt, wt, alphas, _p(mask, ctypes.c_uint32),
                    _p(c, ctypes.c_ulonglong))
    keys = ["add", "mul", "div", "sqrt"]
    return {"amp": dict(zip(keys, map(int, c[:4]))), "colour": dict(zip(keys, map(int, c[4:])))}
