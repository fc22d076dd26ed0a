"""ctypes wrapper of the FP64 MPR oracle (``spring_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.  The product (the CUDA library and its binding) never
imports, links or runs anything here.

Every function takes and returns numpy arrays.  Complex arrays are ``complex128`` with
shape ``(batch, n, n)`` or ``(n, n)``; masks and supports are ``uint8``.  Fourier-space
arrays are in DFT order except for :func:`mpr_run`, which takes detector-centred input.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "spring_oracle.cpp"
_LIB_DIR = _HERE / "_lib"
_LIB = _LIB_DIR / "libspring_oracle.so"

_dp = C.POINTER(C.c_double)
_u8p = C.POINTER(C.c_uint8)
_ip = C.POINTER(C.c_int)
_lp = C.POINTER(C.c_long)
_u32p = C.POINTER(C.c_uint32)


def build(force: bool = False) -> Path:
    """Compile the oracle with g++ (portable flags: it builds on x86-64 and aarch64)."""
    _LIB_DIR.mkdir(exist_ok=True)
    if _LIB.exists() and not force and _LIB.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB
    tmp = _LIB.with_suffix(f".tmp{os.getpid()}.so")
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", str(_SRC), "-o", str(tmp)]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OrcParams(C.Structure):
    _fields_ = [
        ("pop", C.c_int), ("iters_per_gen", C.c_int), ("generations", C.c_int),
        ("algorithm", C.c_int),
        ("beta", C.c_double), ("sw_sigma", C.c_double), ("sw_threshold", C.c_double),
        ("sw_sigma_end", C.c_double), ("sw_threshold_end", C.c_double),
        ("sw_period", C.c_int), ("er_tail", C.c_int),
        ("chi", C.c_double), ("cw", C.c_double), ("cp", C.c_double),
        ("tile_min", C.c_int), ("tile_max", C.c_int), ("init_n_spheres", C.c_int),
        ("init_gamma", C.c_double), ("init_phi_max", C.c_double),
        ("seed", C.c_uint64),
        ("ub_eta", C.c_double), ("ub_max_missing", C.c_double), ("ub_max_saturated", C.c_double),
        ("schedule", C.c_int), ("mode", C.c_int), ("seq_ia", C.c_int), ("seq_er", C.c_int),
        ("seq_eval", C.c_int), ("repetitions", C.c_int), ("ca", C.c_double),
        ("monitor_avg", C.c_int),
    ]


class OrcResult(C.Structure):
    _fields_ = [
        ("rho_avg", _dp), ("rho_best", _dp), ("support_avg", _u8p),
        ("pop_x", _dp), ("pop_S", _u8p), ("pop_err", _dp), ("gen_stats", _dp),
        ("final_error_avg", C.c_double), ("final_error_best", C.c_double),
    ]


class OrcTrace(C.Structure):
    _fields_ = [("err_parents", _dp), ("err_new", _dp), ("replaced", _u8p), ("parents", _ip),
                ("areas", C.c_int64 * 3), ("best", C.c_int), ("gen_stats", C.c_double * 9)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(str(_LIB))
        sig = {
            "orc_set_threads": (None, [C.c_int]),
            "orc_get_threads": (C.c_int, []),
            "orc_fft2": (C.c_int, [_dp, C.c_int, C.c_int, C.c_int]),
            "orc_dft2_naive": (None, [_dp, _dp, C.c_int, C.c_int]),
            "orc_project_modulus": (C.c_int, [_dp, _dp, _dp, _u8p, C.c_int, C.c_int]),
            "orc_project_modulus_ub": (C.c_int, [_dp, _dp, _dp, _u8p, _dp, C.c_int, C.c_int]),
            "orc_upper_bounds": (None, [_dp, _u8p, _u8p, C.c_int, C.c_double, C.c_double,
                                        C.c_double, _dp]),
            "orc_sequence_counts": (None, [C.c_int, C.c_int, C.c_int, C.c_int, _ip]),
            "orc_iterate_ub": (C.c_int, [_dp, _u8p, _dp, _u8p, _dp, C.c_int, C.c_int, C.c_int,
                                         C.c_double, C.c_double, C.c_int]),
            "orc_iterate": (C.c_int, [_dp, _u8p, _dp, _u8p, C.c_int, C.c_int, C.c_int,
                                      C.c_double, C.c_double, C.c_int]),
            "orc_project_support": (None, [_dp, _u8p, C.c_int]),
            "orc_smooth": (None, [_dp, _dp, C.c_int, C.c_int, C.c_double]),
            "orc_update_support": (None, [_dp, _u8p, C.c_int, C.c_int, C.c_double, C.c_double]),
            "orc_update_support_size": (None, [_dp, _u8p, C.c_int, C.c_int, C.c_double, _lp]),
            "orc_fourier_error": (None, [_dp, _u8p, _dp, _u8p, C.c_int, C.c_int, _dp]),
            "orc_philox4x32_10": (None, [_u32p, _u32p, _u32p]),
            "orc_random_choice": (None, [C.c_uint64, C.c_int, C.c_int, C.c_int, _ip]),
            "orc_crossover_map": (None, [C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_int,
                                         C.c_int, C.c_double, _u8p]),
            "orc_map_geometry": (None, [C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_int,
                                        C.c_int, _ip]),
            "orc_cross_correlation": (None, [_dp, _dp, _u8p, C.c_int, _dp, _dp]),
            "orc_reshift": (None, [_dp, _u8p, _dp, _u8p, C.c_int, _dp, _u8p, _ip, _dp]),
            "orc_crossover": (None, [_dp, _u8p, _u8p, C.c_int, C.c_int, C.c_uint64, C.c_int,
                                     C.c_double, C.c_double, C.c_int, C.c_int, _dp, _u8p, _ip]),
            "orc_crossover_ca": (None, [_dp, _u8p, _u8p, C.c_int, C.c_int, C.c_uint64, C.c_int,
                                        C.c_double, C.c_double, C.c_int, C.c_int, C.c_double, _dp,
                                        _dp, _u8p, _ip]),
            "orc_average_moduli": (None, [_dp, _u8p, _u8p, C.c_int, C.c_int, C.c_int, _dp]),
            "orc_select": (C.c_int, [_dp, _dp, C.c_int, _u8p]),
            "orc_average": (None, [_dp, _u8p, _u8p, C.c_int, C.c_int, C.c_int, _dp, _u8p]),
            "orc_complexity": (C.c_double, [_dp, C.c_int, _dp]),
            "orc_initialize": (None, [C.c_uint64, _u8p, _dp, _u8p, C.c_int, C.c_int, C.c_int,
                                      C.c_double, C.c_double, _dp]),
            "orc_mpr_run": (C.c_int, [_dp, _u8p, _u8p, C.c_int, C.POINTER(OrcParams),
                                      C.POINTER(OrcResult)]),
            "orc_mpr_run_sat": (C.c_int, [_dp, _u8p, _u8p, _u8p, C.c_int, C.POINTER(OrcParams),
                                          C.POINTER(OrcResult)]),
            "orc_mpr_step": (C.c_int, [_dp, _u8p, _u8p, C.c_int, C.POINTER(OrcParams), C.c_int,
                                       _dp, _u8p, _dp, C.POINTER(OrcTrace)]),
            "orc_improve": (C.c_int, [_dp, _u8p, _dp, _u8p, C.c_int, C.c_int,
                                      C.POINTER(OrcParams), C.c_double, C.c_double, C.c_long,
                                      C.c_long, _dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# ---------------------------------------------------------------------------- helpers
def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _pd(a):
    return a.ctypes.data_as(_dp)


def _pu8(a):
    return a.ctypes.data_as(_u8p)


def _batched(x):
    x = _c128(x)
    squeeze = x.ndim == 2
    if squeeze:
        x = x[None]
    return x.copy(), squeeze


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


# ---------------------------------------------------------------------------- operators
def fft2(x, inverse=False):
    """Unitary 2D DFT (a1/a3) of each image."""
    x, sq = _batched(x)
    rc = lib().orc_fft2(_pd(x), x.shape[0], x.shape[1], int(inverse))
    if rc:
        raise ValueError("invalid side")
    return x[0] if sq else x


def dft2_naive(x, inverse=False):
    x = _c128(x)
    out = np.empty_like(x)
    lib().orc_dft2_naive(_pd(x), _pd(out), x.shape[0], int(inverse))
    return out


def project_modulus(x, M, mask):
    """P_M x with the masked modulus constraint (Eq. pm, Eq. pm_full)."""
    x, sq = _batched(x)
    out = np.empty_like(x)
    M, mask = _f64(M), _u8(mask)
    lib().orc_project_modulus(_pd(x), _pd(out), _pd(M), _pu8(mask), x.shape[0], x.shape[1])
    return out[0] if sq else out


def project_modulus_ub(x, M, mask, U):
    """P_M x with upper bounds on the missing moduli (Eq. pm_bounds); U in DFT order,
    negative where no bound applies."""
    x, sq = _batched(x)
    out = np.empty_like(x)
    M, mask, U = _f64(M), _u8(mask), _f64(U)
    lib().orc_project_modulus_ub(_pd(x), _pd(out), _pd(M), _pu8(mask), _pd(U), x.shape[0], x.shape[1])
    return out[0] if sq else out


def sequence_counts(seq_ia, seq_er, g, G):
    """(IA, ER) iteration counts of the paper's Sequence at generation g of G."""
    out = np.zeros(2, np.int32)
    lib().orc_sequence_counts(int(seq_ia), int(seq_er), int(g), int(G), out.ctypes.data_as(_ip))
    return int(out[0]), int(out[1])


def upper_bounds(I_centred, mask_centred, saturated=None, eta=1.5, max_missing=0.2, max_saturated=0.05):
    """Per-pixel amplitude bounds sqrt(mu + eta sigma) of the missing, unsaturated pixels
    (Eqs. avgint, stdint, upperbound), detector-centred; -1 where no bound applies."""
    I = _f64(I_centred)
    mask = _u8(mask_centred)
    n = I.shape[0]
    sat = None if saturated is None else _u8(saturated)
    U = np.empty((n, n), np.float64)
    lib().orc_upper_bounds(_pd(I), _pu8(mask), None if sat is None else _pu8(sat), n, float(eta),
                           float(max_missing), float(max_saturated), _pd(U))
    return U


def iterate(x, S, M, mask, alg, beta, chi, n_iter, U=None):
    """n_iter ER/HIO/RAAR iterations (alg 0/1/2) on each image; with U (DFT order,
    negative = no bound) the projection is Eq. pm_bounds."""
    x, sq = _batched(x)
    S = _u8(S)
    if S.ndim == 2:
        S = np.broadcast_to(S, x.shape).copy()
    M, mask = _f64(M), _u8(mask)
    if U is None:
        rc = lib().orc_iterate(_pd(x), _pu8(S), _pd(M), _pu8(mask), x.shape[0], x.shape[1],
                               int(alg), float(beta), float(chi), int(n_iter))
    else:
        U = _f64(U)
        rc = lib().orc_iterate_ub(_pd(x), _pu8(S), _pd(M), _pu8(mask), _pd(U), x.shape[0],
                                  x.shape[1], int(alg), float(beta), float(chi), int(n_iter))
    if rc:
        raise ValueError("invalid arguments")
    return x[0] if sq else x


def project_support(x, S):
    x = _c128(x).copy()
    S = _u8(S)
    lib().orc_project_support(_pd(x), _pu8(S), x.shape[0])
    return x


def smooth(x, sigma):
    x, sq = _batched(x)
    out = np.empty(x.shape, dtype=np.float64)
    lib().orc_smooth(_pd(x), _pd(out), x.shape[0], x.shape[1], float(sigma))
    return out[0] if sq else out


def update_support(x, sigma, tau):
    x, sq = _batched(x)
    S = np.empty(x.shape, dtype=np.uint8)
    lib().orc_update_support(_pd(x), _pu8(S), x.shape[0], x.shape[1], float(sigma), float(tau))
    return S[0] if sq else S


def update_support_size(x, sigma, alpha):
    x, sq = _batched(x)
    S = np.empty(x.shape, dtype=np.uint8)
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, dtype=np.int64), (x.shape[0],)),
                             dtype=C.c_long)
    lib().orc_update_support_size(_pd(x), _pu8(S), x.shape[0], x.shape[1], float(sigma),
                                  a.ctypes.data_as(_lp))
    return S[0] if sq else S


def fourier_error(x, S, M, mask):
    """GetError (Eq. error_calc) of each image."""
    x, sq = _batched(x)
    S = _u8(S)
    if S.ndim == 2:
        S = np.broadcast_to(S, x.shape).copy()
    M, mask = _f64(M), _u8(mask)
    err = np.empty(x.shape[0], dtype=np.float64)
    lib().orc_fourier_error(_pd(x), _pu8(S), _pd(M), _pu8(mask), x.shape[0], x.shape[1], _pd(err))
    return float(err[0]) if sq else err


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    lib().orc_philox4x32_10(c.ctypes.data_as(_u32p), k.ctypes.data_as(_u32p),
                            out.ctypes.data_as(_u32p))
    return out


def random_choice(seed, g, p, P):
    out = (C.c_int * 3)()
    lib().orc_random_choice(C.c_uint64(seed), g, p, P, out)
    return tuple(out)


def crossover_map(seed, g, p, n, tmin, tmax, cp):
    m = np.empty((n, n), dtype=np.uint8)
    lib().orc_crossover_map(C.c_uint64(seed), g, p, n, tmin, tmax, float(cp), _pu8(m))
    return m


def map_geometry(seed, g, p, n, tmin, tmax):
    out = (C.c_int * 5)()
    lib().orc_map_geometry(C.c_uint64(seed), g, p, n, tmin, tmax, out)
    return tuple(out)


def cross_correlation(x, ref, mask):
    x, ref, mask = _c128(x), _c128(ref), _u8(mask)
    c = np.empty_like(x)
    ct = np.empty_like(x)
    lib().orc_cross_correlation(_pd(x), _pd(ref), _pu8(mask), x.shape[0], _pd(c), _pd(ct))
    return c, ct


def reshift(x, S, ref, mask):
    """Align (x, S) onto ref; returns (x', S', (sy, sx, twin), phase)."""
    x, ref, mask = _c128(x), _c128(ref), _u8(mask)
    S = _u8(S) if S is not None else np.zeros(x.shape, np.uint8)
    xo = np.empty_like(x)
    So = np.empty(x.shape, np.uint8)
    info = (C.c_int * 3)()
    ph = C.c_double()
    lib().orc_reshift(_pd(x), _pu8(S), _pd(ref), _pu8(mask), x.shape[0], _pd(xo), _pu8(So),
                      info, C.byref(ph))
    return xo, So, tuple(info), ph.value


def crossover(pop_x, pop_S, mask, seed, g, cw, cp, tmin, tmax, ca=0.0, Mavg=None):
    """Alg. crossover; with ca > 0 the parent a's moduli move towards Mavg (Eq. crossavg)."""
    pop_x, pop_S, mask = _c128(pop_x), _u8(pop_S), _u8(mask)
    P, n = pop_x.shape[0], pop_x.shape[1]
    nx = np.empty_like(pop_x)
    nS = np.empty_like(pop_S)
    par = np.empty((P, 3), dtype=np.int32)
    if ca > 0.0:
        Mavg = _f64(Mavg)
        lib().orc_crossover_ca(_pd(pop_x), _pu8(pop_S), _pu8(mask), P, n, C.c_uint64(seed), g,
                               float(cw), float(cp), tmin, tmax, float(ca), _pd(Mavg), _pd(nx),
                               _pu8(nS), par.ctypes.data_as(_ip))
    else:
        lib().orc_crossover(_pd(pop_x), _pu8(pop_S), _pu8(mask), P, n, C.c_uint64(seed), g,
                            float(cw), float(cp), tmin, tmax, _pd(nx), _pu8(nS),
                            par.ctypes.data_as(_ip))
    return nx, nS, par


def average_moduli(pop_x, pop_S, mask, best):
    """(|F rho_avg| + mean_p |F rho_p|) / 2 (Eqs. avgint1, avgint2), DFT order."""
    pop_x, pop_S, mask = _c128(pop_x), _u8(pop_S), _u8(mask)
    P, n = pop_x.shape[0], pop_x.shape[1]
    out = np.empty((n, n), np.float64)
    lib().orc_average_moduli(_pd(pop_x), _pu8(pop_S), _pu8(mask), P, n, int(best), _pd(out))
    return out


def select(e_old, e_new):
    e_old, e_new = _f64(e_old), _f64(e_new)
    r = np.empty(len(e_old), dtype=np.uint8)
    cnt = lib().orc_select(_pd(e_old), _pd(e_new), len(e_old), _pu8(r))
    return r, int(cnt)


def average(pop_x, pop_S, mask, best):
    pop_x, pop_S, mask = _c128(pop_x), _u8(pop_S), _u8(mask)
    P, n = pop_x.shape[0], pop_x.shape[1]
    avg = np.empty((n, n), np.complex128)
    Sa = np.empty((n, n), np.uint8)
    lib().orc_average(_pd(pop_x), _pu8(pop_S), _pu8(mask), P, n, int(best), _pd(avg), _pu8(Sa))
    return avg, Sa


def complexity(x):
    x = _c128(x)
    s = C.c_double()
    g = lib().orc_complexity(_pd(x), x.shape[0], C.byref(s))
    return float(g), s.value


def initialize(seed, S0, I, mask, P, n_spheres=5, gamma=1.0, phi_max=0.0):
    S0, I, mask = _u8(S0), _f64(I), _u8(mask)
    n = S0.shape[0]
    x = np.empty((P, n, n), np.complex128)
    lib().orc_initialize(C.c_uint64(seed), _pu8(S0), _pd(I), _pu8(mask), n, P, int(n_spheres),
                         float(gamma), float(phi_max), _pd(x))
    return x


DEFAULTS = dict(pop=8, iters_per_gen=100, generations=5, algorithm=2, beta=0.9,
                sw_sigma=1.5, sw_threshold=0.2, sw_sigma_end=None, sw_threshold_end=None,
                sw_period=20, er_tail=10, chi=0.5, cw=0.4, cp=0.6, tile_min=4, tile_max=0,
                init_n_spheres=5, init_gamma=1.0, init_phi_max=0.0, seed=0,
                ub_eta=0.0, ub_max_missing=0.2, ub_max_saturated=0.05,
                schedule=0, mode=0, seq_ia=40, seq_er=40, seq_eval=40, repetitions=3, ca=0.0,
                monitor_avg=0)


def make_params(**kw) -> OrcParams:
    d = dict(DEFAULTS)
    d.update(kw)
    if d["sw_sigma_end"] is None:
        d["sw_sigma_end"] = d["sw_sigma"]
    if d["sw_threshold_end"] is None:
        d["sw_threshold_end"] = d["sw_threshold"]
    return OrcParams(**d)


def improve(x, S, M, mask, params: OrcParams, sigma, tau, a_best, a_eval):
    x, sq = _batched(x)
    S = _u8(S).copy()
    M, mask = _f64(M), _u8(mask)
    err = np.empty(x.shape[0], np.float64)
    rc = lib().orc_improve(_pd(x), _pu8(S), _pd(M), _pu8(mask), x.shape[0], x.shape[1],
                           C.byref(params), float(sigma), float(tau), int(a_best), int(a_eval),
                           _pd(err))
    if rc:
        raise ValueError("invalid arguments")
    return x, S, err


def mpr_step(I_centred, mask_centred, state, saturated=None, **kw):
    """One generation g = state["generation"] + 1 of Alg. mpr from a parent population
    (pop_x P x n x n complex, pop_S, pop_err).  Returns (state after generation g, trace of
    what it decided: improved errors of both populations, replacement flags, parents,
    areas, the alpha_best individual and the gen_stats row)."""
    I, mask = _f64(I_centred), _u8(mask_centred)
    n = I.shape[0]
    pr = make_params(**kw)
    P = pr.pop
    x = np.ascontiguousarray(state["pop_x"], np.complex128).copy()
    S = np.ascontiguousarray(state["pop_S"], np.uint8).copy()
    e = np.ascontiguousarray(state["pop_err"], np.float64).copy()
    tr = {"err_parents": np.full(P, np.nan), "err_new": np.full(P, np.nan),
          "replaced": np.zeros(P, np.uint8), "parents": np.full((P, 3), -1, np.int32)}
    t = OrcTrace(_pd(tr["err_parents"]), _pd(tr["err_new"]), _pu8(tr["replaced"]),
                 tr["parents"].ctypes.data_as(_ip))
    sat = None if saturated is None else _u8(saturated)
    g0 = int(state["generation"])
    rc = lib().orc_mpr_step(_pd(I), _pu8(mask), None if sat is None else _pu8(sat), n, C.byref(pr), g0,
                            _pd(x), _pu8(S), _pd(e), C.byref(t))
    if rc:
        raise ValueError("invalid MPR parameters or generation")
    tr["areas"] = np.array(list(t.areas), np.int64)
    tr["best"] = int(t.best)
    tr["gen_stats"] = np.array(list(t.gen_stats))
    return {"generation": g0 + 1, "pop_x": x, "pop_S": S, "pop_err": e}, tr


def mpr_run(I_centred, mask_centred, S0, keep_population=False, saturated=None, **kw):
    """Full MPR run (Alg. mpr).  Returns a dict with rho_avg, rho_best, support_avg,
    final errors, per-generation stats and (optionally) the final population."""
    I, mask, S0 = _f64(I_centred), _u8(mask_centred), _u8(S0)
    n = I.shape[0]
    pr = make_params(**kw)
    P, G = pr.pop, pr.generations
    avg = np.empty((n, n), np.complex128)
    best = np.empty((n, n), np.complex128)
    Sa = np.empty((n, n), np.uint8)
    stats = np.empty((G, 9), np.float64)
    res = OrcResult()
    res.rho_avg, res.rho_best, res.support_avg, res.gen_stats = _pd(avg), _pd(best), _pu8(Sa), _pd(stats)
    if keep_population:
        px = np.empty((P, n, n), np.complex128)
        pS = np.empty((P, n, n), np.uint8)
        pe = np.empty(P, np.float64)
        res.pop_x, res.pop_S, res.pop_err = _pd(px), _pu8(pS), _pd(pe)
    sat = None if saturated is None else _u8(saturated)
    rc = lib().orc_mpr_run_sat(_pd(I), _pu8(mask), None if sat is None else _pu8(sat), _pu8(S0), n,
                               C.byref(pr), C.byref(res))
    if rc:
        raise ValueError("invalid MPR parameters")
    out = dict(rho_avg=avg, rho_best=best, support_avg=Sa, gen_stats=stats,
               final_error_avg=res.final_error_avg, final_error_best=res.final_error_best)
    if keep_population:
        out.update(pop_x=px, pop_S=pS, pop_err=pe)
    return out
