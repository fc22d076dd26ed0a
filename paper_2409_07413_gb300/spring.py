"""ctypes binding of libspring (include/spring.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; all computation runs
in the library's CUDA kernels.  Operator functions take torch CUDA tensors (complex64 for
densities, float32 moduli, uint8 supports) and run on torch's current stream.  There is no
fallback: if ``libspring.so`` is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

_LIB_PATH = Path(__file__).resolve().parent / "_lib" / "libspring.so"

OK, E_INVALID, E_NOMEM, E_CUDA, E_BUSY, E_TIMEOUT, E_NOT_FOUND, E_NUMERIC, E_CANCELLED = range(9)
KC_ROW_ITER, KC_COL_PM, KC_OTHER, KC_FUSED = 0, 1, 2, 3
ABI_VERSION = 2  # SPRING_ABI_VERSION of the header this binding follows


class SpringError(RuntimeError):
    def __init__(self, status, name, msg):
        super().__init__(f"{name}: status {status} ({msg})")
        self.status = status


class Params(C.Structure):
    _fields_ = [
        ("pop", C.c_int), ("iters_per_gen", C.c_int), ("generations", C.c_int),
        ("algorithm", C.c_int), ("beta", C.c_float), ("sw_sigma", C.c_float),
        ("sw_threshold", C.c_float), ("sw_sigma_end", C.c_float), ("sw_threshold_end", C.c_float),
        ("sw_period", C.c_int), ("er_tail", C.c_int), ("chi", C.c_float), ("cw", C.c_float),
        ("cp", C.c_float), ("tile_min", C.c_int), ("tile_max", C.c_int),
        ("init_n_spheres", C.c_int), ("init_gamma", C.c_float), ("init_phi_max", C.c_float),
        ("precision", C.c_int), ("use_graph", C.c_int), ("schedule", C.c_int), ("mode", C.c_int),
        ("seq_ia", C.c_int), ("seq_er", C.c_int), ("seq_eval", C.c_int), ("repetitions", C.c_int),
        ("ca", C.c_float), ("monitor_avg", C.c_int), ("seed", C.c_uint64),
    ]


class Result(C.Structure):
    _fields_ = [
        ("rho_avg", C.c_void_p), ("rho_best", C.c_void_p), ("support_avg", C.c_void_p),
        ("gen_stats", C.c_void_p), ("final_error_avg", C.c_double),
        ("final_error_best", C.c_double), ("t_submit_s", C.c_double), ("t_admit_s", C.c_double),
        ("t_done_s", C.c_double),
    ]


class Population(C.Structure):
    _fields_ = [("generation", C.c_int), ("pop_x", C.c_void_p), ("pop_S", C.c_void_p),
                ("pop_err", C.c_void_p)]


class GenerationTrace(C.Structure):
    _fields_ = [("err_parents", C.c_void_p), ("err_new", C.c_void_p), ("replaced", C.c_void_p),
                ("parents", C.c_void_p), ("areas", C.c_int64 * 3), ("best", C.c_int32),
                ("gen_stats", C.c_double * 9)]


class Bounds(C.Structure):
    _fields_ = [("eta", C.c_float), ("max_missing", C.c_float), ("max_saturated", C.c_float)]


class KernelStat(C.Structure):
    _fields_ = [("launches", C.c_uint64), ("total_ms", C.c_double), ("timed", C.c_uint64),
                ("bytes_per_launch", C.c_double)]


_vp = C.c_void_p
_i, _f, _u64 = C.c_int, C.c_float, C.c_uint64
_SIGS = {
    "spring_abi_version": (_i, []),
    "spring_check_wait_timeout": (_i, [C.c_longlong]),
    "spring_status_string": (C.c_char_p, [_i]),
    "spring_mpr_step": (_i, [_vp, C.POINTER(Params), C.POINTER(Population), C.POINTER(Population),
                             C.POINTER(GenerationTrace)]),
    "spring_last_error": (C.c_char_p, []),
    "spring_params_default": (None, [C.POINTER(Params)]),
    "spring_init": (_i, [_i, C.c_size_t, C.POINTER(_vp)]),
    "spring_shutdown": (_i, [_vp]),
    "spring_problem_create": (_i, [_vp, _i, _i, _vp, _vp, _vp, C.POINTER(_vp)]),
    "spring_problem_create_device": (_i, [_vp, _i, _i, _vp, _vp, _vp, _vp, C.POINTER(_vp)]),
    "spring_problem_create_bounded": (_i, [_vp, _i, _i, _vp, _vp, _vp, _vp, C.POINTER(Bounds),
                                           C.POINTER(_vp)]),
    "spring_bounds_default": (None, [C.POINTER(Bounds)]),
    "spring_modulus_encode": (_i, [_vp, _vp, _vp, _i, C.POINTER(Bounds), _vp, _vp]),
    "spring_problem_destroy": (_i, [_vp]),
    "spring_footprint_bytes": (C.c_size_t, [_i, C.POINTER(Params)]),
    "spring_mpr_run": (_i, [_vp, C.POINTER(Params), C.POINTER(Result)]),
    "spring_mpr_run_batch": (_i, [_vp, _i, C.POINTER(Params), _vp, _vp]),
    "spring_submit": (_i, [_vp, _vp, C.POINTER(Params), C.POINTER(_u64)]),
    "spring_mpr_run_until": (_i, [_vp, C.POINTER(Params), _i, C.POINTER(Population)]),
    "spring_mpr_resume": (_i, [_vp, C.POINTER(Params), C.POINTER(Population), C.POINTER(Result)]),
    "spring_poll": (_i, [_vp, _u64, _i, C.POINTER(Result)]),
    "spring_cancel": (_i, [_vp, _u64]),
    "spring_serving_stats": (_i, [_vp, C.POINTER(_u64), C.POINTER(_u64)]),
    "spring_fft2": (_i, [_vp, _i, _i, _i, _vp]),
    "spring_project_modulus": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "spring_iterate": (_i, [_vp, _vp, _vp, _i, _i, _i, _f, _f, _i, _vp]),
    "spring_iterate_ex": (_i, [_vp, _vp, _vp, _i, _i, _i, _f, _f, _i, _i, _vp]),
    "spring_iterate_fused": (_i, [_vp, _vp, _vp, _i, _i, _i, _f, _f, _i, _vp]),
    "spring_smooth": (_i, [_vp, _vp, _i, _i, _f, _vp]),
    "spring_update_support": (_i, [_vp, _vp, _i, _i, _f, _f, _vp]),
    "spring_update_support_size": (_i, [_vp, _vp, _i, _i, _f, _vp, _vp]),
    "spring_fourier_error": (_i, [_vp, _vp, _vp, _i, _i, _vp, _vp]),
    "spring_fourier_error_noalloc": (_i, [_vp, _vp, _vp, _i, _i, _vp, _vp]),
    "spring_area_stats": (_i, [_vp, _vp, _i, _i, _i, _i, _vp, _vp]),
    "spring_random_choice": (_i, [_u64, _i, _i, _vp, _vp]),
    "spring_crossover_map": (_i, [_u64, _i, _i, _i, _i, _i, _f, _vp, _vp]),
    "spring_reshift": (_i, [_vp, _vp, _vp, _vp, _i, _i, _vp, _vp, _vp, _vp, _vp]),
    "spring_crossover": (_i, [_vp, _vp, _vp, _i, _i, _u64, _i, _f, _f, _i, _i, _vp, _vp, _vp, _vp]),
    "spring_crossover_ca": (_i, [_vp, _vp, _vp, _i, _i, _u64, _i, _f, _f, _i, _i, _f, _vp, _vp, _vp, _vp, _vp]),
    "spring_average_moduli": (_i, [_vp, _vp, _vp, _vp, _i, _i, _vp, _vp]),
    "spring_select": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _i, _i, _vp, _vp]),
    "spring_average": (_i, [_vp, _vp, _vp, _vp, _i, _i, _vp, _vp, _vp]),
    "spring_initialize": (_i, [_u64, _vp, _vp, _i, _i, _i, _f, _f, _vp, _vp]),
    "spring_set_kernel_variant": (_i, [_i, _i, _i]),
    "spring_get_kernel_variant": (_i, [_i, C.POINTER(_i), C.POINTER(_i)]),
    "spring_autotune": (_i, [_i, _i, _vp]),
    "spring_set_iteration_path": (_i, [_i, _i]),
    "spring_get_iteration_path": (_i, [_i, C.POINTER(_i)]),
    "spring_stats_reset": (None, []),
    "spring_stats_enable_timing": (None, [_i]),
    "spring_stats_get": (None, [_i, C.POINTER(KernelStat)]),
    "spring_launch_count": (_u64, []),
}

# entry points declared in include/spring.h (checked by the ABI test)
EXPORTED = tuple(_SIGS)

_lib = None


def lib_path() -> Path:
    return _LIB_PATH


def lib():
    """Load libspring.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise RuntimeError(f"{_LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(str(_LIB_PATH))
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        if L.spring_abi_version() != ABI_VERSION:
            raise RuntimeError(f"{_LIB_PATH} has ABI version {L.spring_abi_version()}, this binding "
                               f"expects {ABI_VERSION}: rebuild the library")
        _lib = L
    return _lib


def last_error() -> str:
    return lib().spring_last_error().decode(errors="replace")


def _check(status, name):
    if status != OK:
        raise SpringError(status, name, last_error())
    return status


def _call(name, *args):
    return _check(getattr(lib(), name)(*args), name)


# ------------------------------------------------------------------ tensor helpers
def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _batch_n(x):
    if x.dim() == 2:
        return 1, x.shape[-1]
    return x.shape[0], x.shape[-1]


# ------------------------------------------------------------------ parameters
GEN_STATS_COLS = 9  # columns of a result's gen_stats (SPRING_GEN_STATS_COLS)


def params(**kw) -> Params:
    p = Params()
    lib().spring_params_default(C.byref(p))
    ends = {"sw_sigma_end": "sw_sigma", "sw_threshold_end": "sw_threshold"}
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    for e, s in ends.items():
        if e not in kw and s in kw:
            setattr(p, e, kw[s])
    return p


def bounds(**kw) -> Bounds:
    """Upper-bound settings (Eq. pm_bounds); defaults eta 1.5, max_missing 0.2,
    max_saturated 0.05."""
    b = Bounds()
    lib().spring_bounds_default(C.byref(b))
    for k, v in kw.items():
        if not hasattr(b, k):
            raise KeyError(k)
        setattr(b, k, v)
    return b


def spring_modulus_encode(I, mask, saturated=None, bounds_=None, out=None):
    """Modulus array (DFT order) of detector-centred device I / mask (/ saturated)."""
    import torch
    _need(I, torch.float32, "I")
    _need(mask, torch.uint8, "mask")
    n = I.shape[-1]
    M = out if out is not None else torch.empty((n, n), dtype=torch.float32, device=I.device)
    _call("spring_modulus_encode", _ptr(I), _ptr(mask), _ptr(saturated) if saturated is not None else None,
          n, C.byref(bounds_) if bounds_ is not None else None, _ptr(M), _stream())
    return M


def footprint_bytes(n: int, p: Params) -> int:
    return int(lib().spring_footprint_bytes(n, C.byref(p)))


# ------------------------------------------------------------------ operators
def spring_fft2(x, inverse=False):
    import torch
    _need(x, torch.complex64, "x")
    b, n = _batch_n(x)
    _call("spring_fft2", _ptr(x), b, n, int(inverse), _stream())
    return x


def spring_project_modulus(x, M, out=None):
    import torch
    _need(x, torch.complex64, "x")
    _need(M, torch.float32, "M")
    out = torch.empty_like(x) if out is None else out
    b, n = _batch_n(x)
    _call("spring_project_modulus", _ptr(x), _ptr(out), _ptr(M), b, n, _stream())
    return out


def spring_iterate(x, S, M, algorithm, beta, chi, n_iter):
    import torch
    _need(x, torch.complex64, "x")
    _need(S, torch.uint8, "S")
    _need(M, torch.float32, "M")
    b, n = _batch_n(x)
    _call("spring_iterate", _ptr(x), _ptr(S), _ptr(M), b, n, int(algorithm), float(beta),
          float(chi), int(n_iter), _stream())
    return x


def spring_iterate_ex(x, S, M, algorithm, beta, chi, n_iter, precision):
    import torch
    _need(x, torch.complex64, "x")
    _need(S, torch.uint8, "S")
    _need(M, torch.float32, "M")
    b, n = _batch_n(x)
    _call("spring_iterate_ex", _ptr(x), _ptr(S), _ptr(M), b, n, int(algorithm), float(beta),
          float(chi), int(n_iter), int(precision), _stream())
    return x


def spring_iterate_fused(x, S, M, algorithm, beta, chi, n_iter):
    """spring_iterate on chip (N <= 256): one thread-block cluster per image."""
    import torch
    _need(x, torch.complex64, "x")
    _need(S, torch.uint8, "S")
    _need(M, torch.float32, "M")
    b, n = _batch_n(x)
    _call("spring_iterate_fused", _ptr(x), _ptr(S), _ptr(M), b, n, int(algorithm), float(beta),
          float(chi), int(n_iter), _stream())
    return x


def spring_smooth(x, sigma, out=None):
    import torch
    _need(x, torch.complex64, "x")
    out = torch.empty(x.shape, dtype=torch.float32, device=x.device) if out is None else out
    b, n = _batch_n(x)
    _call("spring_smooth", _ptr(x), _ptr(out), b, n, float(sigma), _stream())
    return out


def spring_update_support(x, sigma, tau, S=None):
    import torch
    _need(x, torch.complex64, "x")
    S = torch.empty(x.shape, dtype=torch.uint8, device=x.device) if S is None else S
    b, n = _batch_n(x)
    _call("spring_update_support", _ptr(x), _ptr(S), b, n, float(sigma), float(tau), _stream())
    return S


def spring_update_support_size(x, sigma, alpha, S=None):
    import torch
    _need(x, torch.complex64, "x")
    b, n = _batch_n(x)
    a = torch.as_tensor(alpha, dtype=torch.int64).reshape(-1).expand(b).contiguous().to(x.device)
    S = torch.empty(x.shape, dtype=torch.uint8, device=x.device) if S is None else S
    _call("spring_update_support_size", _ptr(x), _ptr(S), b, n, float(sigma), _ptr(a), _stream())
    return S


def spring_fourier_error(x, S, M):
    import torch
    _need(x, torch.complex64, "x")
    _need(S, torch.uint8, "S")
    _need(M, torch.float32, "M")
    b, n = _batch_n(x)
    err = torch.empty(b, dtype=torch.float64, device=x.device)
    _call("spring_fourier_error", _ptr(x), _ptr(S), _ptr(M), b, n, _ptr(err), _stream())
    return err


def spring_fourier_error_noalloc(x, S, M, err=None):
    """GetError with the library's fixed device scratch (no allocation by the library)."""
    import torch
    _need(x, torch.complex64, "x")
    _need(S, torch.uint8, "S")
    _need(M, torch.float32, "M")
    b, n = _batch_n(x)
    if err is None:
        err = torch.empty(b, dtype=torch.float64, device=x.device)
    _call("spring_fourier_error_noalloc", _ptr(x), _ptr(S), _ptr(M), b, n, _ptr(err), _stream())
    return err


def spring_area_stats(S, err, g, G):
    import torch
    _need(S, torch.uint8, "S")
    P, n = S.shape[0], S.shape[-1]
    out = torch.empty(3, dtype=torch.int64, device=S.device)
    _call("spring_area_stats", _ptr(S), _ptr(err), P, n, int(g), int(G), _ptr(out), _stream())
    return out


def spring_random_choice(seed, g, P, device="cuda"):
    import torch
    abc = torch.empty((P, 3), dtype=torch.int32, device=device)
    _call("spring_random_choice", C.c_uint64(seed), int(g), int(P), _ptr(abc), _stream())
    return abc


def spring_crossover_map(seed, g, p, n, tile_min=4, tile_max=0, cp=0.6, device="cuda"):
    import torch
    m = torch.empty((n, n), dtype=torch.uint8, device=device)
    _call("spring_crossover_map", C.c_uint64(seed), int(g), int(p), int(n), int(tile_min),
          int(tile_max), float(cp), _ptr(m), _stream())
    return m


def spring_reshift(x, S, ref, M):
    """Align each x[b] (and S[b]) onto ref[b]; returns (x', S', info (B, 3), phase (B,))."""
    import torch
    _need(x, torch.complex64, "x")
    _need(ref, torch.complex64, "ref")
    _need(M, torch.float32, "M")
    b, n = _batch_n(x)
    xo = torch.empty_like(x)
    So = torch.empty(x.shape, dtype=torch.uint8, device=x.device) if S is not None else None
    info = torch.empty((b, 3), dtype=torch.int32, device=x.device)
    ph = torch.empty(b, dtype=torch.float32, device=x.device)
    _call("spring_reshift", _ptr(x), _ptr(S), _ptr(ref), _ptr(M), b, n, _ptr(xo), _ptr(So),
          _ptr(info), _ptr(ph), _stream())
    return xo, So, info, ph


def spring_crossover(pop_x, pop_S, M, seed, g, cw=0.4, cp=0.6, tile_min=4, tile_max=0):
    import torch
    _need(pop_x, torch.complex64, "pop_x")
    _need(pop_S, torch.uint8, "pop_S")
    P, n = pop_x.shape[0], pop_x.shape[-1]
    nx = torch.empty_like(pop_x)
    nS = torch.empty_like(pop_S)
    par = torch.empty((P, 3), dtype=torch.int32, device=pop_x.device)
    _call("spring_crossover", _ptr(pop_x), _ptr(pop_S), _ptr(M), P, n, C.c_uint64(seed), int(g),
          float(cw), float(cp), int(tile_min), int(tile_max), _ptr(nx), _ptr(nS), _ptr(par),
          _stream())
    return nx, nS, par


def spring_crossover_ca(pop_x, pop_S, M, seed, g, ca, mavg, cw=0.4, cp=0.6, tile_min=4, tile_max=0):
    import torch
    _need(pop_x, torch.complex64, "pop_x")
    _need(pop_S, torch.uint8, "pop_S")
    P, n = pop_x.shape[0], pop_x.shape[-1]
    nx = torch.empty_like(pop_x)
    nS = torch.empty_like(pop_S)
    par = torch.empty((P, 3), dtype=torch.int32, device=pop_x.device)
    _call("spring_crossover_ca", _ptr(pop_x), _ptr(pop_S), _ptr(M), P, n, C.c_uint64(seed), int(g),
          float(cw), float(cp), int(tile_min), int(tile_max), float(ca),
          _ptr(mavg) if mavg is not None else None, _ptr(nx), _ptr(nS), _ptr(par), _stream())
    return nx, nS, par


def spring_average_moduli(pop_x, pop_S, err, M):
    import torch
    _need(pop_x, torch.complex64, "pop_x")
    P, n = pop_x.shape[0], pop_x.shape[-1]
    out = torch.empty((n, n), dtype=torch.float32, device=pop_x.device)
    _call("spring_average_moduli", _ptr(pop_x), _ptr(pop_S), _ptr(err) if err is not None else None,
          _ptr(M), P, n, _ptr(out), _stream())
    return out


def spring_select(pop_x, pop_S, pop_err, new_x, new_S, new_err):
    import torch
    P, n = pop_x.shape[0], pop_x.shape[-1]
    rep = torch.empty(P, dtype=torch.uint8, device=pop_x.device)
    _call("spring_select", _ptr(pop_x), _ptr(pop_S), _ptr(pop_err), _ptr(new_x), _ptr(new_S),
          _ptr(new_err), P, n, _ptr(rep), _stream())
    return rep


def spring_average(pop_x, pop_S, err, M):
    import torch
    P, n = pop_x.shape[0], pop_x.shape[-1]
    avg = torch.empty((n, n), dtype=torch.complex64, device=pop_x.device)
    Sa = torch.empty((n, n), dtype=torch.uint8, device=pop_x.device)
    _call("spring_average", _ptr(pop_x), _ptr(pop_S), _ptr(err), _ptr(M), P, n, _ptr(avg),
          _ptr(Sa), _stream())
    return avg, Sa


def spring_initialize(seed, S0, M, P, n_spheres=5, gamma=1.0, phi_max=0.0):
    import torch
    n = S0.shape[-1]
    x = torch.empty((P, n, n), dtype=torch.complex64, device=S0.device)
    _call("spring_initialize", C.c_uint64(seed), _ptr(S0), _ptr(M), n, int(P), int(n_spheres),
          float(gamma), float(phi_max), _ptr(x), _stream())
    return x


# ------------------------------------------------------------------ kernel variants
def set_kernel_variant(n, row=-1, col=-1):
    _call("spring_set_kernel_variant", int(n), int(row), int(col))


def get_kernel_variant(n):
    r, c = C.c_int(), C.c_int()
    _call("spring_get_kernel_variant", int(n), C.byref(r), C.byref(c))
    return r.value, c.value


def autotune(n, batch):
    _call("spring_autotune", int(n), int(batch), _stream())
    return get_kernel_variant(n)


# ------------------------------------------------------------------ instrumentation
def set_iteration_path(n, path):
    """0: two passes through HBM per iteration; 1: on chip (N <= 256); 2: the split passes
    (N = 192, 384, 512, 768, 1024: the column transform's first radix-Q stage in the row
    pass, Q = 3 at 192, 384 and 768, 2 at 512, 8 at 1024)."""
    _call("spring_set_iteration_path", int(n), int(path))


def get_iteration_path(n) -> int:
    p = C.c_int()
    _call("spring_get_iteration_path", int(n), C.byref(p))
    return p.value


def stats_reset():
    lib().spring_stats_reset()


def stats_enable_timing(on, stride: int = 1):
    """Per-launch CUDA-event timing of the iteration passes: off, or every `stride`-th
    launch of each timed kernel class."""
    lib().spring_stats_enable_timing(int(stride) if on else 0)


def stats_get(kc: int) -> KernelStat:
    s = KernelStat()
    lib().spring_stats_get(kc, C.byref(s))
    return s


def check_wait_timeout(cycles: int = 1 << 20) -> int:
    """Exercise the bounded-wait failure path (one block waits on a barrier nothing
    completes); returns the library's status, E_TIMEOUT when the path works."""
    return int(lib().spring_check_wait_timeout(int(cycles)))


def launch_count() -> int:
    return int(lib().spring_launch_count())


# ------------------------------------------------------------------ contexts, problems, runs
class Context:
    """A device context (HBM budget, serving scheduler)."""

    def __init__(self, device=0, hbm_budget_bytes=0):
        h = C.c_void_p()
        _call("spring_init", int(device), C.c_size_t(hbm_budget_bytes), C.byref(h))
        self.handle = h

    def close(self):
        if self.handle:
            _call("spring_shutdown", self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def serving_stats(self):
        """(cohorts formed, requests admitted) since the context was opened."""
        k, r = C.c_uint64(), C.c_uint64()
        _call("spring_serving_stats", self.handle, C.byref(k), C.byref(r))
        return k.value, r.value

    def problem(self, intensities, mask, support0, saturated=None, bounds=None):
        """Host numpy arrays (detector-centred I and mask, real-space support); with
        `bounds` (a Bounds) the missing moduli get the upper bounds of Eq. pm_bounds
        (`saturated`: detector-centred map of saturated pixels, optional)."""
        import numpy as np
        I = np.ascontiguousarray(intensities, dtype=np.float32)
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        s = np.ascontiguousarray(support0, dtype=np.uint8)
        h = C.c_void_p()
        if bounds is None and saturated is None:
            _call("spring_problem_create", self.handle, I.shape[0], I.shape[1],
                  I.ctypes.data_as(C.c_void_p), m.ctypes.data_as(C.c_void_p),
                  s.ctypes.data_as(C.c_void_p), C.byref(h))
        else:
            sat = None if saturated is None else np.ascontiguousarray(saturated, dtype=np.uint8)
            _call("spring_problem_create_bounded", self.handle, I.shape[0], I.shape[1],
                  I.ctypes.data_as(C.c_void_p), m.ctypes.data_as(C.c_void_p),
                  s.ctypes.data_as(C.c_void_p), None if sat is None else sat.ctypes.data_as(C.c_void_p),
                  C.byref(bounds) if bounds is not None else None, C.byref(h))
        return Problem(self, h, I.shape[0])

    def problem_device(self, I, mask, support0):
        """torch CUDA tensors (float32, uint8, uint8) on the current stream."""
        h = C.c_void_p()
        _call("spring_problem_create_device", self.handle, I.shape[0], I.shape[1], _ptr(I),
              _ptr(mask), _ptr(support0), _stream(), C.byref(h))
        return Problem(self, h, I.shape[0])

    def run_batch(self, problems, p: Params, seeds, want_arrays=True):
        """Blocking batched run of same-side problems (problem q with seeds[q]); returns
        one result dict per problem, each equal to problems[q].run with that seed."""
        import numpy as np
        K = len(problems)
        if len(seeds) != K:
            raise ValueError("one seed per problem")
        hs = (C.c_void_p * K)(*[pr.handle for pr in problems])
        sd = np.ascontiguousarray(seeds, dtype=np.uint64)
        rs = (Result * K)()
        keeps = []
        for q in range(K):
            r, keep = _result_buffers(problems[q].n if want_arrays else None, p.generations)
            rs[q] = r
            keeps.append(keep)
        _call("spring_mpr_run_batch", C.cast(hs, C.c_void_p), K, C.byref(p),
              sd.ctypes.data_as(C.c_void_p), C.cast(rs, C.c_void_p))
        return [_result_dict(rs[q], keeps[q]) for q in range(K)]

    def submit(self, problem, p: Params) -> int:
        t = C.c_uint64()
        _call("spring_submit", self.handle, problem.handle, C.byref(p), C.byref(t))
        return t.value

    def poll(self, ticket, timeout_us=0, want_arrays=True, generations=None):
        """Returns (status, result dict or None)."""
        import numpy as np
        n, G = self._sizes.get(ticket, (None, None))
        r, keep = _result_buffers(n if want_arrays else None, generations or G)
        st = lib().spring_poll(self.handle, C.c_uint64(ticket), int(timeout_us), C.byref(r))
        if st == OK:
            self._sizes.pop(ticket, None)
            return st, _result_dict(r, keep)
        if st == E_BUSY:
            return st, None
        raise SpringError(st, "spring_poll", last_error())

    def cancel(self, ticket):
        _call("spring_cancel", self.handle, C.c_uint64(ticket))

    _sizes = {}


class Problem:
    def __init__(self, ctx, handle, n):
        self.ctx, self.handle, self.n = ctx, handle, n

    def destroy(self):
        if self.handle:
            _call("spring_problem_destroy", self.handle)
            self.handle = None

    def run(self, p: Params, want_arrays=True):
        """Blocking MPR run; returns a dict with the result arrays and errors."""
        r, keep = _result_buffers(self.n if want_arrays else None, p.generations)
        _call("spring_mpr_run", self.handle, C.byref(p), C.byref(r))
        return _result_dict(r, keep)

    def run_until(self, p: Params, g_stop: int):
        """Checkpoint: Initialize and generations 1..g_stop; returns the population state."""
        import numpy as np
        P, n = p.pop, self.n
        st = {"pop_x": np.empty((P, n, n), np.complex64), "pop_S": np.empty((P, n, n), np.uint8),
              "pop_err": np.empty(P, np.float64)}
        pop = Population(0, st["pop_x"].ctypes.data, st["pop_S"].ctypes.data, st["pop_err"].ctypes.data)
        _call("spring_mpr_run_until", self.handle, C.byref(p), int(g_stop), C.byref(pop))
        st["generation"] = pop.generation
        return st

    def resume(self, p: Params, state, want_arrays=True):
        """Continue from a state returned by run_until; returns the result dict."""
        import numpy as np
        x = np.ascontiguousarray(state["pop_x"], np.complex64)
        S = np.ascontiguousarray(state["pop_S"], np.uint8)
        e = np.ascontiguousarray(state["pop_err"], np.float64)
        pop = Population(int(state["generation"]), x.ctypes.data, S.ctypes.data, e.ctypes.data)
        r, keep = _result_buffers(self.n if want_arrays else None, p.generations)
        _call("spring_mpr_resume", self.handle, C.byref(p), C.byref(pop), C.byref(r))
        return _result_dict(r, keep)

    def step(self, p: Params, state):
        """One generation from a population state (generation g - 1): returns the state after
        generation g and what it decided (spring_mpr_step)."""
        import numpy as np
        P, n = p.pop, self.n
        x = np.ascontiguousarray(state["pop_x"], np.complex64)
        S = np.ascontiguousarray(state["pop_S"], np.uint8)
        e = np.ascontiguousarray(state["pop_err"], np.float64)
        src = Population(int(state["generation"]), x.ctypes.data, S.ctypes.data, e.ctypes.data)
        out = {"pop_x": np.empty((P, n, n), np.complex64), "pop_S": np.empty((P, n, n), np.uint8),
               "pop_err": np.empty(P, np.float64)}
        dst = Population(0, out["pop_x"].ctypes.data, out["pop_S"].ctypes.data, out["pop_err"].ctypes.data)
        tr = {"err_parents": np.full(P, np.nan), "err_new": np.full(P, np.nan),
              "replaced": np.zeros(P, np.uint8), "parents": np.full((P, 3), -1, np.int32)}
        t = GenerationTrace(tr["err_parents"].ctypes.data, tr["err_new"].ctypes.data,
                            tr["replaced"].ctypes.data, tr["parents"].ctypes.data)
        _call("spring_mpr_step", self.handle, C.byref(p), C.byref(src), C.byref(dst), C.byref(t))
        out["generation"] = dst.generation
        tr["areas"] = np.array(list(t.areas), np.int64)
        tr["best"] = int(t.best)
        tr["gen_stats"] = np.array(list(t.gen_stats))
        return out, tr

    def submit(self, p: Params) -> int:
        t = self.ctx.submit(self, p)
        self.ctx._sizes[t] = (self.n, p.generations)
        return t


def _result_buffers(n, generations):
    import numpy as np
    r = Result()
    keep = {}
    if n:
        keep["rho_avg"] = np.zeros((n, n), np.complex64)
        keep["rho_best"] = np.zeros((n, n), np.complex64)
        keep["support_avg"] = np.zeros((n, n), np.uint8)
        r.rho_avg = keep["rho_avg"].ctypes.data
        r.rho_best = keep["rho_best"].ctypes.data
        r.support_avg = keep["support_avg"].ctypes.data
    if generations:
        keep["gen_stats"] = np.zeros((generations, GEN_STATS_COLS), np.float64)
        r.gen_stats = keep["gen_stats"].ctypes.data
    return r, keep


def _result_dict(r, keep):
    d = dict(keep)
    d.update(final_error_avg=r.final_error_avg, final_error_best=r.final_error_best,
             t_submit_s=r.t_submit_s, t_admit_s=r.t_admit_s, t_done_s=r.t_done_s)
    return d
