"""Python binding of ``libsblm.so`` (the C ABI declared in include/sblm.h and include/sblm_cnn.h).

Argument marshalling only: every step of the computation runs in the library's CUDA kernels.
Arrays may be torch tensors (CUDA or CPU) or numpy arrays; CUDA tensors are passed as device
pointers on torch's current stream, host arrays as host pointers (the library stages them).
Importing this module raises if the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsblm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
        "(the SBLM kernels have no CPU fallback)"
    )
_lib = ctypes.CDLL(LIB_PATH)

FP64, MIXED, FP32 = 0, 1, 2
NPAR = 6
MAX_NPAR = 16
MAX_WINDOW = 15
PRECISIONS = {"fp64": FP64, "mixed": MIXED, "fp32": FP32}
BLEND = 16  # OR-ed into a precision: chi^2 of the blended model with f profiled out (Section 4.4)
BLEND_F_MIN = 1e-3
STATUS = {0: "SBLM_OK", 1: "SBLM_EINVAL", 2: "SBLM_ENOMEM", 3: "SBLM_ECUDA", 4: "SBLM_ETIMEOUT", 5: "SBLM_ENUMERIC"}


class Bounds(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * NPAR), ("hi", ctypes.c_double * NPAR)]


class EAParams(ctypes.Structure):
    _fields_ = [
        ("n_pop", ctypes.c_int32),
        ("n_gen", ctypes.c_int32),
        ("p_mut0", ctypes.c_double),
        ("n_tourn", ctypes.c_int32),
        ("stag_window", ctypes.c_int32),
        ("stag_rel", ctypes.c_double),
        ("restart_after", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("polish_fev", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("n_islands", ctypes.c_int32),
        ("migration_interval", ctypes.c_int32),
        ("polish_starts", ctypes.c_int32),
        ("polish_radius", ctypes.c_double),
    ]


class EAState(ctypes.Structure):
    _fields_ = [
        ("p_mut", ctypes.c_double),
        ("best_chi2", ctypes.c_double),
        ("hist", ctypes.c_double * (MAX_WINDOW + 1)),
        ("n_hist", ctypes.c_int32),
        ("stag_run", ctypes.c_int32),
        ("n_restarts", ctypes.c_int32),
        ("generation", ctypes.c_int32),
        ("best_genes", ctypes.c_double * MAX_NPAR),
    ]


class BatchTuning(ctypes.Structure):
    _fields_ = [("group", ctypes.c_int32), ("block", ctypes.c_int32)]


class BatchMonitor(ctypes.Structure):
    _fields_ = [
        ("theta_ref", ctypes.c_void_p),
        ("f_ref", ctypes.c_void_p),
        ("chi2_max", ctypes.c_void_p),
        ("rel_tol", ctypes.c_double),
        ("first_gen", ctypes.c_void_p),
    ]


class BatchArchive(ctypes.Structure):
    _fields_ = [("size", ctypes.c_int32), ("top", ctypes.c_int32), ("radius", ctypes.c_double),
                ("theta", ctypes.c_void_p), ("chi2", ctypes.c_void_p), ("count", ctypes.c_void_p)]


class CnnTrainParams(ctypes.Structure):
    _fields_ = [
        ("batch", ctypes.c_int32),
        ("n_steps", ctypes.c_int32),
        ("warmup", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("lr", ctypes.c_double),
        ("beta1", ctypes.c_double),
        ("beta2", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("weight_decay", ctypes.c_double),
        ("forced_frac", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


_p = ctypes.c_void_p
_i32 = ctypes.c_int32
_u64 = ctypes.c_uint64
_SIGS = {
    "sblm_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "sblm_last_error": (ctypes.c_char_p, []),
    "sblm_ea_params_default": (None, [ctypes.POINTER(EAParams)]),
    "sblm_magnification": (ctypes.c_int, [_p, _i32, _p, _i32, _p, _p, _i32, _p]),
    "sblm_chi2": (ctypes.c_int, [_p, _i32, _p, _p, _p, _i32, _p, _i32, _p]),
    "sblm_chi2_genes": (ctypes.c_int, [_p, _i32, ctypes.POINTER(Bounds), _p, _p, _p, _i32, _p, _i32, _p]),
    "sblm_chi2_blend": (ctypes.c_int, [_p, _i32, _p, _p, _p, _i32, _p, _p, _i32, _p]),
    "sblm_ea_init": (ctypes.c_int, [_p, _i32, _i32, ctypes.POINTER(EAParams), _u64, _p, _p]),
    "sblm_ea_generation": (ctypes.c_int, [_p, _p, _i32, _i32, ctypes.POINTER(EAParams), _u64, _i32, _p, _p]),
    "sblm_ea_generation_noalloc": (ctypes.c_int, [_p, _p, _i32, _i32, ctypes.POINTER(EAParams), _u64, _i32, _p, _p]),
    "sblm_ea_generation_batch": (ctypes.c_int, [_p, _p, _i32, _i32, _i32, ctypes.POINTER(EAParams), _u64, _i32, _p, _p]),
    "sblm_fit": (ctypes.c_int, [_p, _p, _p, _i32, ctypes.POINTER(Bounds), ctypes.POINTER(EAParams), _p, _p, _p, _p]),
    "sblm_peak_rates": (ctypes.c_int, [_p, _p, _p]),
    "sblm_fit_batch_tuned": (
        ctypes.c_int,
        [_p, _p, _p, _p, _i32, ctypes.POINTER(Bounds), ctypes.POINTER(EAParams), ctypes.POINTER(BatchTuning), _p, _p, _p],
    ),
    "sblm_autotune_batch": (
        ctypes.c_int,
        [_p, _p, _p, _p, _i32, ctypes.POINTER(Bounds), ctypes.POINTER(EAParams), _i32, ctypes.POINTER(BatchTuning),
         ctypes.POINTER(ctypes.c_double), _p],
    ),
    "sblm_fit_batch": (
        ctypes.c_int,
        [_p, _p, _p, _p, _i32, ctypes.POINTER(Bounds), ctypes.POINTER(EAParams), _p, _p, _p],
    ),
    "sblm_fit_batch_seeded": (
        ctypes.c_int,
        [_p, _p, _p, _p, _i32, ctypes.POINTER(Bounds), ctypes.POINTER(EAParams), ctypes.POINTER(BatchTuning), _p,
         _i32, _p, _p, _p],
    ),
    "sblm_fit_batch_cnn": (
        ctypes.c_int,
        [_p, _p, _p, _p, _i32, ctypes.POINTER(Bounds), ctypes.POINTER(EAParams), ctypes.POINTER(BatchTuning), _p,
         ctypes.c_double, _p, _p, _p],
    ),
    "sblm_fit_batch_monitored": (
        ctypes.c_int,
        [_p, _p, _p, _p, _i32, ctypes.POINTER(Bounds), ctypes.POINTER(EAParams), ctypes.POINTER(BatchTuning), _p,
         ctypes.c_double, ctypes.POINTER(BatchMonitor), _p, _p, _p],
    ),
    "sblm_fit_batch_archived": (
        ctypes.c_int,
        [_p, _p, _p, _p, _i32, ctypes.POINTER(Bounds), ctypes.POINTER(EAParams), ctypes.POINTER(BatchTuning),
         ctypes.POINTER(BatchArchive), _p, _p, _p],
    ),
    "sblm_polish_batch": (
        ctypes.c_int,
        [_p, _p, _p, _p, _i32, ctypes.POINTER(Bounds), _p, _i32, _i32, _p, _p, _p],
    ),
    "sblm_cnn_train_params_default": (None, [ctypes.POINTER(CnnTrainParams)]),
    "sblm_cnn_num_params": (ctypes.c_int32, []),
    "sblm_cnn_init": (ctypes.c_int, [_p, _u64, _p]),
    "sblm_cnn_make_batch": (ctypes.c_int, [_u64, ctypes.c_int64, _i32, ctypes.c_double, _i32, _p, _p, _p, _p]),
    "sblm_cnn_bin": (ctypes.c_int, [_p, _p, _p, _p, _i32, _p, _p, _p]),
    "sblm_cnn_forward": (ctypes.c_int, [_p, _p, _i32, _p, _p]),
    "sblm_cnn_loss_grad": (ctypes.c_int, [_p, _p, _p, _i32, _p, _p, _p]),
    "sblm_cnn_adamw": (ctypes.c_int, [_p, _p, _p, ctypes.POINTER(CnnTrainParams), ctypes.c_int64, _p]),
    "sblm_cnn_train": (ctypes.c_int, [_p, _p, ctypes.POINTER(CnnTrainParams), ctypes.c_int64, _i32, _p, _p]),
    "sblm_cnn_propose": (ctypes.c_int, [_p, _p, _i32, ctypes.POINTER(Bounds), _i32, _u64, _p, _p]),
    "sblm_cnn_selftest_timeout": (ctypes.c_int, [_i32, _p]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class SBLMError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.sblm_last_error().decode()
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")


def _check(status, where):
    if status != 0:
        raise SBLMError(status, where)


def _precision(p):
    """An SBLM precision code from "fp64" / "mixed" / "fp32", optionally with "+blend" (the
    blended-model flag of the batched fitters and the polish), or an int."""
    if not isinstance(p, str):
        return int(p)
    base, _, flag = p.partition("+")
    if flag not in ("", "blend"):
        raise ValueError(f"unknown precision flag {flag!r}")
    return PRECISIONS[base] | (BLEND if flag else 0)


def _ptr(x):
    """(pointer, keep-alive) of a torch tensor or numpy array; None -> NULL."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data, x
    import torch

    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr(), x
    raise TypeError(f"unsupported array type {type(x)}")


def _stream(stream, *arrays):
    """cudaStream_t handle: the given one, else torch's current stream when any array is on the
    GPU, else the legacy default stream."""
    if stream is not None:
        return int(stream)
    try:
        import torch

        if any(isinstance(a, torch.Tensor) and a.is_cuda for a in arrays):
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def _like(ref, shape, dtype):
    """A new output array on the same side (GPU / host) as ``ref``."""
    try:
        import torch

        if isinstance(ref, torch.Tensor):
            tdt = {np.float64: torch.float64, np.float32: torch.float32, np.uint8: torch.uint8}[dtype]
            return torch.empty(shape, dtype=tdt, device=ref.device)
    except ImportError:
        pass
    return np.empty(shape, dtype=dtype)


def params(**kw):
    """An EAParams filled with the library's defaults (the paper's), then ``kw``."""
    p = EAParams()
    _lib.sblm_ea_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if k == "precision":
            v = _precision(v)
        setattr(p, k, v)
    return p


def bounds(lo, hi):
    b = Bounds()
    for j in range(NPAR):
        b.lo[j] = float(lo[j])
        b.hi[j] = float(hi[j])
    return b


def magnification(theta, t, precision="fp64", flags=False, out=None, flags_out=None, stream=None):
    """A[c, k] for parameter rows theta [n_cand, 6] at epochs t [n_ep]; optionally per-epoch flags."""
    n_cand, n_ep = int(theta.shape[0]), int(t.shape[0])
    if out is None:
        out = _like(theta, (n_cand, n_ep), np.float64)
    if flags and flags_out is None:
        flags_out = _like(theta, (n_cand, n_ep), np.uint8)
    pt, _a = _ptr(theta)
    pe, _b = _ptr(t)
    po, _c = _ptr(out)
    pf, _d = _ptr(flags_out if flags else None)
    s = _stream(stream, theta, t, out)
    _check(_lib.sblm_magnification(pt, n_cand, pe, n_ep, po, pf, _precision(precision), s), "sblm_magnification")
    return (out, flags_out) if flags else out


def chi2(theta, t, flux, sigma, precision="fp64", out=None, stream=None):
    """chi^2 of each parameter row against the lightcurve (t, flux, sigma)."""
    n_cand, n_ep = int(theta.shape[0]), int(t.shape[0])
    if out is None:
        out = _like(theta, (n_cand,), np.float64)
    args = [_ptr(a) for a in (theta, t, flux, sigma, out)]
    s = _stream(stream, theta, t, flux, sigma, out)
    st = _lib.sblm_chi2(args[0][0], n_cand, args[1][0], args[2][0], args[3][0], n_ep, args[4][0], _precision(precision), s)
    _check(st, "sblm_chi2")
    return out


def chi2_blend(theta, t, flux, sigma, precision="fp64", out=None, f_out=None, stream=None):
    """(chi^2, f) of each parameter row against the lightcurve for the blended model
    f A + (1 - f) of Section 4.4 with the blending fraction f profiled out."""
    n_cand, n_ep = int(theta.shape[0]), int(t.shape[0])
    if out is None:
        out = _like(theta, (n_cand,), np.float64)
    if f_out is None:
        f_out = _like(theta, (n_cand,), np.float64)
    args = [_ptr(a) for a in (theta, t, flux, sigma, out, f_out)]
    s = _stream(stream, theta, t, flux, sigma, out)
    st = _lib.sblm_chi2_blend(args[0][0], n_cand, args[1][0], args[2][0], args[3][0], n_ep, args[4][0], args[5][0],
                              _precision(precision), s)
    _check(st, "sblm_chi2_blend")
    return out, f_out


def chi2_genes(P, t, flux, sigma, lo, hi, precision="fp64", out=None, stream=None):
    """chi^2 of each encoded row of P [n_pop, 6] (genes in [0, 1] over the domains [lo, hi],
    gene 5 = log10 q) against the lightcurve (t, flux, sigma)."""
    n_pop, n_ep = int(P.shape[0]), int(t.shape[0])
    if out is None:
        out = _like(P, (n_pop,), np.float64)
    b = bounds(lo, hi)
    args = [_ptr(a) for a in (P, t, flux, sigma, out)]
    s = _stream(stream, P, t, flux, sigma, out)
    st = _lib.sblm_chi2_genes(args[0][0], n_pop, ctypes.byref(b), args[1][0], args[2][0], args[3][0], n_ep,
                              args[4][0], _precision(precision), s)
    _check(st, "sblm_chi2_genes")
    return out


def new_state_buffer(device=None):
    """Storage for one sblm_ea_state: a torch uint8 tensor on ``device`` or a host EAState."""
    if device is None:
        return EAState()
    import torch

    return torch.zeros(ctypes.sizeof(EAState), dtype=torch.uint8, device=device)


def _state_ptr(state):
    if isinstance(state, EAState):
        return ctypes.addressof(state), state
    return _ptr(state)


def read_state(state):
    """An EAState copy of a state held on the device (or the host struct itself)."""
    if isinstance(state, EAState):
        return state
    raw = state.detach().cpu().numpy().tobytes()
    return EAState.from_buffer_copy(raw)


def ea_init(P, n_par, p, stream_id, state, stream=None):
    n_pop = int(P.shape[0])
    pp, _a = _ptr(P)
    ps, _b = _state_ptr(state)
    s = _stream(stream, P, state)
    _check(_lib.sblm_ea_init(pp, n_pop, n_par, ctypes.byref(p), stream_id, ps, s), "sblm_ea_init")


def ea_generation(P, chi2_values, p, stream_id, generation, state, stream=None):
    """In place: P(t) -> P(t+1) given the fitness of the rows of P(t)."""
    n_pop, n_par = int(P.shape[0]), int(P.shape[1])
    pp, _a = _ptr(P)
    pc, _b = _ptr(chi2_values)
    ps, _c = _state_ptr(state)
    s = _stream(stream, P, chi2_values, state)
    st = _lib.sblm_ea_generation(pp, pc, n_pop, n_par, ctypes.byref(p), stream_id, generation, ps, s)
    _check(st, "sblm_ea_generation")


def ea_generation_batch(P, chi2_values, p, stream_id0, generation, states, stream=None):
    """In place for n_pops populations at once: P [n_pops, n_pop, n_par] (or n_pops * n_pop rows with
    p.n_pop rows each), chi2 [n_pops * n_pop], states [n_pops, state bytes] (device) or a list of
    EAState (host, updated in place)."""
    n_pop = int(p.n_pop)
    n_rows, n_par = (int(P.shape[0]) * int(P.shape[1]), int(P.shape[2])) if P.ndim == 3 else (int(P.shape[0]),
                                                                                            int(P.shape[1]))
    if n_rows % n_pop:
        raise ValueError("P must hold whole populations of p.n_pop rows")
    n_pops = n_rows // n_pop
    pp, _a = _ptr(P)
    pc, _b = _ptr(chi2_values)
    host_states = None
    if isinstance(states, (list, tuple)):
        host_states = states
        buf = (EAState * n_pops)(*states)
        ps, _c = ctypes.addressof(buf), buf
    else:
        ps, _c = _ptr(states)
    s = _stream(stream, P, chi2_values, states if host_states is None else P)
    st = _lib.sblm_ea_generation_batch(pp, pc, n_pops, n_pop, n_par, ctypes.byref(p), stream_id0, generation, ps, s)
    _check(st, "sblm_ea_generation_batch")
    if host_states is not None:
        for k in range(n_pops):
            ctypes.memmove(ctypes.addressof(host_states[k]), ctypes.addressof(buf[k]), ctypes.sizeof(EAState))


def ea_generation_noalloc(P, chi2_values, p, stream_id, generation, state, stream=None):
    """As ea_generation, for device tensors only, without any allocation (fixed scratch)."""
    n_pop, n_par = int(P.shape[0]), int(P.shape[1])
    pp, _a = _ptr(P)
    pc, _b = _ptr(chi2_values)
    ps, _c = _state_ptr(state)
    s = _stream(stream, P, chi2_values, state)
    st = _lib.sblm_ea_generation_noalloc(pp, pc, n_pop, n_par, ctypes.byref(p), stream_id, generation, ps, s)
    _check(st, "sblm_ea_generation_noalloc")


def fit(t, flux, sigma, lo, hi, p, trace=False, stream=None):
    """Best theta (t0, tE, u0, alpha, d, q) and chi^2 of one lightcurve; optionally the trace."""
    n_ep = int(t.shape[0])
    b = bounds(lo, hi)
    best = np.empty(6)
    best_chi2 = np.empty(1)
    tr = np.empty((p.n_gen, 4)) if trace else None
    a = [_ptr(x) for x in (t, flux, sigma)]
    ptr_tr, _k = _ptr(tr)
    s = _stream(stream, t, flux, sigma)
    st = _lib.sblm_fit(a[0][0], a[1][0], a[2][0], n_ep, ctypes.byref(b), ctypes.byref(p), best.ctypes.data,
                       best_chi2.ctypes.data, ptr_tr, s)
    _check(st, "sblm_fit")
    return (best, float(best_chi2[0]), tr) if trace else (best, float(best_chi2[0]))


def _tuning(tuning, t, flux, sigma, offsets, lo, hi, p, stream):
    if isinstance(tuning, str) and tuning == "auto":
        tuning = autotune_batch(t, flux, sigma, offsets, lo, hi, p, stream=stream)
    if isinstance(tuning, tuple):
        tuning = BatchTuning(*tuning)
    return tuning


def fit_batch(t, flux, sigma, offsets, lo, hi, p, tuning=None, seed_genes=None, stream=None):
    """Best theta [n_lc, 6] and chi^2 [n_lc] of lightcurves concatenated at ``offsets`` [n_lc + 1]
    (int64). ``tuning``: a BatchTuning, a (group, block) pair, "auto" (the cached autotuner result
    for this workload's shape, tuned on first use) or None (the library's defaults).
    ``seed_genes`` [n_lc, n_seed, 6]: rows that replace the last n_seed rows of each first population."""
    if seed_genes is not None:
        n_lc = int(offsets.shape[0]) - 1
        b = bounds(lo, hi)
        best = np.empty((n_lc, 6))
        best_chi2 = np.empty(n_lc)
        tuning = _tuning(tuning, t, flux, sigma, offsets, lo, hi, p, stream)
        a = [_ptr(x) for x in (t, flux, sigma, offsets, seed_genes)]
        s = _stream(stream, t, flux, sigma, seed_genes)
        tp = ctypes.byref(tuning) if tuning is not None else None
        st = _lib.sblm_fit_batch_seeded(a[0][0], a[1][0], a[2][0], a[3][0], n_lc, ctypes.byref(b), ctypes.byref(p), tp,
                                        a[4][0], int(seed_genes.shape[1]), best.ctypes.data, best_chi2.ctypes.data, s)
        _check(st, "sblm_fit_batch_seeded")
        return best, best_chi2
    n_lc = int(offsets.shape[0]) - 1
    b = bounds(lo, hi)
    best = np.empty((n_lc, 6))
    best_chi2 = np.empty(n_lc)
    if isinstance(tuning, str) and tuning == "auto":
        tuning = autotune_batch(t, flux, sigma, offsets, lo, hi, p, stream=stream)
    if isinstance(tuning, tuple):
        tuning = BatchTuning(*tuning)
    a = [_ptr(x) for x in (t, flux, sigma, offsets)]
    s = _stream(stream, t, flux, sigma)
    tp = ctypes.byref(tuning) if tuning is not None else None
    st = _lib.sblm_fit_batch_tuned(a[0][0], a[1][0], a[2][0], a[3][0], n_lc, ctypes.byref(b), ctypes.byref(p), tp,
                                   best.ctypes.data, best_chi2.ctypes.data, s)
    _check(st, "sblm_fit_batch")
    return best, best_chi2


TUNE_CACHE = os.environ.get("SBLM_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "sblm_tune.json"))


def _tune_key(offsets, p):
    import json

    off = np.asarray(offsets.cpu() if hasattr(offsets, "cpu") else offsets)
    n = np.diff(off)
    return json.dumps({"n_lc": int(n.size), "max_ep": int(2 ** np.ceil(np.log2(max(1, n.max())))),
                       "mean_ep": int(round(n.mean(), -2)), "n_pop": int(p.n_pop), "precision": int(p.precision)},
                      sort_keys=True)


def autotune_batch(t, flux, sigma, offsets, lo, hi, p, trial_generations=2, stream=None, cache=TUNE_CACHE):
    """The fastest launch shape of the batched fitter for this workload's shape (times a few
    generations of each candidate shape on the device); results persist in a JSON file."""
    import json

    key = _tune_key(offsets, p)
    table = {}
    if cache and os.path.exists(cache):
        try:
            table = json.load(open(cache))
        except (OSError, ValueError):
            table = {}
    if key in table:
        return BatchTuning(*table[key]["tuning"])
    n_lc = int(offsets.shape[0]) - 1
    b = bounds(lo, hi)
    best = BatchTuning()
    ms = ctypes.c_double()
    a = [_ptr(x) for x in (t, flux, sigma, offsets)]
    s = _stream(stream, t, flux, sigma)
    st = _lib.sblm_autotune_batch(a[0][0], a[1][0], a[2][0], a[3][0], n_lc, ctypes.byref(b), ctypes.byref(p),
                                  trial_generations, ctypes.byref(best), ctypes.byref(ms), s)
    _check(st, "sblm_autotune_batch")
    table[key] = {"tuning": [best.group, best.block], "ms": ms.value, "trial_generations": trial_generations}
    if cache:
        try:
            os.makedirs(os.path.dirname(cache), exist_ok=True)
            json.dump(table, open(cache, "w"), indent=1, sort_keys=True)
        except OSError:
            pass
    return best


def fit_batch_archived(t, flux, sigma, offsets, lo, hi, p, size=8, radius=0.05, top=0, tuning=None, stream=None):
    """fit_batch plus the solution archive (include/sblm.h: sblm_batch_archive): (best theta, chi^2,
    archive theta [n_lc, size, 6], archive chi^2 [n_lc, size], solutions kept [n_lc]); unused
    archive entries are NaN."""
    n_lc = int(offsets.shape[0]) - 1
    b = bounds(lo, hi)
    best = np.empty((n_lc, 6))
    best_chi2 = np.empty(n_lc)
    a_th = np.empty((n_lc, size, 6))
    a_c = np.empty((n_lc, size))
    a_n = np.empty(n_lc, dtype=np.int32)
    arc = BatchArchive(int(size), int(top), float(radius), a_th.ctypes.data, a_c.ctypes.data, a_n.ctypes.data)
    tuning = _tuning(tuning, t, flux, sigma, offsets, lo, hi, p, stream)
    a = [_ptr(x) for x in (t, flux, sigma, offsets)]
    s = _stream(stream, t, flux, sigma)
    tp = ctypes.byref(tuning) if tuning is not None else None
    st = _lib.sblm_fit_batch_archived(a[0][0], a[1][0], a[2][0], a[3][0], n_lc, ctypes.byref(b), ctypes.byref(p), tp,
                                      ctypes.byref(arc), best.ctypes.data, best_chi2.ctypes.data, s)
    _check(st, "sblm_fit_batch_archived")
    return best, best_chi2, a_th, a_c, a_n


def polish_batch(t, flux, sigma, offsets, lo, hi, genes, maxfev, precision="mixed", stream=None):
    """Amoeba fine-tuning of start genes [n_lc, 6]: (polished genes, chi^2)."""
    n_lc = int(offsets.shape[0]) - 1
    b = bounds(lo, hi)
    g_out = np.empty((n_lc, 6))
    c_out = np.empty(n_lc)
    a = [_ptr(x) for x in (t, flux, sigma, offsets, genes)]
    s = _stream(stream, t, flux, sigma, genes)
    st = _lib.sblm_polish_batch(a[0][0], a[1][0], a[2][0], a[3][0], n_lc, ctypes.byref(b), a[4][0], int(maxfev),
                                _precision(precision), g_out.ctypes.data, c_out.ctypes.data, s)
    _check(st, "sblm_polish_batch")
    return g_out, c_out


def fit_batch_cnn(t, flux, sigma, offsets, lo, hi, p, weights, seed_frac=0.5, tuning=None, stream=None):
    """The proposal-seeded batched fit: the network's seed rows replace round(seed_frac * n_pop)
    rows of each first population (weights None: the paper's fitter)."""
    n_lc = int(offsets.shape[0]) - 1
    b = bounds(lo, hi)
    best = np.empty((n_lc, 6))
    best_chi2 = np.empty(n_lc)
    tuning = _tuning(tuning, t, flux, sigma, offsets, lo, hi, p, stream)
    a = [_ptr(x) for x in (t, flux, sigma, offsets, weights)]
    s = _stream(stream, t, flux, sigma, weights)
    tp = ctypes.byref(tuning) if tuning is not None else None
    st = _lib.sblm_fit_batch_cnn(a[0][0], a[1][0], a[2][0], a[3][0], n_lc, ctypes.byref(b), ctypes.byref(p), tp,
                                 a[4][0], float(seed_frac), best.ctypes.data, best_chi2.ctypes.data, s)
    _check(st, "sblm_fit_batch_cnn")
    return best, best_chi2


def fit_batch_monitored(t, flux, sigma, offsets, lo, hi, p, theta_ref, chi2_max, f_ref=None, rel_tol=0.1,
                        weights=None, seed_frac=0.5, tuning=None, stream=None):
    """fit_batch_cnn plus the success monitor: (best theta, chi^2, first generation at which some
    evaluated row had chi^2 < chi2_max and every parameter within rel_tol of theta_ref, -1 if
    none) per lightcurve."""
    n_lc = int(offsets.shape[0]) - 1
    b = bounds(lo, hi)
    best = np.empty((n_lc, 6))
    best_chi2 = np.empty(n_lc)
    first = np.empty(n_lc, dtype=np.int32)

    def f64(x):  # float64 torch tensors (host or device) pass through; anything else becomes a float64 array
        if hasattr(x, "data_ptr"):
            import torch

            if x.dtype != torch.float64:
                raise TypeError("monitor arrays must be float64")
            return x.contiguous()
        return np.ascontiguousarray(x, dtype=np.float64)

    ref, cmax = _ptr(f64(theta_ref)), _ptr(f64(chi2_max))
    fr = _ptr(None if f_ref is None else f64(f_ref))
    mon = BatchMonitor(ref[0], fr[0], cmax[0], float(rel_tol), first.ctypes.data)
    tuning = _tuning(tuning, t, flux, sigma, offsets, lo, hi, p, stream)
    a = [_ptr(x) for x in (t, flux, sigma, offsets, weights)]
    s = _stream(stream, t, flux, sigma, weights)
    tp = ctypes.byref(tuning) if tuning is not None else None
    st = _lib.sblm_fit_batch_monitored(a[0][0], a[1][0], a[2][0], a[3][0], n_lc, ctypes.byref(b), ctypes.byref(p),
                                       tp, a[4][0], float(seed_frac), ctypes.byref(mon), best.ctypes.data,
                                       best_chi2.ctypes.data, s)
    _check(st, "sblm_fit_batch_monitored")
    return best, best_chi2, first


# ------------------------------------------------------------------------------------------
# learned proposal (include/sblm_cnn.h)
# ------------------------------------------------------------------------------------------
CNN_BINS = 256


def cnn_num_params():
    return int(_lib.sblm_cnn_num_params())


def cnn_train_params(**kw):
    """A CnnTrainParams with the library's defaults, then ``kw``."""
    p = CnnTrainParams()
    _lib.sblm_cnn_train_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if k == "precision":
            v = _precision(v)
        setattr(p, k, v)
    return p


def _empty(device, shape, dtype):
    if device is None:
        return np.empty(shape, dtype=dtype)
    import torch

    tdt = {np.float64: torch.float64, np.float32: torch.float32}[dtype]
    return torch.empty(shape, dtype=tdt, device=device)


def cnn_init(seed=0, device="cuda", stream=None):
    """Initial FP32 weights [N] on ``device`` (None: host numpy)."""
    w = _empty(device, (cnn_num_params(),), np.float32)
    pw, _a = _ptr(w)
    _check(_lib.sblm_cnn_init(pw, seed, _stream(stream, w)), "sblm_cnn_init")
    return w


def cnn_make_batch(seed, step, batch, forced_frac=0.1, precision="mixed", device="cuda", stream=None):
    """Training batch drawn at optimiser step ``step``: x [B, 256, 2], y [B, 6], theta [B, 6]."""
    x = _empty(device, (batch, CNN_BINS, 2), np.float32)
    y = _empty(device, (batch, 6), np.float32)
    th = _empty(device, (batch, 6), np.float64)
    px, _a = _ptr(x)
    py, _b = _ptr(y)
    pt, _c = _ptr(th)
    st = _lib.sblm_cnn_make_batch(seed, step, batch, float(forced_frac), _precision(precision), px, py, pt,
                                  _stream(stream, x))
    _check(st, "sblm_cnn_make_batch")
    return x, y, th


def cnn_bin(t, flux, sigma, offsets, stream=None):
    """Network inputs x [n_lc, 256, 2] and windows (c, h) [n_lc, 2] of concatenated lightcurves."""
    n_lc = int(offsets.shape[0]) - 1
    x = _like(t, (n_lc, CNN_BINS, 2), np.float32)
    w = _like(t, (n_lc, 2), np.float64)
    a = [_ptr(v) for v in (t, flux, sigma, offsets, x, w)]
    st = _lib.sblm_cnn_bin(a[0][0], a[1][0], a[2][0], a[3][0], n_lc, a[4][0], a[5][0], _stream(stream, t, x))
    _check(st, "sblm_cnn_bin")
    return x, w


def cnn_forward(weights, x, stream=None):
    """Network outputs [B, 12]: 6 means then 6 log-variances."""
    B = int(x.shape[0])
    out = _like(x, (B, 12), np.float32)
    a = [_ptr(v) for v in (weights, x, out)]
    _check(_lib.sblm_cnn_forward(a[0][0], a[1][0], B, a[2][0], _stream(stream, weights, x)), "sblm_cnn_forward")
    return out


def cnn_loss_grad(weights, x, y, stream=None):
    """(loss, gradient [N]) of the Gaussian NLL for the batch (x, y)."""
    B = int(x.shape[0])
    g = _like(weights, (cnn_num_params(),), np.float32)
    loss = np.empty(1)
    a = [_ptr(v) for v in (weights, x, y, g)]
    st = _lib.sblm_cnn_loss_grad(a[0][0], a[1][0], a[2][0], B, loss.ctypes.data, a[3][0],
                                 _stream(stream, weights, x))
    _check(st, "sblm_cnn_loss_grad")
    return float(loss[0]), g


def cnn_adamw(weights, state, grad, p, t, stream=None):
    """One AdamW step in place (state [2 N]: first then second moments)."""
    a = [_ptr(v) for v in (weights, state, grad)]
    st = _lib.sblm_cnn_adamw(a[0][0], a[1][0], a[2][0], ctypes.byref(p), int(t), _stream(stream, weights))
    _check(st, "sblm_cnn_adamw")


def cnn_train(weights, state, p, first_step=0, n_run=None, stream=None):
    """Steps first_step .. first_step + n_run - 1 of the schedule on the device; returns the
    per-step batch losses (numpy)."""
    n_run = p.n_steps - first_step if n_run is None else n_run
    hist = np.empty(max(0, n_run), dtype=np.float32)
    a = [_ptr(v) for v in (weights, state)]
    st = _lib.sblm_cnn_train(a[0][0], a[1][0], ctypes.byref(p), int(first_step), int(n_run), hist.ctypes.data,
                             _stream(stream, weights))
    _check(st, "sblm_cnn_train")
    return hist


def cnn_propose(out, window, lo, hi, n_seed, seed, stream=None):
    """Seed rows [n_lc, n_seed, 6] (genes) drawn from the network outputs."""
    n_lc = int(out.shape[0])
    b = bounds(lo, hi)
    g = _like(window, (n_lc, n_seed, 6), np.float64)
    a = [_ptr(v) for v in (out, window, g)]
    st = _lib.sblm_cnn_propose(a[0][0], a[1][0], n_lc, ctypes.byref(b), n_seed, seed, a[2][0],
                               _stream(stream, out, window))
    _check(st, "sblm_cnn_propose")
    return g


def cnn_selftest_timeout(polls=1000, stream=None):
    """Status (an int) of the bounded-wait self-test: SBLM_ETIMEOUT (4) when the wait on a barrier
    that nothing arrives on gave up and the flag came back through the entry points' check."""
    return int(_lib.sblm_cnn_selftest_timeout(int(polls), stream))


def peak_rates(stream=None):
    """Measured FP32 and FP64 FMA throughput of the current device, TFLOP/s."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(_lib.sblm_peak_rates(ctypes.byref(a), ctypes.byref(b), stream), "sblm_peak_rates")
    return a.value, b.value


def exported_symbols():
    """Names of the C entry points this binding declares."""
    return list(_SIGS)
