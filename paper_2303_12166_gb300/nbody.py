"""ctypes binding of include/nbody.h -- argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: all work runs in libnbody.so (CUDA kernels for
sm_103a).  Importing this module fails loudly if the library has not been
built; there is no fallback.

Non-OK statuses raise :class:`NbError` (status code + nb_last_error text),
except ``nb_poll``'s NB_PENDING, which is returned.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libnbody.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libnbody.so not found at {LIB_PATH}; build it with "
        "`python -m paper_2303_12166_gb300.build` (needs nvcc, CUDA 13)")

_lib = ctypes.CDLL(LIB_PATH)

_D = ctypes.c_double
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_P = ctypes.c_void_p

NB_OK, NB_EINVAL, NB_ENOMEM, NB_EBUDGET, NB_ECUDA = 0, 1, 2, 3, 4
NB_ENONFINITE, NB_ETIMEOUT, NB_PENDING, NB_ENOTFOUND = 5, 6, 7, 8
NB_GRAVITY_ONLY, NB_NO_SPIN = 1, 2


class nb_params(ctypes.Structure):
    _fields_ = [("G", _D), ("eps", _D), ("dt", _D), ("beta", _D), ("kappa_gamma", _D),
                ("rl_coeff", _D), ("force_prec", _I32), ("flags", _U32)]


class nb_desc(ctypes.Structure):
    _fields_ = [("n_donor", _I64), ("n_accretor", _I64), ("q", _D), ("sep", _D),
                ("f_donor", _D), ("f_accretor", _D), ("expand_rate", _D),
                ("expand_steps", _I64), ("sigma_v", _D), ("seed", _U64), ("stream", _U64),
                ("xv_in", ctypes.POINTER(_D)), ("mrg_in", ctypes.POINTER(_D)), ("ecc", _D)]


class nb_diag(ctypes.Structure):
    _fields_ = [("step", _I64), ("time", _D), ("e_kin", _D), ("e_grav", _D), ("e_rep", _D),
                ("e_tot", _D), ("p", _D * 3), ("l", _D * 3), ("com", _D * 3),
                ("com_donor", _D * 3), ("com_accretor", _D * 3), ("separation", _D),
                ("r_donor", _D), ("n_past_L1", _I64), ("m_past_L1", _D),
                ("n_nonfinite", _I64), ("n_in_accretor_lobe", _I64), ("m_in_accretor_lobe", _D),
                ("n_unbound", _I64), ("m_unbound", _D)]


class nb_ckpt_meta(ctypes.Structure):
    _fields_ = [("n", _I64), ("step", _I64), ("origin", _D * 3)]


class nb_prof(ctypes.Structure):
    _fields_ = [("pair_launches", _I64), ("pair_ms", _D), ("contact_launches", _I64),
                ("contact_ms", _D), ("update_launches", _I64), ("update_ms", _D),
                ("kernels", _I64), ("pairs", _D)]


class nb_pair_cfg(ctypes.Structure):
    _fields_ = [("tile", _I32), ("i_per_thread", _I32), ("threads", _I32),
                ("min_blocks", _I32), ("nr_slots", _I32), ("i_packed", _I32),
                ("shared_rcp", _I32), ("symmetric", _I32), ("ms", _D)]


class nb_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("reserved", _I32), ("n", _I64), ("steps", _I64),
                ("t_submit", _D), ("t_start", _D), ("t_finish", _D), ("diag", nb_diag)]


class nb_server_stats(ctypes.Structure):
    _fields_ = [(k, _I64) for k in (
        "capacity_elements", "budget_bytes", "bytes_in_use", "elements_in_use",
        "requests_running", "requests_queued", "peak_requests", "peak_elements", "peak_bytes",
        "admissions_deferred", "device_bytes", "max_request_bytes")]


class nb_unit_rates(ctypes.Structure):
    _fields_ = [("sm_count", _I32), ("mufu_sqrt_per_s_sm", _D), ("mufu_rcp_per_s_sm", _D),
                ("fp32_lanes_per_s_sm", _D), ("pair_mix_evals_per_s_sm", _D)]


class nb_info(ctypes.Structure):
    _fields_ = [("n", _I64), ("n_donor", _I64), ("n_accretor", _I64), ("m_donor", _D),
                ("m_accretor", _D), ("r_donor0", _D), ("r_accretor", _D),
                ("gamma_donor", _D), ("gamma_accretor", _D), ("rl_donor", _D),
                ("rl_accretor", _D), ("x_L1", _D), ("device_bytes", _I64)]


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("nb_abi_version", ctypes.c_int, [])
_sig("nb_status_str", ctypes.c_char_p, [ctypes.c_int])
_sig("nb_last_error", ctypes.c_char_p, [])
_sig("nb_params_default", ctypes.c_int, [ctypes.POINTER(nb_params)])
_sig("nb_desc_default", ctypes.c_int, [ctypes.POINTER(nb_desc)])
_sig("nb_roche_rL", _D, [_D, _D])
_sig("nb_roche_L1", _D, [_D])
_sig("nb_preset", ctypes.c_int, [_I32, _I64, ctypes.POINTER(nb_desc), ctypes.POINTER(nb_params)])
_sig("nb_initial_state", ctypes.c_int,
     [ctypes.POINTER(nb_desc), ctypes.POINTER(nb_params), _P, _P])
_sig("nb_create_system", ctypes.c_int,
     [ctypes.POINTER(nb_desc), ctypes.POINTER(nb_params), _P, ctypes.POINTER(_P)])
_sig("nb_destroy", None, [_P])
_sig("nb_get_info", ctypes.c_int, [_P, ctypes.POINTER(nb_info)])
_sig("nb_forces", ctypes.c_int, [_P, _P, ctypes.c_int])
_sig("nb_forces_rows", ctypes.c_int, [_P, _I64, _I64, _P, ctypes.c_int])
_sig("nb_step", ctypes.c_int, [_P, _I64])
_sig("nb_sync", ctypes.c_int, [_P])
_sig("nb_diagnostics", ctypes.c_int, [_P, ctypes.POINTER(nb_diag)])
_sig("nb_get_state", ctypes.c_int, [_P, _P, _P, ctypes.POINTER(nb_ckpt_meta)])
_sig("nb_set_state", ctypes.c_int, [_P, _P, _P, ctypes.POINTER(nb_ckpt_meta)])
_sig("nb_profile", ctypes.c_int, [_P, ctypes.c_int])
_sig("nb_selftest_device_wait", ctypes.c_int, [_I64, _P])
_sig("nb_autotune", ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(nb_pair_cfg)])
_sig("nb_pair_forces_noalloc", ctypes.c_int, [_P, _I64, _D, _D, _P, _P])
_sig("nb_batch_create", ctypes.c_int,
     [ctypes.POINTER(nb_desc), ctypes.POINTER(nb_params), _I32, _P, ctypes.POINTER(_P)])
_sig("nb_batch_destroy", None, [_P])
_sig("nb_batch_info", ctypes.c_int, [_P, _I32, ctypes.POINTER(nb_info)])
_sig("nb_batch_step", ctypes.c_int, [_P, _I64])
_sig("nb_batch_sync", ctypes.c_int, [_P])
_sig("nb_batch_forces", ctypes.c_int, [_P, _I32, _P, ctypes.c_int])
_sig("nb_batch_diagnostics", ctypes.c_int, [_P, _I32, ctypes.POINTER(nb_diag)])
_sig("nb_batch_get_state", ctypes.c_int, [_P, _I32, _P, _P, ctypes.POINTER(nb_ckpt_meta)])
_sig("nb_batch_set_pair_cfg", ctypes.c_int, [_P, ctypes.POINTER(nb_pair_cfg)])
_sig("nb_batch_set_contact_lanes", ctypes.c_int, [_P, _I32])
_sig("nb_batch_get_contact_lanes", ctypes.c_int, [_P, ctypes.POINTER(_I32)])
_sig("nb_set_contact_lanes", ctypes.c_int, [_P, _I32])
_sig("nb_get_contact_lanes", ctypes.c_int, [_P, ctypes.POINTER(_I32)])
_sig("nb_batch_set_state", ctypes.c_int, [_P, _I32, _P, _P, ctypes.POINTER(nb_ckpt_meta)])
_sig("nb_batch_autotune", ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(nb_pair_cfg)])
_sig("nb_batch_profile", ctypes.c_int, [_P, ctypes.c_int])
_sig("nb_batch_profile_read", ctypes.c_int, [_P, ctypes.POINTER(nb_prof), ctypes.c_int])
_sig("nb_server_create", ctypes.c_int, [ctypes.c_size_t, _I32, _I64, _I32, _P, ctypes.POINTER(_P)])
_sig("nb_server_info", ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64),
                                      ctypes.POINTER(_I64)])
_sig("nb_submit", ctypes.c_int, [_P, ctypes.POINTER(nb_desc), ctypes.POINTER(nb_params), _I64,
                                 ctypes.POINTER(_U64)])
_sig("nb_poll", ctypes.c_int, [_P, _U64, ctypes.POINTER(nb_result)])
_sig("nb_server_drain", ctypes.c_int, [_P, _D])
_sig("nb_server_clock", _D, [_P])
_sig("nb_server_pair_cfg", ctypes.c_int, [_P, ctypes.POINTER(nb_pair_cfg)])
_sig("nb_server_stats_read", ctypes.c_int, [_P, ctypes.POINTER(nb_server_stats)])
_sig("nb_measure_unit_rates", ctypes.c_int, [ctypes.POINTER(nb_unit_rates), _P])
_sig("nb_server_destroy", None, [_P])
_sig("nb_set_pair_cfg", ctypes.c_int, [_P, ctypes.POINTER(nb_pair_cfg)])
_sig("nb_get_pair_cfg", ctypes.c_int, [_P, ctypes.POINTER(nb_pair_cfg)])
_sig("nb_pair_cfg_variants", ctypes.c_int,
     [ctypes.POINTER(nb_pair_cfg), _I32, ctypes.POINTER(_I32)])
_sig("nb_profile_read", ctypes.c_int, [_P, ctypes.POINTER(nb_prof), ctypes.c_int])


class NbError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        msg = _lib.nb_last_error().decode(errors="replace")
        name = _lib.nb_status_str(self.status).decode()
        super().__init__(f"{where}: {name} ({self.status}): {msg}")


def _check(status: int, where: str) -> int:
    if status != NB_OK:
        raise NbError(status, where)
    return status


def _stream_ptr(stream) -> int:
    """Accept None (default stream), an int handle or a torch.cuda.Stream."""
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(_D))


# ------------------------------------------------------------------ library
def nb_abi_version() -> int:
    return int(_lib.nb_abi_version())


def nb_status_str(status: int) -> str:
    return _lib.nb_status_str(int(status)).decode()


def nb_last_error() -> str:
    return _lib.nb_last_error().decode(errors="replace")


def nb_params_default(**overrides) -> nb_params:
    p = nb_params()
    _check(_lib.nb_params_default(ctypes.byref(p)), "nb_params_default")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def nb_desc_default(**overrides) -> nb_desc:
    d = nb_desc()
    _check(_lib.nb_desc_default(ctypes.byref(d)), "nb_desc_default")
    for k, v in overrides.items():
        setattr(d, k, v)
    return d


def nb_roche_rL(q: float, coeff: float = 0.69) -> float:
    return float(_lib.nb_roche_rL(float(q), float(coeff)))


def nb_roche_L1(q: float) -> float:
    return float(_lib.nb_roche_L1(float(q)))


NB_PRESET_COMPACT_ACCRETOR, NB_PRESET_TWO_MAIN_SEQUENCE, NB_PRESET_RED_GIANT = 0, 1, 2


def nb_preset(which: int, n: int):
    """(desc, params) of a scenario preset with n elements."""
    d, p = nb_desc(), nb_params()
    _check(_lib.nb_preset(int(which), int(n), ctypes.byref(d), ctypes.byref(p)), "nb_preset")
    return d, p


def nb_initial_state(desc: nb_desc, params: nb_params):
    """(xv (n,6), mrg (n,3)): the initial state a system built from (desc,
    params) starts from -- positions and velocities, and per element mass,
    initial radius and gamma.  Host only; no system is created."""
    if desc.xv_in or desc.mrg_in:
        raise ValueError("pass a descriptor without caller arrays")
    n = int(desc.n_donor) + int(desc.n_accretor)
    if n < 1:
        raise ValueError("need at least one element")
    xv = np.empty((n, 6), dtype=np.float64)
    mrg = np.empty((n, 3), dtype=np.float64)
    _check(_lib.nb_initial_state(ctypes.byref(desc), ctypes.byref(params),
                                 xv.ctypes.data_as(_P), mrg.ctypes.data_as(_P)),
           "nb_initial_state")
    return xv, mrg


def dump_state(system, path: str) -> None:
    """Headless snapshot of a System: positions/velocities, step and the FP64
    diagnostics, as a numpy .npz file."""
    xv, a, meta = system.get_state()
    d = system.diagnostics()
    np.savez(path, xv=xv, a=a, step=meta.step, origin=np.array(meta.origin[:]),
             **{f"diag_{k}": np.asarray(v) for k, v in d.items()})


def _host_rows(arr, n: int, k: int, name: str) -> np.ndarray:
    """`arr` as a flat C-contiguous float64 array of n rows of k values; the
    library reads exactly n * k doubles through the pointer, so the size is
    checked here."""
    a = np.ascontiguousarray(arr, dtype=np.float64).reshape(-1)
    if a.size != n * k:
        raise ValueError(f"{name} must hold {n} x {k} values, got {a.size}")
    return a


def _desc_n(desc: nb_desc) -> int:
    return int(desc.n_donor) + int(desc.n_accretor)


# ------------------------------------------------------------------ single system
def nb_create_system(desc: nb_desc, params: nb_params, stream=None, xv_in=None, mrg_in=None):
    """Returns an opaque handle (int).  xv_in (n,6) / mrg_in (n,3) are optional
    host arrays copied during the call."""
    # both arrays checked before the descriptor points at either
    xv = None if xv_in is None else _host_rows(xv_in, _desc_n(desc), 6, "xv_in")
    mrg = None if mrg_in is None else _host_rows(mrg_in, _desc_n(desc), 3, "mrg_in")
    h = _P()
    try:
        desc.xv_in = None if xv is None else _dptr(xv)
        desc.mrg_in = None if mrg is None else _dptr(mrg)
        _check(_lib.nb_create_system(ctypes.byref(desc), ctypes.byref(params),
                                     _P(_stream_ptr(stream)), ctypes.byref(h)),
               "nb_create_system")
    finally:
        desc.xv_in = None
        desc.mrg_in = None
    return h.value


def nb_destroy(h) -> None:
    _lib.nb_destroy(_P(h))


def nb_get_info(h) -> nb_info:
    info = nb_info()
    _check(_lib.nb_get_info(_P(h), ctypes.byref(info)), "nb_get_info")
    return info


def nb_forces(h, out=None):
    """Accelerations (n,3) FP64 at the current state.  With ``out`` a CUDA
    tensor of n*3 float64 the result is written there (device pointer);
    otherwise a new numpy array is returned."""
    n = nb_get_info(h).n
    if out is not None and hasattr(out, "data_ptr"):
        import torch
        if (out.dtype != torch.float64 or out.numel() != 3 * n or not out.is_cuda or
                not out.is_contiguous()):
            raise ValueError(f"out must be a contiguous CUDA float64 tensor of {3 * n} values")
        _check(_lib.nb_forces(_P(h), _P(out.data_ptr()), 1), "nb_forces")
        return out
    if out is not None and (out.shape != (n, 3) or out.dtype != np.float64 or
                            not out.flags.c_contiguous):
        raise ValueError("out must be a C-contiguous float64 (n, 3) array")
    a = np.empty((n, 3), dtype=np.float64) if out is None else out
    _check(_lib.nb_forces(_P(h), a.ctypes.data_as(_P), 0), "nb_forces")
    return a


def nb_forces_rows(h, lo: int, hi: int):
    """Accelerations of rows [lo, hi) only: (hi - lo, 3) float64, bit for
    bit those rows of nb_forces."""
    n = nb_get_info(h).n
    if not (0 <= lo < hi <= n):
        raise ValueError(f"rows [{lo}, {hi}) are not a range of 0 .. {n}")
    a = np.empty((hi - lo, 3), dtype=np.float64)
    _check(_lib.nb_forces_rows(_P(h), int(lo), int(hi), a.ctypes.data_as(_P), 0),
           "nb_forces_rows")
    return a


def nb_step(h, nsteps: int) -> None:
    _check(_lib.nb_step(_P(h), int(nsteps)), "nb_step")


def nb_sync(h) -> None:
    _check(_lib.nb_sync(_P(h)), "nb_sync")


def _diag_dict(d: nb_diag) -> dict:
    out = {}
    for name, _ in nb_diag._fields_:
        v = getattr(d, name)
        out[name] = np.array(v[:]) if isinstance(v, ctypes.Array) else v
    return out


def nb_diagnostics(h) -> dict:
    d = nb_diag()
    _check(_lib.nb_diagnostics(_P(h), ctypes.byref(d)), "nb_diagnostics")
    return _diag_dict(d)


def nb_get_state(h, with_acc: bool = True, out=None):
    """Returns (xv (n,6), a (n,3) or None, meta).  ``out`` = (xv, a): caller
    arrays (C-contiguous float64, e.g. views of page-locked memory) to fill
    instead of new ones."""
    n = nb_get_info(h).n
    if out is not None:
        xv, a = out
        if xv.shape != (n, 6) or xv.dtype != np.float64 or not xv.flags.c_contiguous:
            raise ValueError("out xv must be a C-contiguous float64 (n, 6) array")
        if a is not None and (a.shape != (n, 3) or a.dtype != np.float64 or
                              not a.flags.c_contiguous):
            raise ValueError("out a must be a C-contiguous float64 (n, 3) array")
    else:
        xv = np.empty((n, 6), dtype=np.float64)
        a = np.empty((n, 3), dtype=np.float64) if with_acc else None
    meta = nb_ckpt_meta()
    _check(_lib.nb_get_state(_P(h), xv.ctypes.data_as(_P),
                             a.ctypes.data_as(_P) if a is not None else None,
                             ctypes.byref(meta)), "nb_get_state")
    return xv, a, meta


def nb_set_state(h, xv, a, meta: nb_ckpt_meta) -> None:
    n = nb_get_info(h).n
    xv = _host_rows(xv, n, 6, "xv")
    a = None if a is None else _host_rows(a, n, 3, "a")
    _check(_lib.nb_set_state(_P(h), xv.ctypes.data_as(_P),
                             a.ctypes.data_as(_P) if a is not None else None,
                             ctypes.byref(meta)), "nb_set_state")


def _cfg_dict(c: nb_pair_cfg) -> dict:
    return {name: getattr(c, name) for name, _ in nb_pair_cfg._fields_}


def nb_autotune(h, reps: int = 3) -> dict:
    c = nb_pair_cfg()
    _check(_lib.nb_autotune(_P(h), int(reps), ctypes.byref(c)), "nb_autotune")
    return _cfg_dict(c)


def nb_set_pair_cfg(h, tile: int, i_per_thread: int, threads: int, min_blocks: int,
                    nr_slots: int = 0, i_packed: int = 0, shared_rcp: int = 0,
                    symmetric: int = 0) -> None:
    c = nb_pair_cfg(tile, i_per_thread, threads, min_blocks, nr_slots, i_packed, shared_rcp,
                    symmetric, 0.0)
    _check(_lib.nb_set_pair_cfg(_P(h), ctypes.byref(c)), "nb_set_pair_cfg")


def nb_get_pair_cfg(h) -> dict:
    c = nb_pair_cfg()
    _check(_lib.nb_get_pair_cfg(_P(h), ctypes.byref(c)), "nb_get_pair_cfg")
    return _cfg_dict(c)


def nb_set_contact_lanes(h, lanes: int) -> None:
    _check(_lib.nb_set_contact_lanes(_P(h), int(lanes)), "nb_set_contact_lanes")


def nb_get_contact_lanes(h) -> int:
    v = _I32()
    _check(_lib.nb_get_contact_lanes(_P(h), ctypes.byref(v)), "nb_get_contact_lanes")
    return v.value


def nb_measure_unit_rates(stream=None) -> dict:
    """MUFU and FP32 issue rates per SM per second on the current device."""
    r = nb_unit_rates()
    _check(_lib.nb_measure_unit_rates(ctypes.byref(r), _stream_ptr(stream)),
           "nb_measure_unit_rates")
    return {name: getattr(r, name) for name, _ in nb_unit_rates._fields_}


PAIR_CFG_FIELDS = ("tile", "i_per_thread", "threads", "min_blocks", "nr_slots", "i_packed",
                   "shared_rcp", "symmetric")


def nb_pair_cfg_variants() -> list:
    """Every built pair-kernel variant as a tuple in PAIR_CFG_FIELDS order."""
    count = _I32(0)
    _check(_lib.nb_pair_cfg_variants(None, 0, ctypes.byref(count)), "nb_pair_cfg_variants")
    arr = (nb_pair_cfg * max(count.value, 1))()
    _check(_lib.nb_pair_cfg_variants(arr, count.value, ctypes.byref(count)),
           "nb_pair_cfg_variants")
    return [tuple(getattr(arr[i], f) for f in PAIR_CFG_FIELDS) for i in range(count.value)]


NB_NOALLOC_MAX_N = 16384


def nb_pair_forces_noalloc(xyzm_ptr: int, n: int, G: float, eps: float, acc_ptr: int,
                           stream=None) -> None:
    """Pair term of Eq. 4 into caller-owned device memory, without any
    allocation by the library (see include/nbody.h).  Pointers are device
    addresses (e.g. tensor.data_ptr()): xyzm n x 4 doubles, acc n x 3."""
    _check(_lib.nb_pair_forces_noalloc(_P(xyzm_ptr), int(n), float(G), float(eps),
                                       _P(acc_ptr), _P(_stream_ptr(stream))),
           "nb_pair_forces_noalloc")


def nb_selftest_device_wait(budget_clocks: int, stream=None) -> int:
    """Returns the status (NB_ETIMEOUT expected); does not raise."""
    return int(_lib.nb_selftest_device_wait(int(budget_clocks), _P(_stream_ptr(stream))))


def nb_profile(h, enable: bool) -> None:
    _check(_lib.nb_profile(_P(h), 1 if enable else 0), "nb_profile")


def nb_profile_read(h, reset: bool = False) -> dict:
    p = nb_prof()
    _check(_lib.nb_profile_read(_P(h), ctypes.byref(p), 1 if reset else 0), "nb_profile_read")
    return {name: getattr(p, name) for name, _ in nb_prof._fields_}


# ------------------------------------------------------------------ batches
def nb_batch_create(descs, params, stream=None):
    """descs/params: sequences of nb_desc / nb_params (same length)."""
    n = len(descs)
    if n != len(params) or n < 1:
        raise ValueError("need as many params as descs, at least one")
    da = (nb_desc * n)(*descs)
    pa = (nb_params * n)(*params)
    h = _P()
    _check(_lib.nb_batch_create(da, pa, n, _P(_stream_ptr(stream)), ctypes.byref(h)),
           "nb_batch_create")
    return h.value


def nb_batch_destroy(h) -> None:
    _lib.nb_batch_destroy(_P(h))


def nb_batch_info(h, sys: int) -> nb_info:
    info = nb_info()
    _check(_lib.nb_batch_info(_P(h), int(sys), ctypes.byref(info)), "nb_batch_info")
    return info


def nb_batch_step(h, nsteps: int) -> None:
    _check(_lib.nb_batch_step(_P(h), int(nsteps)), "nb_batch_step")


def nb_batch_sync(h) -> None:
    _check(_lib.nb_batch_sync(_P(h)), "nb_batch_sync")


def nb_batch_forces(h, sys: int):
    n = nb_batch_info(h, sys).n
    a = np.empty((n, 3), dtype=np.float64)
    _check(_lib.nb_batch_forces(_P(h), int(sys), a.ctypes.data_as(_P), 0), "nb_batch_forces")
    return a


def nb_batch_diagnostics(h, sys: int) -> dict:
    d = nb_diag()
    _check(_lib.nb_batch_diagnostics(_P(h), int(sys), ctypes.byref(d)), "nb_batch_diagnostics")
    return _diag_dict(d)


def nb_batch_get_state(h, sys: int, with_acc: bool = True):
    n = nb_batch_info(h, sys).n
    xv = np.empty((n, 6), dtype=np.float64)
    a = np.empty((n, 3), dtype=np.float64) if with_acc else None
    meta = nb_ckpt_meta()
    _check(_lib.nb_batch_get_state(_P(h), int(sys), xv.ctypes.data_as(_P),
                                   a.ctypes.data_as(_P) if a is not None else None,
                                   ctypes.byref(meta)), "nb_batch_get_state")
    return xv, a, meta


def nb_batch_set_state(h, sys: int, xv, a, meta: nb_ckpt_meta) -> None:
    n = nb_batch_info(h, sys).n
    xv = _host_rows(xv, n, 6, "xv")
    a = None if a is None else _host_rows(a, n, 3, "a")
    _check(_lib.nb_batch_set_state(_P(h), int(sys), xv.ctypes.data_as(_P),
                                   a.ctypes.data_as(_P) if a is not None else None,
                                   ctypes.byref(meta)), "nb_batch_set_state")


def nb_batch_set_pair_cfg(h, tile, i_per_thread, threads, min_blocks, nr_slots=0,
                          i_packed=0, shared_rcp=0, symmetric=0) -> None:
    c = nb_pair_cfg(tile, i_per_thread, threads, min_blocks, nr_slots, i_packed, shared_rcp,
                    symmetric, 0.0)
    _check(_lib.nb_batch_set_pair_cfg(_P(h), ctypes.byref(c)), "nb_batch_set_pair_cfg")


def nb_batch_set_contact_lanes(h, lanes: int) -> None:
    _check(_lib.nb_batch_set_contact_lanes(_P(h), int(lanes)), "nb_batch_set_contact_lanes")


def nb_batch_get_contact_lanes(h) -> int:
    v = _I32()
    _check(_lib.nb_batch_get_contact_lanes(_P(h), ctypes.byref(v)), "nb_batch_get_contact_lanes")
    return v.value


def nb_batch_autotune(h, reps: int = 2) -> dict:
    c = nb_pair_cfg()
    _check(_lib.nb_batch_autotune(_P(h), int(reps), ctypes.byref(c)), "nb_batch_autotune")
    return _cfg_dict(c)


def nb_batch_profile(h, enable: bool) -> None:
    _check(_lib.nb_batch_profile(_P(h), 1 if enable else 0), "nb_batch_profile")


def nb_batch_profile_read(h, reset: bool = False) -> dict:
    p = nb_prof()
    _check(_lib.nb_batch_profile_read(_P(h), ctypes.byref(p), 1 if reset else 0),
           "nb_batch_profile_read")
    return {name: getattr(p, name) for name, _ in nb_prof._fields_}


class Batch:
    """Owning wrapper of an nb_batch_t handle."""

    def __init__(self, descs, params, stream=None):
        self.h = nb_batch_create(descs, params, stream)
        self.nsys = len(descs)

    def info(self, s):
        return nb_batch_info(self.h, s)

    def step(self, nsteps):
        nb_batch_step(self.h, nsteps)

    def sync(self):
        nb_batch_sync(self.h)

    def forces(self, s):
        return nb_batch_forces(self.h, s)

    def diagnostics(self, s):
        return nb_batch_diagnostics(self.h, s)

    def get_state(self, s, with_acc=True):
        return nb_batch_get_state(self.h, s, with_acc)

    def set_state(self, s, xv, a, meta):
        nb_batch_set_state(self.h, s, xv, a, meta)

    def set_pair_cfg(self, *cfg):
        nb_batch_set_pair_cfg(self.h, *cfg)

    def set_contact_lanes(self, lanes):
        nb_batch_set_contact_lanes(self.h, lanes)

    def contact_lanes(self):
        return nb_batch_get_contact_lanes(self.h)

    def autotune(self, reps=2):
        return nb_batch_autotune(self.h, reps)

    def profile(self, enable=True):
        nb_batch_profile(self.h, enable)

    def profile_read(self, reset=False):
        return nb_batch_profile_read(self.h, reset)

    def close(self):
        if self.h:
            nb_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving
def nb_server_create(hbm_budget_bytes: int, max_slots: int, max_n: int, prec: int = 32,
                     stream=None):
    h = _P()
    _check(_lib.nb_server_create(int(hbm_budget_bytes), int(max_slots), int(max_n), int(prec),
                                 _P(_stream_ptr(stream)), ctypes.byref(h)), "nb_server_create")
    return h.value


def nb_server_info(h) -> dict:
    ns, sn, db = _I32(), _I64(), _I64()
    _check(_lib.nb_server_info(_P(h), ctypes.byref(ns), ctypes.byref(sn), ctypes.byref(db)),
           "nb_server_info")
    return {"nslots": ns.value, "slot_n": sn.value, "device_bytes": db.value}


def nb_server_stats_read(h) -> dict:
    st = nb_server_stats()
    _check(_lib.nb_server_stats_read(_P(h), ctypes.byref(st)), "nb_server_stats_read")
    return {name: int(getattr(st, name)) for name, _ in nb_server_stats._fields_}


def nb_server_pair_cfg(h) -> dict:
    c = nb_pair_cfg()
    _check(_lib.nb_server_pair_cfg(_P(h), ctypes.byref(c)), "nb_server_pair_cfg")
    return _cfg_dict(c)


def nb_submit(h, desc: nb_desc, params: nb_params, nsteps: int, xv_in=None, mrg_in=None) -> int:
    # both arrays checked before the descriptor points at either
    xv = None if xv_in is None else _host_rows(xv_in, _desc_n(desc), 6, "xv_in")
    mrg = None if mrg_in is None else _host_rows(mrg_in, _desc_n(desc), 3, "mrg_in")
    t = _U64()
    try:
        desc.xv_in = None if xv is None else _dptr(xv)
        desc.mrg_in = None if mrg is None else _dptr(mrg)
        _check(_lib.nb_submit(_P(h), ctypes.byref(desc), ctypes.byref(params), int(nsteps),
                              ctypes.byref(t)), "nb_submit")
    finally:
        desc.xv_in = None
        desc.mrg_in = None
    return t.value


def nb_poll(h, ticket: int):
    """Returns a dict when the run has finished, None while it is pending."""
    r = nb_result()
    st = _lib.nb_poll(_P(h), _U64(int(ticket)), ctypes.byref(r))
    if st == NB_PENDING:
        return None
    _check(st, "nb_poll")
    out = {name: getattr(r, name) for name, _ in nb_result._fields_ if name != "diag"}
    out["diag"] = _diag_dict(r.diag)
    return out


def nb_server_drain(h, timeout_s: float) -> None:
    _check(_lib.nb_server_drain(_P(h), float(timeout_s)), "nb_server_drain")


def nb_server_clock(h) -> float:
    return float(_lib.nb_server_clock(_P(h)))


def nb_server_destroy(h) -> None:
    _lib.nb_server_destroy(_P(h))


class System:
    """Owning wrapper of an nb_system_t handle."""

    def __init__(self, desc: nb_desc | None = None, params: nb_params | None = None,
                 stream=None, xv_in=None, mrg_in=None):
        self.desc = desc if desc is not None else nb_desc_default()
        self.params = params if params is not None else nb_params_default()
        self.h = nb_create_system(self.desc, self.params, stream, xv_in=xv_in, mrg_in=mrg_in)
        self.info = nb_get_info(self.h)

    @property
    def n(self) -> int:
        return int(self.info.n)

    def forces(self, out=None):
        return nb_forces(self.h, out)

    def forces_rows(self, lo: int, hi: int):
        return nb_forces_rows(self.h, lo, hi)

    def step(self, nsteps: int):
        nb_step(self.h, nsteps)

    def sync(self):
        nb_sync(self.h)

    def diagnostics(self) -> dict:
        return nb_diagnostics(self.h)

    def get_state(self, with_acc: bool = True, out=None):
        return nb_get_state(self.h, with_acc, out)

    def set_state(self, xv, a, meta):
        nb_set_state(self.h, xv, a, meta)

    def autotune(self, reps: int = 3) -> dict:
        return nb_autotune(self.h, reps)

    def set_pair_cfg(self, tile, i_per_thread, threads, min_blocks, nr_slots=0, i_packed=0,
                     shared_rcp=0, symmetric=0):
        nb_set_pair_cfg(self.h, tile, i_per_thread, threads, min_blocks, nr_slots, i_packed,
                        shared_rcp, symmetric)

    def pair_cfg(self) -> dict:
        return nb_get_pair_cfg(self.h)

    def set_contact_lanes(self, lanes: int):
        nb_set_contact_lanes(self.h, lanes)

    def contact_lanes(self) -> int:
        return nb_get_contact_lanes(self.h)

    def profile(self, enable: bool = True):
        nb_profile(self.h, enable)

    def profile_read(self, reset: bool = False) -> dict:
        return nb_profile_read(self.h, reset)

    def close(self):
        if self.h:
            nb_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
