"""Thin ctypes binding of libsbse.so (C ABI in include/sbse.h), with the same function names.

Only argument marshalling happens here: every step of the computation runs in the library's CUDA
kernels. Importing works without a GPU; loading the library requires it to have been built
(`paper_2205_06690_gb300.build.build()`), and there is no fallback if it is missing.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SBSE_DEBUG_BOUNDS=1 loads the debug build (device-side index checks, see sbse_debug_bounds)
LIB_PATH = os.path.join(_HERE, "libsbse_dbg.so" if os.environ.get("SBSE_DEBUG_BOUNDS") == "1" else "libsbse.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "sbse.h")

SBSE_OK = 0
SBSE_ERR_INVALID_ARG = -1
SBSE_ERR_SHAPE = -2
SBSE_ERR_OOM = -3
SBSE_ERR_DEVICE_TIMEOUT = -4
SBSE_ERR_NOT_READY = -5
SBSE_ERR_NUMERIC = -6
SBSE_ERR_CUDA = -7
SBSE_ERR_UNSUPPORTED = -8
SBSE_FP64 = 0
SBSE_MIXED = 1
SBSE_COEFF_GAUSSIAN = 0
SBSE_COEFF_SIGN = 1
SBSE_EXCHANGE = 1
SBSE_DIRECT = 2
SBSE_DIRECT_PARTIAL = 4
SBSE_Q_OCCUPIED = 0
SBSE_Q_CONDUCTION = 1
SBSE_OPT_TENSOR_CORES = 1
SBSE_OPT_CHUNK_MB = 2
SBSE_OPT_PERSISTENT = 3
SBSE_OPT_TMA_PLANES = 4
SBSE_OPT_GRAPH = 5
SBSE_OPT_MEM_LIMIT_MB = 6
SBSE_OPT_WAIT_LIMIT = 7

_ERR_NAMES = {v: k for k, v in globals().items() if k.startswith("SBSE_ERR_")}


class SbseError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class sbse_tdh_params(C.Structure):
    _fields_ = [("n_s", C.c_int), ("n_steps", C.c_int), ("clean_every", C.c_int),
                ("dt", C.c_double), ("gamma", C.c_double), ("alpha", C.c_double),
                ("seed", C.c_uint64), ("coeff_dist", C.c_int), ("feedback", C.c_int)]


@dataclasses.dataclass
class TDHParams:
    n_s: int = 10
    n_steps: int = 200
    clean_every: int = 10
    dt: float = 0.05
    gamma: float = 0.1
    alpha: float = 1e-4
    seed: int = 0
    coeff_dist: int = SBSE_COEFF_GAUSSIAN
    feedback: int = 1

    def to_c(self) -> sbse_tdh_params:
        return sbse_tdh_params(self.n_s, self.n_steps, self.clean_every, self.dt, self.gamma,
                               self.alpha, self.seed, self.coeff_dist, int(self.feedback))


_lib = None


def load() -> C.CDLL:
    """Load libsbse.so; raise if it has not been built (there is no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2205_06690_gb300.build")
    lib = C.CDLL(LIB_PATH)
    vp, i, d, dp, ip = C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_int)
    sig = {
        "sbse_create": (i, [C.POINTER(vp), i, i]),
        "sbse_destroy": (None, [vp]),
        "sbse_set_grid": (i, [vp, i, d, dp]),
        "sbse_set_orbitals": (i, [vp, i, i, i, dp, dp, d]),
        "sbse_coefficients": (i, [C.c_uint64, i, i, i, dp]),
        "sbse_apply_W": (i, [vp, C.POINTER(sbse_tdh_params), i, ip, ip, dp, dp]),
        "sbse_build_A": (i, [vp, C.c_uint, dp]),
        "sbse_set_W": (i, [vp, i, ip, ip, dp]),
        "sbse_get_W": (i, [vp, i, ip, ip, dp]),
        "sbse_spectrum": (i, [vp, i, dp, dp]),
        "sbse_absorption": (i, [vp, i, i, d, i, dp, dp, dp]),
        "sbse_last_error": (C.c_char_p, [vp]),
        "sbse_get_stream": (i, [vp, C.POINTER(vp)]),
        "sbse_profile": (i, [vp, i]),
        "sbse_kernel_launches": (i, [C.POINTER(C.c_longlong)]),
        "sbse_set_option": (i, [vp, i, i]),
        "sbse_spectrum_noalloc": (i, [vp, i, i, vp, vp]),
        "sbse_phase_time": (i, [vp, i, dp, C.POINTER(C.c_longlong)]),
        "sbse_boundary_potential": (i, [vp, dp]),
        "sbse_fit_inverse_dielectric": (i, [i, i, dp, dp, dp]),
        "sbse_set_scissor": (i, [vp, d]),
        "sbse_localize_occupied": (i, [vp, i, d, dp]),
        "sbse_pair_weights": (i, [vp, dp]),
        "sbse_get_direct": (i, [vp, i, ip, ip, dp]),
        "sbse_set_direct": (i, [vp, dp]),
        "sbse_apply_A_mixed": (i, [vp, i, dp, dp]),
        "sbse_mixed_bounds": (i, [vp, i, i, i, dp, dp]),
        "sbse_absorption_mixed": (i, [vp, i, i, i, d, d, d, i, dp, dp, dp]),
    }
    fp = C.POINTER(C.c_float)
    sig.update({
        "sbse_fno_create": (i, [C.POINTER(vp), i, i, i, i, i, i]),
        "sbse_fno_destroy": (None, [vp]),
        "sbse_fno_last_error": (C.c_char_p, [vp]),
        "sbse_fno_num_params": (C.c_longlong, [vp]),
        "sbse_fno_set_params": (i, [vp, fp]),
        "sbse_fno_get_params": (i, [vp, fp, fp]),
        "sbse_fno_forward": (i, [vp, i, vp, vp]),
        "sbse_fno_gradients": (i, [vp, i, vp, vp]),
        "sbse_fno_train_step": (i, [vp, i, vp, vp, C.c_float, dp]),
        "sbse_fno_pair_inputs": (i, [vp, i, ip, ip, d, d, vp]),
        "sbse_surrogate_W": (i, [vp, vp, i, ip, ip, d, d, d]),
        "sbse_bare_W": (i, [vp, i, ip, ip]),
        "sbse_apply_W_range": (i, [vp, C.POINTER(sbse_tdh_params), i, ip, ip, dp, dp, i, i]),
        "sbse_debug_bounds": (i, [C.POINTER(C.c_int), C.POINTER(C.c_ulonglong)]),
        "sbse_state_bytes": (i, [vp, C.POINTER(C.c_size_t)]),
        "sbse_save_state": (i, [vp, vp, C.c_size_t]),
        "sbse_load_state": (i, [vp, vp, C.c_size_t]),
        "sbse_add_W": (i, [vp, i, ip, ip, vp, d]),
        "sbse_resample": (i, [vp, i, i, vp, i, vp]),
    })
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def header_symbols() -> list[str]:
    """Names of the functions declared in include/sbse.h."""
    with open(HEADER) as f:
        txt = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*(sbse_\w+)\s*\(", txt, re.M)))


def _dptr(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(ctx, rc):
    if rc != SBSE_OK:
        raise SbseError(rc, sbse_last_error(ctx))


def sbse_last_error(ctx) -> str:
    s = load().sbse_last_error(ctx)
    return s.decode() if s else ""


def sbse_create(device: int = 0, precision: int = SBSE_FP64):
    h = C.c_void_p()
    _check(None, load().sbse_create(C.byref(h), device, precision))
    return h


def sbse_destroy(ctx) -> None:
    load().sbse_destroy(ctx)


def sbse_set_grid(ctx, n: int, box: float, v_loc) -> None:
    v = _f64(v_loc)
    if v.size != n ** 3:
        raise ValueError("v_loc must have n^3 values")
    _check(ctx, load().sbse_set_grid(ctx, n, box, _dptr(v)))


def sbse_set_orbitals(ctx, n_occ: int, n_o: int, n_c: int, phi, eps, scissor: float) -> None:
    ph, ep = _f64(phi), _f64(eps)
    if ep.size < n_occ + n_c or ph.size % (n_occ + n_c) != 0:
        raise ValueError("phi must be (n_occ + n_c) x n^3 and eps n_occ + n_c")
    _check(ctx, load().sbse_set_orbitals(ctx, n_occ, n_o, n_c, _dptr(ph), _dptr(ep), scissor))


def sbse_coefficients(seed: int, n_s: int, n_occ: int, dist: int = SBSE_COEFF_GAUSSIAN):
    out = np.empty((n_s, n_occ))
    rc = load().sbse_coefficients(C.c_uint64(seed), n_s, n_occ, dist, _dptr(out))
    if rc != SBSE_OK:
        raise SbseError(rc, "invalid arguments")
    return out


def sbse_apply_W(ctx, params: TDHParams, pairs, coeff=None, n_g: int | None = None):
    """Run the stochastic TDH for `pairs` [(i, j), ...]; returns W (n_pairs x n_g) when n_g is given,
    else keeps the results on the device and returns None."""
    pi = np.ascontiguousarray([p[0] for p in pairs], dtype=np.int32)
    pj = np.ascontiguousarray([p[1] for p in pairs], dtype=np.int32)
    cf = None if coeff is None else _f64(coeff)
    out = None if n_g is None else np.empty((len(pairs), n_g))
    cp = params.to_c()
    ip = C.POINTER(C.c_int)
    _check(ctx, load().sbse_apply_W(ctx, C.byref(cp), len(pairs), pi.ctypes.data_as(ip),
                                    pj.ctypes.data_as(ip), _dptr(cf), _dptr(out)))
    return out


def sbse_set_W(ctx, pairs, w) -> None:
    """Store W_ij (n_pairs x n^3, host) for `pairs` [(i, j), ...]."""
    pi = np.ascontiguousarray([p[0] for p in pairs], dtype=np.int32)
    pj = np.ascontiguousarray([p[1] for p in pairs], dtype=np.int32)
    wa = _f64(w)
    ip = C.POINTER(C.c_int)
    _check(ctx, load().sbse_set_W(ctx, len(pairs), pi.ctypes.data_as(ip), pj.ctypes.data_as(ip),
                                  _dptr(wa)))


def _pairs_c(pairs):
    pi = np.ascontiguousarray([p[0] for p in pairs], dtype=np.int32)
    pj = np.ascontiguousarray([p[1] for p in pairs], dtype=np.int32)
    ip = C.POINTER(C.c_int)
    return pi, pj, pi.ctypes.data_as(ip), pj.ctypes.data_as(ip)


def sbse_get_W(ctx, pairs, n_g: int):
    pi, pj, a, b = _pairs_c(pairs)
    out = np.empty((len(pairs), n_g))
    _check(ctx, load().sbse_get_W(ctx, len(pairs), a, b, _dptr(out)))
    return out


def sbse_fno_pair_inputs(ctx, pairs, s_rho: float, s_v: float, x_ptr: int) -> None:
    pi, pj, a, b = _pairs_c(pairs)
    _check(ctx, load().sbse_fno_pair_inputs(ctx, len(pairs), a, b, s_rho, s_v, C.c_void_p(x_ptr)))


def sbse_surrogate_W(ctx, fno_handle, pairs, s_rho: float, s_v: float, s_w: float) -> None:
    pi, pj, a, b = _pairs_c(pairs)
    _check(ctx, load().sbse_surrogate_W(ctx, fno_handle, len(pairs), a, b, s_rho, s_v, s_w))


def sbse_apply_W_range(ctx, params: TDHParams, pairs, n_begin: int, n_end: int, coeff=None,
                       n_g: int | None = None):
    """Time steps [n_begin, n_end) of the propagation of `pairs` (checkpoint / resume); returns W
    when n_end == params.n_steps and n_g is given."""
    pi, pj, a, b = _pairs_c(pairs)
    cf = None if coeff is None else _f64(coeff)
    out = None if (n_g is None or n_end < params.n_steps) else np.empty((len(pairs), n_g))
    cp = params.to_c()
    _check(ctx, load().sbse_apply_W_range(ctx, C.byref(cp), len(pairs), a, b, _dptr(cf), _dptr(out),
                                          n_begin, n_end))
    return out


def sbse_debug_bounds():
    """(enabled, first_fault): whether this is the debug build, and the first out-of-range index
    recorded since the last call (0: none); reading clears the records."""
    en, f = C.c_int(), C.c_ulonglong()
    rc = load().sbse_debug_bounds(C.byref(en), C.byref(f))
    if rc not in (SBSE_OK, SBSE_ERR_NUMERIC):
        _check(None, rc)
    return bool(en.value), int(f.value)


def sbse_save_state(ctx) -> np.ndarray:
    """The propagation state held by the context, as a host byte array."""
    n = C.c_size_t()
    _check(ctx, load().sbse_state_bytes(ctx, C.byref(n)))
    buf = np.empty(n.value, dtype=np.uint8)
    _check(ctx, load().sbse_save_state(ctx, buf.ctypes.data_as(C.c_void_p), n.value))
    return buf


def sbse_load_state(ctx, buf: np.ndarray) -> None:
    a = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(ctx, load().sbse_load_state(ctx, a.ctypes.data_as(C.c_void_p), a.size))


def sbse_bare_W(ctx, pairs) -> None:
    """W_ij = q_ij = v(phi_i phi_j) for the pairs (the bare part of W)."""
    pi, pj, a, b = _pairs_c(pairs)
    _check(ctx, load().sbse_bare_W(ctx, len(pairs), a, b))


def sbse_add_W(ctx, pairs, y_ptr: int, scale: float) -> None:
    """W_ij += scale * y[k] from a device array of FP32 fields on the context's grid."""
    pi, pj, a, b = _pairs_c(pairs)
    _check(ctx, load().sbse_add_W(ctx, len(pairs), a, b, C.c_void_p(y_ptr), scale))


def sbse_resample(ctx, count: int, n_src: int, src_ptr: int, n_dst: int, dst_ptr: int) -> None:
    """Periodic trilinear resampling of device FP32 fields between grids of the same box."""
    _check(ctx, load().sbse_resample(ctx, count, n_src, C.c_void_p(src_ptr), n_dst, C.c_void_p(dst_ptr)))


def sbse_build_A(ctx, terms: int = SBSE_EXCHANGE | SBSE_DIRECT, n: int | None = None):
    """Assemble A on the device; returns it (n x n) when n = n_o * n_c is given."""
    out = None if n is None else np.empty((n, n))
    _check(ctx, load().sbse_build_A(ctx, terms, _dptr(out)))
    return out


def sbse_spectrum(ctx, k: int, n: int | None = None):
    """Lowest k excitons; given n = n_o n_c, also their eigenvectors as an (n, k) array."""
    ev = np.empty(k)
    if n is None:
        _check(ctx, load().sbse_spectrum(ctx, k, _dptr(ev), None))
        return ev
    vec = np.empty((n, k))
    _check(ctx, load().sbse_spectrum(ctx, k, _dptr(ev), _dptr(vec)))
    return ev, vec


def sbse_absorption(ctx, axis: int, n_terms: int, broadening: float, omega):
    """sigma(omega) (Sec. II.C) and the Chebyshev residues R_n; see include/sbse.h."""
    om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64).reshape(-1))
    sig = np.empty_like(om)
    res = np.empty(n_terms, dtype=np.float64)
    _check(ctx, load().sbse_absorption(ctx, axis, n_terms, float(broadening), len(om), _dptr(om),
                                       _dptr(sig), _dptr(res)))
    return sig, res


def sbse_get_stream(ctx) -> int:
    s = C.c_void_p()
    _check(ctx, load().sbse_get_stream(ctx, C.byref(s)))
    return int(s.value or 0)


def sbse_set_option(ctx, option: int, value: int) -> None:
    _check(ctx, load().sbse_set_option(ctx, option, value))


def sbse_kernel_launches() -> int:
    n = C.c_longlong()
    _check(None, load().sbse_kernel_launches(C.byref(n)))
    return n.value


def sbse_spectrum_noalloc(a_dev: int, n: int, k: int, evals_dev: int, stream: int = 0) -> None:
    """Allocation-free eigenvalues: device pointers in and out (see include/sbse.h)."""
    _check(None, load().sbse_spectrum_noalloc(C.c_void_p(a_dev), n, k, C.c_void_p(evals_dev),
                                              C.c_void_p(stream)))


def sbse_boundary_potential(ctx) -> float:
    """v_bndry of the context's system (finite-box correction, see include/sbse.h)."""
    v = C.c_double()
    _check(ctx, load().sbse_boundary_potential(ctx, C.byref(v)))
    return v.value


def sbse_fit_inverse_dielectric(E, v) -> float:
    """eps_eff^-1 from the exciton lists E (n_box x k) and boundary potentials v (n_box)."""
    Ea = _f64(np.asarray(E, dtype=np.float64))
    va = _f64(np.asarray(v, dtype=np.float64))
    s = C.c_double()
    _check(None, load().sbse_fit_inverse_dielectric(Ea.shape[0], Ea.shape[1], _dptr(Ea), _dptr(va),
                                                     C.byref(s)))
    return s.value


def sbse_localize_occupied(ctx, n_o: int, max_sweeps: int = 100, tol: float = 1e-12):
    """Rotate the occupied window to localized orbitals; returns U (n_o x n_o)."""
    U = np.empty((n_o, n_o))
    _check(ctx, load().sbse_localize_occupied(ctx, max_sweeps, tol, _dptr(U)))
    return U


def sbse_pair_weights(ctx, n_o: int):
    """Pair-density norms of the window pairs, canonical order."""
    w = np.empty(n_o * (n_o + 1) // 2)
    _check(ctx, load().sbse_pair_weights(ctx, _dptr(w)))
    return w


def sbse_get_direct(ctx, pairs, n_c: int):
    """Direct-element columns of `pairs` (n_c^2 x len(pairs)), see include/sbse.h."""
    pi = np.ascontiguousarray([p[0] for p in pairs], dtype=np.int32)
    pj = np.ascontiguousarray([p[1] for p in pairs], dtype=np.int32)
    out = np.empty((n_c * n_c, len(pairs)))
    ip = C.POINTER(C.c_int)
    _check(ctx, load().sbse_get_direct(ctx, len(pairs), pi.ctypes.data_as(ip), pj.ctypes.data_as(ip), _dptr(out)))
    return out


def sbse_set_direct(ctx, dab) -> None:
    _check(ctx, load().sbse_set_direct(ctx, _dptr(_f64(dab))))


def sbse_apply_A_mixed(ctx, projector: int, f):
    """A f in the mixed hole-grid representation (f: n_o x n^3 host array)."""
    fa = _f64(f)
    out = np.empty_like(fa)
    _check(ctx, load().sbse_apply_A_mixed(ctx, projector, _dptr(fa), _dptr(out)))
    return out


def sbse_mixed_bounds(ctx, projector: int, axis: int, n_lanczos: int):
    lo, hi = C.c_double(), C.c_double()
    _check(ctx, load().sbse_mixed_bounds(ctx, projector, axis, n_lanczos, C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


def sbse_absorption_mixed(ctx, projector: int, axis: int, n_terms: int, lo: float, hi: float, broadening: float,
                          omega):
    om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64).reshape(-1))
    sig = np.empty_like(om)
    res = np.empty(n_terms)
    _check(ctx, load().sbse_absorption_mixed(ctx, projector, axis, n_terms, float(lo), float(hi), float(broadening),
                                             len(om), _dptr(om), _dptr(sig), _dptr(res)))
    return sig, res


def sbse_set_scissor(ctx, scissor: float) -> None:
    _check(ctx, load().sbse_set_scissor(ctx, C.c_double(scissor)))


def sbse_profile(ctx, enable: bool) -> None:
    _check(ctx, load().sbse_profile(ctx, int(enable)))


def sbse_phase_time(ctx, phase: int):
    ms = C.c_double()
    n = C.c_longlong()
    _check(ctx, load().sbse_phase_time(ctx, phase, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def _fcheck(h, rc):
    if rc != SBSE_OK:
        msg = load().sbse_fno_last_error(h) if h else None
        raise SbseError(rc, (msg.decode() if msg else "") or sbse_last_error(None))


class FNO:
    """Owning wrapper of the FNO surrogate (sbse_fno_*). Tensor arguments are device pointers
    (ints, e.g. torch's data_ptr()) of FP32 arrays."""

    def __init__(self, n, width=32, modes=12, layers=4, max_batch=4, device=0):
        h = C.c_void_p()
        _fcheck(None, load().sbse_fno_create(C.byref(h), device, n, width, modes, layers, max_batch))
        self.h = h
        self.n, self.width, self.modes, self.layers, self.max_batch = n, width, modes, layers, max_batch
        self.n_params = int(load().sbse_fno_num_params(h))

    def close(self):
        if self.h:
            load().sbse_fno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        a = np.ascontiguousarray(p, dtype=np.float32)
        assert a.size == self.n_params
        _fcheck(self.h, load().sbse_fno_set_params(self.h, a.ctypes.data_as(C.POINTER(C.c_float))))

    def get_params(self):
        p = np.empty(self.n_params, np.float32)
        g = np.empty(self.n_params, np.float32)
        fp = C.POINTER(C.c_float)
        _fcheck(self.h, load().sbse_fno_get_params(self.h, p.ctypes.data_as(fp), g.ctypes.data_as(fp)))
        return p, g

    def forward(self, batch, x_ptr, y_ptr):
        _fcheck(self.h, load().sbse_fno_forward(self.h, batch, C.c_void_p(x_ptr), C.c_void_p(y_ptr)))

    def gradients(self, batch, x_ptr, dy_ptr):
        _fcheck(self.h, load().sbse_fno_gradients(self.h, batch, C.c_void_p(x_ptr), C.c_void_p(dy_ptr)))

    def train_step(self, batch, x_ptr, t_ptr, lr):
        loss = C.c_double()
        _fcheck(self.h, load().sbse_fno_train_step(self.h, batch, C.c_void_p(x_ptr), C.c_void_p(t_ptr),
                                                   C.c_float(lr), C.byref(loss)))
        return loss.value


class Context:
    """Owning wrapper: `with Context(device, precision) as c: c.set_grid(...)`."""

    def __init__(self, device: int = 0, precision: int = SBSE_FP64):
        self.h = sbse_create(device, precision)
        self.n_g = None
        self.n = None

    def close(self):
        if self.h:
            sbse_destroy(self.h)
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

    def set_grid(self, n, box, v_loc):
        sbse_set_grid(self.h, n, box, v_loc)
        self.n_g = n ** 3

    def set_orbitals(self, n_occ, n_o, n_c, phi, eps, scissor):
        sbse_set_orbitals(self.h, n_occ, n_o, n_c, phi, eps, scissor)
        self.n = n_o * n_c

    def apply_W(self, params, pairs, coeff=None, copy_out=False):
        return sbse_apply_W(self.h, params, pairs, coeff, self.n_g if copy_out else None)

    def build_A(self, terms=SBSE_EXCHANGE | SBSE_DIRECT, copy_out=True):
        return sbse_build_A(self.h, terms, self.n if copy_out else None)

    def spectrum(self, k, vectors=False):
        return sbse_spectrum(self.h, k, self.n if vectors else None)

    def absorption(self, axis, n_terms, broadening, omega):
        return sbse_absorption(self.h, axis, n_terms, broadening, omega)
