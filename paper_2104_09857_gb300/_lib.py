"""ctypes binding of libgwchi (include/gwchi.h): argument marshalling only.

Every computation happens in the CUDA library.  If the library has not been
built, or cannot be loaded, importing this module raises: there is no CPU
fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgwchi.so")

GW_OK = 0
GW_FP64, GW_FP32, GW_BF16X3, GW_BF16X6, GW_FP16X3 = 0, 1, 2, 3, 4
GW_SCREEN_BOUND, GW_SCREEN_MLP = 0, 1

ERRORS = {
    -1: "GW_ERR_INVALID_ARG",
    -2: "GW_ERR_ORDER",
    -3: "GW_ERR_ASYM",
    -4: "GW_ERR_NONFINITE",
    -5: "GW_ERR_OOM",
    -6: "GW_ERR_CUDA",
    -7: "GW_ERR_TIMEOUT",
    -8: "GW_ERR_NOT_SPD",
    -9: "GW_ERR_UNSUPPORTED",
    -10: "GW_ERR_NOT_CONVERGED",
}
GW_GRID_TIME, GW_GRID_FREQ = 0, 1
GW_GRID_MAX_N = 64

PRECISIONS = {"fp64": GW_FP64, "fp32": GW_FP32, "bf16x3": GW_BF16X3, "bf16x6": GW_BF16X6,
              "fp16x3": GW_FP16X3}


class GwError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class gw_stats(ctypes.Structure):
    _fields_ = [
        ("flops_useful", ctypes.c_double),
        ("flops_a", ctypes.c_double),
        ("flops_b", ctypes.c_double),
        ("flops_c", ctypes.c_double),
        ("flops_issued", ctypes.c_double),
        ("ms_greens", ctypes.c_double),
        ("ms_step_ab", ctypes.c_double),
        ("ms_filter", ctypes.c_double),
        ("ms_step_c", ctypes.c_double),
        ("ms_total", ctypes.c_double),
        ("ms_step_c_kernel", ctypes.c_double),
        ("c_launches", ctypes.c_longlong),
        ("tiles_total", ctypes.c_longlong),
        ("tiles_active", ctypes.c_longlong),
        ("slabs_total", ctypes.c_longlong),
        ("slabs_active", ctypes.c_longlong),
        ("kernel_launches", ctypes.c_longlong),
        ("bytes_operands", ctypes.c_double),
        ("n_batches", ctypes.c_int),
        ("tasks_seen", ctypes.c_longlong),
        ("tasks_skipped", ctypes.c_longlong),
        ("batches_skipped", ctypes.c_longlong),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class gw_tune_trial(ctypes.Structure):
    _fields_ = [
        ("knob", ctypes.c_char * 32),
        ("value", ctypes.c_double),
        ("ms", ctypes.c_double),
        ("panel_staged", ctypes.c_int),
        ("c_split_k", ctypes.c_int),
        ("batch_bytes", ctypes.c_double),
        ("mu_chunk_atoms", ctypes.c_int),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["knob"] = self.knob.decode()
        return d


_P = ctypes.c_void_p
_I = ctypes.c_int
_LL = ctypes.c_longlong
_D = ctypes.c_double

# (name, restype, argtypes) of every entry point declared in include/gwchi.h
SIGNATURES = [
    ("gw_create", _I, [ctypes.POINTER(_P), _I, _P]),
    ("gw_destroy", None, [_P]),
    ("gw_last_error", ctypes.c_char_p, [_P]),
    ("gw_set_basis", _I, [_P, _I, _P, _P, _P]),
    ("gw_set_3c_tensor", _I, [_P, _LL, _P, _P, _LL]),
    ("gw_set_greens", _I, [_P, _P, _P, _I, _D, _P, _I]),
    ("gw_chi_tau", _I, [_P, _I, _I, _D, _I, _I, _P, _I]),
    ("gw_get_stats", _I, [_P, ctypes.POINTER(gw_stats)]),
    ("gw_set_option", _I, [_P, ctypes.c_char_p, _D]),
    ("gw_chi_tau_noalloc", _I, [_P, _I, _D, _P]),
    ("gw_chi_to_w", _I, [_P, _P, _I, _P, _P, _P, _I, _P, _I]),
    ("gw_sigma_tau", _I, [_P, _P, _I, _P, _I, _D, _I, _P]),
    ("gw_qp_g0w0", _I, [_P, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    ("gw_sigma_x", _I, [_P, _P, _I, _P, _I, _D, _I, _P]),
    ("gw_ri_metric", _I, [_P, _P, _I, _P, _I, _P, _I]),
    ("gw_mlp_log", _I, [_P, _I, _I, _D, _I, _P, _P, _LL, ctypes.POINTER(_LL)]),
    ("gw_mlp_init", _I, [_P, ctypes.c_ulonglong]),
    ("gw_mlp_set_params", _I, [_P, _P, _LL]),
    ("gw_mlp_get_params", _I, [_P, _P, _LL]),
    ("gw_mlp_grad", _I, [_P, _P, _P, _LL, _P, _P]),
    ("gw_mlp_train", _I, [_P, _P, _P, _LL, _I, _LL, ctypes.c_float, ctypes.c_ulonglong, _P]),
    ("gw_mlp_predict", _I, [_P, _P, _LL, _P]),
    ("gw_minimax_grid", _I, [_I, _I, _D, _D, _P, _P, ctypes.POINTER(_D)]),
    ("gw_transform_weights", _I, [_P, _I, _P, _I, _D, _D, _P, _P, _P, _P]),
    ("gw_sigma_ao_tau", _I, [_P, _P, _I, _D, _P, _I]),
    ("gw_evgw", _I, [_P, _P, _I, _P, _P, _P, _P, _P, _I, _P, _D, _I, _I, _D, _P,
                     ctypes.POINTER(_I)]),
    ("gw_autotune", _I, [_P, _I, _D, _I, ctypes.POINTER(gw_tune_trial), _I, ctypes.POINTER(_I)]),
    ("gw_sigma_tau_batch", _I, [_P, _I, _P, _I, _P, _P, _D, _I, _P]),
]

MLP_FEATURES = 8
MLP_PARAMS = 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"libgwchi is not built ({path} missing); run "
            "`python -c 'import __graft_entry__ as g; g.build()'` on a machine with nvcc")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _check(ctx, rc: int) -> None:
    if rc != GW_OK:
        msg = lib().gw_last_error(ctx).decode() if ctx else ""
        raise GwError(rc, msg)


# ---------------------------------------------------------------------------
# thin functions with the C names
# ---------------------------------------------------------------------------

def gw_sigma_ao_tau(ctx: int, w_tau, n_tau: int, nao: int, thr: float) -> np.ndarray:
    """Sigma_{mu nu}(+-i tau) [n_tau, 2, n_ao, n_ao] (host) from a host W."""
    w = np.ascontiguousarray(w_tau, dtype=np.float64)
    out = np.zeros((n_tau, 2, nao, nao))
    _check(ctx, lib().gw_sigma_ao_tau(ctx, _ptr(w), 0, thr, _ptr(out), 0))
    return out


def gw_evgw(ctx: int, v, omega, gamma, delta, s_weights, orbitals, vxc, thr: float,
            precision: int = GW_FP64, max_cycles: int = 20, tol: float = 1e-6):
    """(energies [n_orb], cycles run) of eigenvalue-self-consistent GW for the
    listed orbitals; all inputs host arrays."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    delta = np.ascontiguousarray(delta, dtype=np.float64)
    s_weights = np.ascontiguousarray(s_weights, dtype=np.float64)
    orbitals = np.ascontiguousarray(orbitals, dtype=np.int32)
    vxc = np.ascontiguousarray(vxc, dtype=np.float64)
    out = np.zeros(len(orbitals))
    cycles = _I(0)
    _check(ctx, lib().gw_evgw(ctx, _ptr(v), len(omega), _ptr(omega), _ptr(gamma), _ptr(delta),
                              _ptr(s_weights), _ptr(orbitals), len(orbitals), _ptr(vxc), thr,
                              precision, max_cycles, tol, _ptr(out), ctypes.byref(cycles)))
    return out, cycles.value


def gw_minimax_grid(kind: int, n: int, e_min: float, e_max: float):
    """(nodes [n], weights [n], max_err) of the minimax time (GW_GRID_TIME) or
    frequency (GW_GRID_FREQ) grid for transition energies in [e_min, e_max].
    Host code: needs no context and no GPU."""
    nodes = np.zeros(max(n, 1), np.float64)
    weights = np.zeros(max(n, 1), np.float64)
    err = _D(0.0)
    rc = lib().gw_minimax_grid(int(kind), int(n), float(e_min), float(e_max), _ptr(nodes),
                               _ptr(weights), ctypes.byref(err))
    if rc != GW_OK:
        raise GwError(rc, "gw_minimax_grid")
    return nodes[:n], weights[:n], err.value


def gw_transform_weights(tau, omega, e_min: float, e_max: float):
    """(gamma [n_omega, n_tau], delta [n_tau, n_omega], s [n_omega, n_tau],
    fit errors [3]) for the grids tau and omega and transition energies in
    [e_min, e_max].  Host code: needs no context and no GPU."""
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    nt, nw = len(tau), len(omega)
    gamma = np.zeros((max(nw, 1), max(nt, 1)))
    delta = np.zeros((max(nt, 1), max(nw, 1)))
    s = np.zeros((max(nw, 1), max(nt, 1)))
    err = np.zeros(3)
    rc = lib().gw_transform_weights(_ptr(tau), nt, _ptr(omega), nw, float(e_min), float(e_max),
                                    _ptr(gamma), _ptr(delta), _ptr(s), _ptr(err))
    if rc != GW_OK:
        raise GwError(rc, "gw_transform_weights")
    return gamma, delta, s, err


def gw_create(device: int = 0, stream: int | None = None) -> int:
    out = _P()
    rc = lib().gw_create(ctypes.byref(out), device, stream or None)
    if rc != GW_OK:
        raise GwError(rc, "gw_create failed")
    return out.value


def gw_destroy(ctx: int) -> None:
    lib().gw_destroy(ctx)


def gw_set_basis(ctx: int, xyz, n_ao, n_ri) -> None:
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n_ao = np.ascontiguousarray(n_ao, dtype=np.int32)
    n_ri = np.ascontiguousarray(n_ri, dtype=np.int32)
    _check(ctx, lib().gw_set_basis(ctx, len(n_ao), _ptr(xyz), _ptr(n_ao), _ptr(n_ri)))


def gw_set_3c_tensor(ctx: int, blocks, data) -> None:
    blocks = np.ascontiguousarray(blocks, dtype=np.int32)
    data = np.ascontiguousarray(data, dtype=np.float64)
    _check(ctx, lib().gw_set_3c_tensor(ctx, blocks.shape[0], _ptr(blocks), _ptr(data), data.size))


def gw_set_greens(ctx: int, C, eps, n_occ: int, mu_fermi: float, tau) -> None:
    C = np.ascontiguousarray(C, dtype=np.float64)
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    _check(ctx, lib().gw_set_greens(ctx, _ptr(C), _ptr(eps), int(n_occ), float(mu_fermi),
                                    _ptr(tau), tau.size))


def gw_chi_tau(ctx: int, tau_first: int, tau_count: int, thr: float, precision: int,
               screening: int, out_ptr: int, out_on_device: bool) -> None:
    _check(ctx, lib().gw_chi_tau(ctx, tau_first, tau_count, float(thr), precision, screening,
                                 out_ptr, int(bool(out_on_device))))


def gw_chi_tau_noalloc(ctx: int, tau_index: int, thr: float, out_ptr: int) -> None:
    """FP64 chi for one tau point into a device buffer, with no device
    allocation inside the library (fixed work array; see include/gwchi.h)."""
    _check(ctx, lib().gw_chi_tau_noalloc(ctx, int(tau_index), float(thr), out_ptr))


def gw_chi_to_w(ctx: int, V, gamma, delta, chi_ptr: int, chi_on_device: bool, out_ptr: int,
                out_on_device: bool) -> None:
    V = np.ascontiguousarray(V, dtype=np.float64)
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    delta = np.ascontiguousarray(delta, dtype=np.float64)
    _check(ctx, lib().gw_chi_to_w(ctx, _ptr(V), gamma.shape[0], _ptr(gamma), _ptr(delta), chi_ptr,
                                  int(bool(chi_on_device)), out_ptr, int(bool(out_on_device))))


def gw_sigma_tau(ctx: int, w_ptr: int, w_on_device: bool, orbitals, n_tau: int, thr: float,
                 precision: int = GW_FP64) -> np.ndarray:
    """[n_orb, n_tau, 2]: (Sigma^c_n(i tau), Sigma^c_n(-i tau)) for the orbitals."""
    orbitals = np.ascontiguousarray(orbitals, dtype=np.int32)
    out = np.zeros((orbitals.size, n_tau, 2))
    _check(ctx, lib().gw_sigma_tau(ctx, w_ptr, int(bool(w_on_device)), _ptr(orbitals), orbitals.size,
                                   float(thr), int(precision), _ptr(out)))
    return out


def gw_ri_metric(ctx: int, s, m) -> np.ndarray:
    """S^-1 M[k] S^-1 for host matrices m [n_mat, n_ri, n_ri] (or one matrix)."""
    ss = np.ascontiguousarray(s, dtype=np.float64)
    mm = np.ascontiguousarray(m, dtype=np.float64)
    one = mm.ndim == 2
    if one:
        mm = mm[None]
    out = np.zeros_like(mm)
    _check(ctx, lib().gw_ri_metric(ctx, _ptr(ss), mm.shape[0], _ptr(mm), 0, _ptr(out), 0))
    return out[0] if one else out


def gw_sigma_x(ctx: int, v, orbitals, thr: float, precision: int = GW_FP64) -> np.ndarray:
    """Sigma^x_n (Eq. 11) [n_orb] for the orbitals; v: host [n_ri, n_ri]."""
    vv = np.ascontiguousarray(v, dtype=np.float64)
    orbitals = np.ascontiguousarray(orbitals, dtype=np.int32)
    out = np.zeros(orbitals.size)
    _check(ctx, lib().gw_sigma_x(ctx, _ptr(vv), 0, _ptr(orbitals), orbitals.size, float(thr),
                                 int(precision), _ptr(out)))
    return out


def gw_qp_g0w0(ctx: int, sigma_c, omega, gamma, s_weights, eps, vxc, sx):
    """(quasiparticle energies [n_orb], Newton iterations [n_orb]) from
    sigma_c [n_orb, n_tau, 2] (the layout of gw_sigma_tau)."""
    sig = np.ascontiguousarray(sigma_c, dtype=np.float64)
    n_orb, n_tau = sig.shape[0], sig.shape[1]
    om = np.ascontiguousarray(omega, dtype=np.float64)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    sw = np.ascontiguousarray(s_weights, dtype=np.float64)
    e, v, x = (np.ascontiguousarray(a, dtype=np.float64) for a in (eps, vxc, sx))
    out = np.zeros(n_orb)
    it = np.zeros(n_orb, dtype=np.int32)
    _check(ctx, lib().gw_qp_g0w0(ctx, n_orb, n_tau, om.size, _ptr(sig), _ptr(om), _ptr(g), _ptr(sw),
                                 _ptr(e), _ptr(v), _ptr(x), _ptr(out), _ptr(it)))
    return out, it


def gw_mlp_log(ctx: int, tau_first: int, tau_count: int, thr: float, precision: int,
               cap: int = 1 << 22):
    """(features [n, 8], log10 contribution norms [n]) of every step-C task."""
    feat = np.zeros((cap, MLP_FEATURES), dtype=np.float32)
    tgt = np.zeros(cap, dtype=np.float32)
    n = _LL(0)
    _check(ctx, lib().gw_mlp_log(ctx, tau_first, tau_count, float(thr), int(precision), _ptr(feat),
                                 _ptr(tgt), cap, ctypes.byref(n)))
    m = min(n.value, cap)
    return feat[:m].copy(), tgt[:m].copy()


def gw_mlp_init(ctx: int, seed: int) -> None:
    _check(ctx, lib().gw_mlp_init(ctx, int(seed)))


def gw_mlp_set_params(ctx: int, theta) -> None:
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    _check(ctx, lib().gw_mlp_set_params(ctx, _ptr(theta), theta.size))


def gw_mlp_get_params(ctx: int) -> np.ndarray:
    theta = np.zeros(MLP_PARAMS, dtype=np.float32)
    _check(ctx, lib().gw_mlp_get_params(ctx, _ptr(theta), theta.size))
    return theta


def gw_mlp_grad(ctx: int, feat, tgt):
    feat = np.ascontiguousarray(feat, dtype=np.float32)
    tgt = np.ascontiguousarray(tgt, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    grad = np.zeros(MLP_PARAMS, dtype=np.float32)
    _check(ctx, lib().gw_mlp_grad(ctx, _ptr(feat), _ptr(tgt), tgt.size, _ptr(loss), _ptr(grad)))
    return float(loss[0]), grad


def gw_mlp_train(ctx: int, feat, tgt, epochs: int, batch: int, lr: float, seed: int) -> np.ndarray:
    feat = np.ascontiguousarray(feat, dtype=np.float32)
    tgt = np.ascontiguousarray(tgt, dtype=np.float32)
    losses = np.zeros(max(epochs, 1), dtype=np.float32)
    _check(ctx, lib().gw_mlp_train(ctx, _ptr(feat), _ptr(tgt), tgt.size, int(epochs), int(batch),
                                   float(lr), int(seed), _ptr(losses)))
    return losses[:epochs]


def gw_mlp_predict(ctx: int, feat) -> np.ndarray:
    feat = np.ascontiguousarray(feat, dtype=np.float32)
    pred = np.zeros(feat.shape[0], dtype=np.float32)
    _check(ctx, lib().gw_mlp_predict(ctx, _ptr(feat), feat.shape[0], _ptr(pred)))
    return pred


def gw_sigma_tau_batch(ctxs: list, w_taus: list, orbitals: list, thr: float, precision: int) -> list:
    """Diagonal Sigma^c of several molecules (one context each) in one call:
    w_taus[i] host arrays [n_tau, n_RI_i, n_RI_i]; returns numpy arrays
    [n_orb_i, n_tau, 2] per molecule."""
    n = len(ctxs)
    ws = [np.ascontiguousarray(w, dtype=np.float64) for w in w_taus]
    orbs = [np.ascontiguousarray(o, dtype=np.int32) for o in orbitals]
    n_tau = ws[0].shape[0]
    outs = [np.zeros((o.size, n_tau, 2)) for o in orbs]
    c_ctx = (_P * n)(*ctxs)
    c_w = (_P * n)(*[w.ctypes.data for w in ws])
    c_o = (_P * n)(*[o.ctypes.data for o in orbs])
    c_n = (ctypes.c_int * n)(*[o.size for o in orbs])
    c_out = (_P * n)(*[o.ctypes.data for o in outs])
    _check(ctxs[0], lib().gw_sigma_tau_batch(c_ctx, n, c_w, 0, c_o, c_n, float(thr), int(precision), c_out))
    return outs


def gw_autotune(ctx: int, tau_index: int, thr: float, precision: int, max_trials: int = 64) -> list:
    """Schedule search of the tensor-core route; returns the logged trials
    (dicts), the first being the starting point; the context keeps the
    fastest setting of each knob."""
    arr = (gw_tune_trial * max_trials)()
    n = ctypes.c_int(0)
    _check(ctx, lib().gw_autotune(ctx, int(tau_index), float(thr), int(precision), arr, max_trials,
                                  ctypes.byref(n)))
    return [arr[i].as_dict() for i in range(min(n.value, max_trials))]


def gw_get_stats(ctx: int) -> dict:
    st = gw_stats()
    _check(ctx, lib().gw_get_stats(ctx, ctypes.byref(st)))
    return st.as_dict()


def gw_set_option(ctx: int, key: str, value: float) -> None:
    _check(ctx, lib().gw_set_option(ctx, key.encode(), float(value)))
