"""GB300-native imaginary-time polarizability chi_PQ(i tau) of low-scaling GW
(arXiv 2104.09857, Eq. 2-3), computed by the CUDA library libgwchi.

`Context` wraps one library context; its methods mirror the C ABI in
include/gwchi.h (set_basis, set_3c_tensor, set_greens, chi_tau).  Device
buffers and streams come from PyTorch; all arithmetic runs in libgwchi's
kernels.
"""

from __future__ import annotations

import numpy as np

from . import _lib
from ._lib import GwError, PRECISIONS, GW_SCREEN_BOUND, GW_SCREEN_MLP


class Context:
    """One libgwchi context on a CUDA device, bound to a torch stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        self._torch = torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self.ctx = _lib.gw_create(device, stream.cuda_stream)
        self.nri = 0
        self.n_tau = 0

    def close(self) -> None:
        if getattr(self, "ctx", None):
            _lib.gw_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- inputs ---------------------------------------------------------------
    def set_basis(self, xyz, n_ao, n_ri) -> None:
        _lib.gw_set_basis(self.ctx, xyz, n_ao, n_ri)
        self.nri = int(np.sum(n_ri))

    def set_3c_tensor(self, blocks, data) -> None:
        _lib.gw_set_3c_tensor(self.ctx, blocks, data)

    def set_greens(self, C, eps, n_occ, mu_fermi, tau) -> None:
        _lib.gw_set_greens(self.ctx, C, eps, n_occ, mu_fermi, tau)
        self.n_tau = len(tau)

    def set_option(self, key: str, value: float) -> None:
        _lib.gw_set_option(self.ctx, key, value)

    def load_case(self, case) -> None:
        """Feed a synth.Case (system, 3c tensor, orbitals, tau grid)."""
        s = case.system
        self.set_basis(s.xyz, s.n_ao, s.n_ri)
        self.set_3c_tensor(case.t3c.blocks, case.t3c.data)
        self.set_greens(case.C, case.eps, case.n_occ, case.mu_fermi, case.tau)

    # -- chi ------------------------------------------------------------------
    def chi_tau(self, thr: float, precision: str = "fp64", tau_first: int = 0,
                tau_count: int | None = None, out=None, screening: int = GW_SCREEN_BOUND):
        """chi(i tau_j) for j in [tau_first, tau_first + tau_count) as a
        [tau_count, n_RI, n_RI] float64 torch tensor on the device (or into
        `out`, a device tensor or a host numpy array)."""
        torch = self._torch
        if tau_count is None:
            tau_count = self.n_tau - tau_first
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if out is None:
            out = torch.empty((tau_count, self.nri, self.nri), dtype=torch.float64,
                              device=f"cuda:{self.device}")
        if isinstance(out, np.ndarray):
            assert out.dtype == np.float64 and out.flags.c_contiguous
            assert out.size >= tau_count * self.nri * self.nri
            _lib.gw_chi_tau(self.ctx, tau_first, tau_count, thr, prec, screening,
                            out.ctypes.data, False)
        else:
            assert out.dtype == torch.float64 and out.is_contiguous() and out.is_cuda
            assert out.numel() >= tau_count * self.nri * self.nri
            _lib.gw_chi_tau(self.ctx, tau_first, tau_count, thr, prec, screening,
                            out.data_ptr(), True)
        return out

    def chi_to_w(self, chi, V, gamma, delta, out=None):
        """W^c(i tau) from chi(i tau) through the FP64 screening chain (Eqs. 7-9
        with cosine transforms).  `chi`: device tensor or host array
        [n_tau, n_RI, n_RI]; returns a device tensor unless `out` is a host array."""
        torch = self._torch
        n_tau = len(gamma[0]) if np.ndim(gamma) == 2 else 0
        shape = (n_tau, self.nri, self.nri)
        if isinstance(chi, np.ndarray):
            chi = np.ascontiguousarray(chi, dtype=np.float64)
            chi_ptr, chi_dev = chi.ctypes.data, False
        else:
            assert chi.dtype == torch.float64 and chi.is_contiguous()
            chi_ptr, chi_dev = chi.data_ptr(), True
        if out is None:
            out = torch.empty(shape, dtype=torch.float64, device=f"cuda:{self.device}")
        if isinstance(out, np.ndarray):
            _lib.gw_chi_to_w(self.ctx, V, gamma, delta, chi_ptr, chi_dev, out.ctypes.data, False)
        else:
            _lib.gw_chi_to_w(self.ctx, V, gamma, delta, chi_ptr, chi_dev, out.data_ptr(), True)
        return out

    def sigma_tau(self, w_tau, orbitals, thr: float, precision: str = "fp64"):
        """Diagonal Sigma^c_n(+-i tau) (Eq. 10): numpy [n_orb, n_tau, 2]."""
        torch = self._torch
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if isinstance(w_tau, np.ndarray):
            w = np.ascontiguousarray(w_tau, dtype=np.float64)
            return _lib.gw_sigma_tau(self.ctx, w.ctypes.data, False, orbitals, self.n_tau, thr, prec)
        assert w_tau.dtype == torch.float64 and w_tau.is_contiguous()
        return _lib.gw_sigma_tau(self.ctx, w_tau.data_ptr(), True, orbitals, self.n_tau, thr, prec)

    def stats(self) -> dict:
        return _lib.gw_get_stats(self.ctx)


__all__ = ["Context", "GwError", "PRECISIONS"]
