"""Preprocessing on the device (Sect. 2.2, Eqs. 1-3): far field, source-cube convolution, screen
smoothing.  Marshals torch tensors into the C ABI (gateau_beam_far_field / gateau_convolve_source /
gateau_smooth_screen); every step runs in libgateau_b300.so."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def beam_far_field(nu_hz, n_a: int, n_e: int, d_az: float, d_el: float, R_tel: float, t_edge_db: float, stream=None):
    """F [n_freq, n_a, n_e] (device float32), offset (q d_az, p d_el) at index (q mod n_a, p mod n_e)."""
    import torch
    nu = np.ascontiguousarray(np.asarray(nu_hz, dtype=np.float64).ravel())
    out = torch.empty((nu.size, n_a, n_e), dtype=torch.float32, device="cuda")
    L.check(L.lib().gateau_beam_far_field(nu.ctypes.data_as(L.dp), nu.size, n_a, n_e, d_az, d_el, R_tel, t_edge_db,
                                          out.data_ptr(), _stream(stream)))
    return out


def convolve_source(I, nu_hz, el0: float, d_az: float, d_el: float, R_tel: float, t_edge_db: float, stream=None):
    """P_src [n_az, n_el, n_freq] (W/Hz, device) from the specific-intensity cube I (same layout, Eq. 1)."""
    import torch
    assert I.is_cuda and I.dtype == torch.float32 and I.is_contiguous() and I.dim() == 3
    nu = np.ascontiguousarray(np.asarray(nu_hz, dtype=np.float64).ravel())
    assert nu.size == I.shape[2]
    out = torch.empty_like(I)
    L.check(L.lib().gateau_convolve_source(I.data_ptr(), I.shape[0], I.shape[1], I.shape[2], nu.ctypes.data_as(L.dp),
                                           el0, d_az, d_el, R_tel, t_edge_db, out.data_ptr(), _stream(stream)))
    return out


def smooth_screen(screen, pitch_m: float, R_tel: float, t_edge_db: float, stream=None):
    """The periodic screen [ny, nx] smoothed by the normalised aperture footprint (device)."""
    import torch
    assert screen.is_cuda and screen.dtype == torch.float32 and screen.is_contiguous() and screen.dim() == 2
    out = torch.empty_like(screen)
    L.check(L.lib().gateau_smooth_screen(screen.data_ptr(), screen.shape[1], screen.shape[0], pitch_m, R_tel, t_edge_db,
                                         out.data_ptr(), _stream(stream)))
    return out
