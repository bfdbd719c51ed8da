"""Helpers for the GPU tests: device buffers and the C-ABI calls by pointer."""
import ctypes

import numpy as np


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def hptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def unpack_spectrum(spec, N, M):
    """packed N x M/2 complex (as N x M doubles) -> standard half spectrum N x (M/2+1)."""
    z = spec[:, 0::2] + 1j * spec[:, 1::2]
    L = M // 2
    out = np.zeros((N, L + 1), complex)
    out[:, 1:L] = z[:, 1:L]
    Z = z[:, 0]
    Zm = np.conj(Z[(-np.arange(N)) % N])
    out[:, 0] = (Z + Zm) / 2
    out[:, L] = (Z - Zm) / 2j
    return out


def pack_spectrum(half, N, M):
    """inverse of unpack_spectrum."""
    L = M // 2
    z = half[:, :L].copy()
    z[:, 0] = half[:, 0] + 1j * half[:, L]
    out = np.empty((N, M))
    out[:, 0::2] = z.real
    out[:, 1::2] = z.imag
    return out
