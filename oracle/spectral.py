"""Pseudo-spectral operators on the periodic box [0, 2*pi)^d (Sec. 2.2).

Test infrastructure only (see oracle/__init__.py).

Functions u on the grid x_l = 2*pi*l/n are represented by their Fourier coefficients
(Sec. 2.2); differential operators are applied as "two FFTs and a diagonal scaling".
FFTs are numpy's (unnormalised forward, 1/n on the inverse).

Readings:
* Wavenumbers: the printed range "n_j/2+1 <= k_j <= n_j/2" is read as
  -n_j/2+1 <= k_j <= n_j/2 (the minus sign is missing in the text).
* Even-order symbols |k|^{2s} use the full k, including the Nyquist mode |k_j| = n_j/2.
* First-derivative symbols use k~_j = k_j for |k_j| < n_j/2 and 0 at the Nyquist mode,
  so that derivatives of real fields stay real; the Leray projector uses k~ too.
* Regularisation seminorm of order s (Sec. 1.1 Eq. (1a) for s=2; Sec. 3.6 uses s=3; the
  s=1 H1 seminorm is the same construction): L^ = |k|^{2s}, reg(v) = alpha/2 <v, L v>.
* Inverse with the kernel fixed (Sec. 2.2, last paragraph): the zero entries of L^ are set
  to one before inverting, so (alpha L)^{-1} acts as 1/alpha on the k = 0 mode.
"""
from __future__ import annotations

import numpy as np


def int_wavenumbers(ni):
    """Integer wavenumbers of an axis in numpy FFT order (Nyquist slot holds -ni/2)."""
    return np.fft.fftfreq(ni, d=1.0 / ni)


def wavenumber_grids(n):
    """Full-grid broadcastable wavenumber arrays k_c (Nyquist included)."""
    return np.meshgrid(*[int_wavenumbers(ni) for ni in n], indexing="ij")


def deriv_wavenumber_grids(n):
    """Derivative wavenumbers k~_c: k_c with the Nyquist mode (even n_c) set to zero."""
    out = []
    for c, kc in enumerate(wavenumber_grids(n)):
        kt = kc.copy()
        if n[c] % 2 == 0:
            kt[kc == -(n[c] // 2)] = 0.0
        out.append(kt)
    return out


def fftn(u):
    return np.fft.fftn(u)


def ifftn_real(uh):
    return np.real(np.fft.ifftn(uh))


def symbol_L(n, s):
    """L^(k) = |k|^{2s} for the H^s seminorm regulariser."""
    ks = wavenumber_grids(n)
    k2 = sum(k * k for k in ks)
    return k2 ** s


def apply_L(v, s):
    """L v componentwise: F^{-1}[|k|^{2s} F v_c]."""
    Lh = symbol_L(v.shape[1:], s)
    return np.stack([ifftn_real(Lh * fftn(vc)) for vc in v])


def apply_alphaL_inv(v, s, alpha):
    """(alpha L)^{-1} v with the zero symbol entries of L set to one (Sec. 2.2)."""
    Lh = symbol_L(v.shape[1:], s)
    Lfix = np.where(Lh == 0.0, 1.0, Lh)
    return np.stack([ifftn_real(fftn(vc) / (alpha * Lfix)) for vc in v])


def grad(f):
    """Spectral gradient (d, *n) of a scalar field f: F^{-1}[i k~_c F f]."""
    fh = fftn(f)
    return np.stack([ifftn_real(1j * kt * fh) for kt in deriv_wavenumber_grids(f.shape)])


def line_derivative(f_line):
    """Spectral derivative (grid spacing 2 pi / L) of one periodic grid line of L samples, with the
    Nyquist entry zeroed. The derivative of a field along axis a restricted to a grid line along a
    equals this line derivative: the transforms along the other axes cancel."""
    L = f_line.shape[-1]
    k = int_wavenumbers(L)
    kt = np.where(2 * np.abs(k) == L, 0.0, k)
    return np.real(np.fft.ifft(1j * kt * np.fft.fft(f_line, axis=-1), axis=-1))


def div(v):
    """Spectral divergence sum_c F^{-1}[i k~_c F v_c]."""
    kts = deriv_wavenumber_grids(v.shape[1:])
    acc = np.zeros(v.shape[1:], dtype=complex)
    for c in range(v.shape[0]):
        acc += 1j * kts[c] * fftn(v[c])
    return ifftn_real(acc)


def leray(v):
    """Leray projection P v with P^ = I - k~ k~^T / |k~|^2 (identity where k~ = 0) (Sec. 3.6)."""
    kts = deriv_wavenumber_grids(v.shape[1:])
    vh = [fftn(vc) for vc in v]
    k2 = sum(k * k for k in kts)
    kdotv = sum(k * vc for k, vc in zip(kts, vh))
    ratio = np.where(k2 > 0.0, kdotv / np.where(k2 > 0.0, k2, 1.0), 0.0)
    return np.stack([ifftn_real(vc - k * ratio) for k, vc in zip(kts, vh)])


def cell_volume(n):
    """h^d = prod_i 2*pi/n_i, the weight of the L2 quadrature on the grid."""
    return float(np.prod([2.0 * np.pi / ni for ni in n]))


def inner(a, b, n):
    """Discrete L2 inner product <a, b> = h^d * sum(a * b) over all components."""
    return cell_volume(n) * float(np.sum(a * b))
