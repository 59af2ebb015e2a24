"""Spectrum from the autocorrelation function (Sec. 3.1) - oracle side.

Test infrastructure only (see the package docstring).

The absorption-type spectrum the paper shows for pyrazine is the Fourier
transform of the autocorrelation C(t) = <psi(0)|psi(t)> damped by a
phenomenological factor exp(-|t|/tau) (Sec. 3.1). Because C(-t) = conj(C(t))
the transform over the whole time axis is twice the real part of the
half-axis transform:

    I(E) = 1/(pi hbar) Re int_0^T C(t) exp(+i E t / hbar) exp(-t / tau) dt,

normalised so that a single stationary state C(t) = exp(-i E0 t/hbar) gives a
Lorentzian of unit area centred at E0 (T -> infinity). On samples
C_k = C(k dt), k = 0..N, the integral is the trapezoidal rule with end
weights 1/2. Energies in eV, times in fs.
"""
from __future__ import annotations

import numpy as np

from vibmodels import HBAR_EV_FS


def spectrum(c_t, dt_fs: float, tau_fs: float, energies_ev) -> np.ndarray:
    """I(E) for every E in energies_ev from the samples c_t[k] = C(k dt)."""
    c = np.asarray(c_t, dtype=np.complex128)
    n = c.size
    t = dt_fs * np.arange(n)
    w = np.full(n, dt_fs)
    w[0] *= 0.5
    w[-1] *= 0.5
    damp = np.exp(-t / tau_fs)
    out = np.zeros(len(energies_ev))
    for j, e in enumerate(energies_ev):
        phase = np.exp(1j * e * t / HBAR_EV_FS)
        out[j] = float(np.real(np.sum(w * c * phase * damp))) / (np.pi * HBAR_EV_FS)
    return out
