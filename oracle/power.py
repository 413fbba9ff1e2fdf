"""Convergence power spectrum of a square flat-sky map in FP64 (test infrastructure only).

The map statistic used to compare convergence maps (Sec. 6.2 of arXiv 2405.12913 compares C_ell):
  kappa_tilde(n) = FFT2(kappa)(n) * dtheta^2,  P(ell) = <|kappa_tilde|^2>_bin / Theta^2,  Theta = M dtheta,
  ell(n) = 2 pi |n| / Theta for the signed integer frequency n = (n_x, n_y) of the full M x M transform;
  bins are log-spaced between ell_min and ell_max, left-closed; the bin of a mode is
  b = floor(nbins * ln(ell / ell_min) / ln(ell_max / ell_min) + 1e-9) and modes with b outside
  [0, nbins) (and the n = 0 mode) are dropped; the reported bin centre is the mean ell of its modes.
The 1e-9 offset places a mode that sits on a bin edge in exact arithmetic into the upper bin whatever the
rounding of the logarithm.  Subtracting the map mean only changes the dropped n = 0 mode.
"""
from __future__ import annotations

import math

import numpy as np


def kappa_power(kappa: np.ndarray, dtheta: float, nbins: int, ell_min: float | None = None,
                ell_max: float | None = None):
    m = kappa.shape[0]
    theta = m * dtheta
    if ell_min is None:
        ell_min = 2.0 * math.pi / theta
    if ell_max is None:
        ell_max = math.pi / dtheta
    kt = np.fft.fft2(np.asarray(kappa, dtype=np.float64)) * dtheta ** 2
    p = np.abs(kt) ** 2 / theta ** 2
    n = np.fft.fftfreq(m, d=1.0 / m).round()
    n2 = n[:, None] ** 2 + n[None, :] ** 2
    ell = 2.0 * math.pi * np.sqrt(n2) / theta
    with np.errstate(divide="ignore"):
        t = nbins * np.log(ell / ell_min) / math.log(ell_max / ell_min) + 1e-9
    valid = (n2 > 0) & (t >= 0) & (t < nbins)
    b = np.floor(np.where(valid, t, -1)).astype(np.int64)
    ell_c = np.zeros(nbins)
    p_b = np.zeros(nbins)
    count = np.zeros(nbins, dtype=np.int64)
    for i in range(nbins):
        sel = valid & (b == i)
        count[i] = int(sel.sum())
        if count[i]:
            ell_c[i] = ell[sel].mean()
            p_b[i] = p[sel].mean()
    return ell_c, p_b, count
