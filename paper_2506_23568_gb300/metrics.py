"""Image-quality metrics of the paper's evaluation (Sec. V-B, Table II), computed on the host
from finished images (numpy).  The paper names the metrics but not their definitions; these
are the readings:

  NRMSE   20 log10(||f - f_ref||_2 / ||f_ref||_2) over all voxels, complex.
  PSNR    -10 log10(mean |f/M - f_ref/M|^2), M = max |f_ref|, complex values (the magnitude
          variant compares |f| and |f_ref|).
  Point-spread metrics of a 1-D complex slice through a scatterer, in |f|:
    mainlobe width  the -3 dB width around the peak, linear interpolation between samples;
    PSLR            the highest sidelobe outside the first nulls (the nearest local minima of
                    |f| on either side of the peak), relative to the peak, in dB;
    ISLR            sidelobe energy over mainlobe energy (between the first nulls), in dB.
"""
from __future__ import annotations

import numpy as np


def nrmse_db(f, ref):
    f, ref = np.asarray(f, np.complex128).ravel(), np.asarray(ref, np.complex128).ravel()
    return float(20 * np.log10(np.linalg.norm(f - ref) / np.linalg.norm(ref)))


def psnr_db(f, ref, magnitude=False):
    f, ref = np.asarray(f, np.complex128).ravel(), np.asarray(ref, np.complex128).ravel()
    m = np.abs(ref).max()
    a, b = (np.abs(f) / m, np.abs(ref) / m) if magnitude else (f / m, ref / m)
    return float(-10 * np.log10(np.mean(np.abs(a - b) ** 2)))


def _first_nulls(a, k):
    """Indices of the first local minima of a on either side of index k (the ends when none)."""
    lo = k
    while lo > 0 and a[lo - 1] < a[lo]:
        lo -= 1
    hi = k
    while hi < len(a) - 1 and a[hi + 1] < a[hi]:
        hi += 1
    return lo, hi


def psf_metrics(line, spacing):
    """(mainlobe width in the units of spacing, PSLR dB, ISLR dB) of a complex 1-D slice
    through a point response sampled at `spacing`."""
    a = np.abs(np.asarray(line))
    k = int(np.argmax(a))
    peak = a[k]
    half = peak / np.sqrt(2.0)  # -3 dB

    def crossing(step):
        i = k
        while 0 <= i + step < len(a) and a[i + step] >= half:
            i += step
        j = i + step
        if not (0 <= j < len(a)):
            return float(i)
        return i + step * (a[i] - half) / (a[i] - a[j])  # linear interpolation between i and j

    width = (crossing(1) - crossing(-1)) * spacing
    lo, hi = _first_nulls(a, k)
    side = np.concatenate([a[:lo], a[hi + 1:]])
    pslr = float(20 * np.log10(side.max() / peak)) if side.size else float("-inf")
    e_main = float((a[lo:hi + 1] ** 2).sum())
    e_side = float((side ** 2).sum())
    islr = float(10 * np.log10(e_side / e_main)) if e_side > 0 else float("-inf")
    return float(width), pslr, islr
