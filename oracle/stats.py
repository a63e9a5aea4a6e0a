"""Diagnostics of the runs (Section 3: time-averaged and RMS fields, flame surface), FP64.
Test infrastructure like the rest of the oracle.

* running statistics: mean and RMS fluctuation (population standard deviation) of a field over
  the sampled steps, straight from their definitions;
* flame length: length of the iso-line c = level of the progress variable c = (T - T_u)/(T_b - T_u)
  in 2-D, over the squares whose four corners are fluid cell centres, by marching squares:
  on each edge whose end values straddle the level (a value equal to the level counts as above)
  the crossing is placed by linear interpolation; two crossings make one segment; four (a
  saddle) make two, paired by the value at the square's centre (mean of the corners): centre
  above the level joins each crossing to the neighbouring crossing that keeps the above-level
  corners connected;
* probe spectra: Welch's estimate of the one-sided power spectral density of a sampled series
  (segments of L samples advancing by L/2, mean removed, periodic Hann window
  w_j = (1 - cos(2 pi j / L)) / 2, |DFT|^2 averaged over segments, times dt / sum w^2, doubled
  except at 0 and L/2), with numpy's FFT for the DFT.
"""
import math

import numpy as np


def running_stats(samples):
    """samples: list of arrays of equal shape. Returns (mean, rms)."""
    n = len(samples)
    mean = sum(np.asarray(s, dtype=np.float64) for s in samples) / n
    var = sum((np.asarray(s, dtype=np.float64) - mean) ** 2 for s in samples) / n
    return mean, np.sqrt(var)


def _cross(p, q, vp, vq, level):
    t = (level - vp) / (vq - vp)
    return (p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1]))


def flame_length(c, fluid, level):
    """c, fluid: arrays [ny, nx] (cell-centre values, fluid mask). Length in cell units."""
    ny, nx = c.shape
    total = 0.0
    for y in range(ny - 1):
        for x in range(nx - 1):
            if not (fluid[y, x] and fluid[y, x + 1] and fluid[y + 1, x + 1] and fluid[y + 1, x]):
                continue
            # corners counter-clockwise: (x, y), (x+1, y), (x+1, y+1), (x, y+1)
            P = [(0.0, 0.0), (1.0, 0.0), (1.0, 1.0), (0.0, 1.0)]
            V = [c[y, x], c[y, x + 1], c[y + 1, x + 1], c[y + 1, x]]
            above = [v >= level for v in V]
            pts = {}
            for e in range(4):
                a, b = e, (e + 1) % 4
                if above[a] != above[b]:
                    pts[e] = _cross(P[a], P[b], V[a], V[b], level)
            if len(pts) == 2:
                (p, q) = list(pts.values())
                total += math.hypot(p[0] - q[0], p[1] - q[1])
            elif len(pts) == 4:
                centre_above = sum(V) / 4.0 >= level
                # corner k lies between edges k-1 and k; an above-level corner is cut off from the
                # rest when the centre is below, a below-level corner when the centre is above
                cut = [k for k in range(4) if above[k] != centre_above]
                for k in cut:
                    p, q = pts[(k - 1) % 4], pts[k]
                    total += math.hypot(p[0] - q[0], p[1] - q[1])
    return total


def welch_psd(x, dt, L):
    """One-sided PSD (units^2/Hz) at the frequencies f / (L dt), f = 0 .. L/2."""
    x = np.asarray(x, dtype=np.float64)
    hop = L // 2
    nseg = (x.size - L) // hop + 1
    j = np.arange(L)
    w = 0.5 - 0.5 * np.cos(2.0 * np.pi * j / L)
    acc = np.zeros(L // 2 + 1)
    for s in range(nseg):
        seg = x[s * hop: s * hop + L]
        X = np.fft.rfft(w * (seg - seg.mean()))
        acc += np.abs(X) ** 2
    psd = acc / nseg * dt / (w * w).sum()
    psd[1:-1] *= 2.0
    return np.arange(L // 2 + 1) / (L * dt), psd
