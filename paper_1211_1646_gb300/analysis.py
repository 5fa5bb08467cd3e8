"""Analysis of time series sampled from a run (host-side statistics; the
simulation itself runs in the library's kernels).

Sec. 3.3 tunes the maximum move d and the trial moves per cell n_M by the
autocorrelation time of the average orientational order parameter, measured
in wall-clock seconds.  integrated_autocorrelation_time estimates that time
from a sampled series; tune_sampling compares candidate (d, n_M) pairs by it.
"""
import math
import time

import numpy as np


def autocorrelation(x):
    """Normalised autocorrelation rho(t), t = 0 .. n-1, of a real or complex
    series (for complex x, the real part of <conj(x(s)) x(s+t)> over the
    variance), by FFT with zero padding."""
    x = np.asarray(x)
    x = x - x.mean()
    n = len(x)
    f = np.fft.fft(x, 2 * n)
    acf = np.fft.ifft(f * np.conj(f))[:n].real
    if acf[0] <= 0:
        raise ValueError("constant series")
    return acf / acf[0]


def integrated_autocorrelation_time(x, c=5.0, min_length=50.0):
    """tau = 1 + 2 sum_{t=1}^{W} rho(t), in sampling intervals, with the
    window W chosen as the smallest W >= c tau(W) (Sokal's automatic
    windowing); its relative statistical error is about sqrt(2 (2W + 1) / n).
    For an AR(1) series of coefficient a, tau = (1 + a)/(1 - a).  A series
    shorter than min_length * tau is refused (ValueError)."""
    rho = autocorrelation(x)
    tau = 2.0 * np.cumsum(rho) - 1.0
    w = np.arange(len(rho))
    ok = w >= c * tau
    if not ok.any():
        raise ValueError("series too short for its autocorrelation time")
    t = float(tau[int(np.argmax(ok))])
    if len(rho) < min_length * t:
        raise ValueError("series of %d samples is shorter than %g autocorrelation times (%.1f)"
                         % (len(rho), min_length, t))
    return t


def tune_sampling(make_system, candidates, sweeps, every, r_cut=1.4, equilibrate=0, observable=None, sync=None):
    """For each (d, n_M) in candidates: a fresh system make_system(d, n_M),
    `equilibrate` sweeps, then `sweeps` sweeps sampling an observable every
    `every` sweeps: by default the mean psi_6 of a disk system (the
    criterion of Sec. 3.3); observable(system) may give any real or complex
    number instead (e.g. for spheres).  Only the sweeps are timed (sync,
    default torch.cuda.synchronize, waits for them).  Returns a list of
    dicts (d, nselect, tau_sweeps, seconds_per_sweep, tau_seconds), sorted
    by tau_seconds (best first)."""
    if sync is None:
        import torch
        sync = torch.cuda.synchronize
    if observable is None:
        def observable(s):
            return s.psi6(r_cut)[0]
    out = []
    for d, nm in candidates:
        s = make_system(d, nm)
        if equilibrate:
            s.sweep(equilibrate)
        series = []
        sync()
        t_run = 0.0
        for _ in range(sweeps // every):
            t0 = time.perf_counter()
            s.sweep(every)
            sync()
            t_run += time.perf_counter() - t0
            series.append(observable(s))
        tau = integrated_autocorrelation_time(np.array(series)) * every
        sps = t_run / (sweeps // every * every)
        out.append({"d": d, "nselect": nm, "tau_sweeps": tau, "seconds_per_sweep": sps,
                    "tau_seconds": tau * sps})
        s.close()
    return sorted(out, key=lambda r: r["tau_seconds"])
