"""Vortex-shedding validation of the solver (the supplement's "Validation of
the Fluid Simulator"): flow past a cylinder, the shedding frequency taken
from a velocity probe in the wake and compared with the empirical
Strouhal relation St = 0.198 (1 - 19.7 / Re), f = St U / D, quoted there for
250 < Re < 2.5e5.  The flow is advanced by the CUDA step (uf.Grid); this
module only samples the probe and analyses the signal."""
from __future__ import annotations

import numpy as np

NU_AIR = 1.5e-5   # kinematic viscosity of the step [m^2/s]


def strouhal_formula(U: float, D: float, nu: float = NU_AIR) -> float:
    """St = 0.198 (1 - 19.7 / Re), Re = U D / nu."""
    return 0.198 * (1.0 - 19.7 / (U * D / nu))


def dominant_frequency(signal, dt: float, pad: int = 16) -> float:
    """Frequency of the largest spectral peak of a sampled signal: linear
    trend removed, Hann window, zero-padded to `pad` times the next power of
    two, peak located by a parabola through the log-magnitudes of the
    highest bin and its two neighbours.  0 for a signal that is a straight
    line (nothing left after the trend)."""
    s = np.asarray(signal, dtype=np.float64)
    n = s.size
    if n < 4:
        return 0.0
    t = np.arange(n)
    scale = np.max(np.abs(s))
    s = s - np.polyval(np.polyfit(t, s, 1), t)
    if np.max(np.abs(s)) <= 1e-9 * (1.0 + scale):
        return 0.0
    m = pad * (1 << int(np.ceil(np.log2(n))))
    spec = np.abs(np.fft.rfft(s * np.hanning(n), m))
    k = 1 + int(np.argmax(spec[1:-1]))
    if spec[k] <= 0.0 or k < 1:
        return 0.0
    a, b, c = np.log(spec[k - 1] + 1e-300), np.log(spec[k]), np.log(spec[k + 1] + 1e-300)
    den = a - 2 * b + c
    off = 0.5 * (a - c) / den if den != 0 else 0.0
    return (k + off) / (m * dt)


def shedding_run(U: float, dt: float | None = None, cfl: float | None = None, periods: int = 12,
                 samples_per_period: int = 40, precision: str = "f32", transient_flows: float = 2.5,
                 **kw) -> dict:
    """Runs the cylinder benchmark at inflow speed U with the time step dt
    (the supplement's 1e-4 s by default) or the one of cell Courant number
    `cfl` at U; discards `transient_flows` flow-through times of the channel
    (at 20 m/s the street is still growing after 1.2 of them: its amplitude
    is a fifth below the settled one and its frequency 6 % low), then
    samples the cross-stream velocity 3 D behind the cylinder on the
    channel axis over `periods` periods of the formula's frequency.
    Returns the measured and formula frequencies and Strouhal numbers, the
    probe amplitude (and that of each half of the sample, equal once the
    street has settled) and the run's time step and step count."""
    from . import layouts, uf
    sc = layouts.karman_cylinder(U, **kw)
    if cfl is not None:
        sc.fixed_dt = cfl * sc.h / U
    elif dt is not None:
        sc.fixed_dt = dt
    step = sc.fixed_dt
    g = uf.Grid(sc.nx, sc.ny, sc.nz, precision=precision, **sc.params())
    g.set_porosity(sc.phi.astype(g.np_dtype))
    g.init_state()
    st_f = strouhal_formula(U, sc.D)
    f_f = st_f * U / sc.D
    period = 1.0 / f_f / step
    transient = int(transient_flows * sc.ny * sc.h / U / step)
    every = max(1, int(round(period / samples_per_period)))
    n_samples = int(periods * period / every)
    g.run(transient, stats=False)
    ip = int(sc.centre[0] / sc.h)
    jp = int((sc.centre[1] + 3 * sc.D) / sc.h)
    sig = np.empty(n_samples)
    for n in range(n_samples):
        g.run(every, stats=False)
        sig[n] = g.get_state("u")[0, jp, ip]
    f_m = dominant_frequency(sig, every * step)
    out = {"U": U, "dt": step, "cfl": U * step / sc.h, "steps": transient + n_samples * every,
           "Re": U * sc.D / NU_AIR, "f": f_m, "f_formula": f_f, "St": f_m * sc.D / U, "St_formula": st_f,
           "amplitude": float(np.std(sig)),
           "amplitude_halves": (float(np.std(sig[: n_samples // 2])), float(np.std(sig[n_samples // 2:]))),
           "divergence": g.divergence()}
    g.close()
    return out
