"""Reproduce the hysteresis energies of Sec. IV and the second-derivative minima of Sec. V
on the GPU.

    python -m paper_2108_13410_gb300.reproduce [--p 0.12 0.50] [--dg 1e-5] [--dt 0.02]
                                               [--red 0.05 0.15 0.25] [--table1]

3x3 torus, unitary-gauge form (18 link qubits), J = h = 1/2.  psi_1 prepared at O is
carried along the g axis to P(p, 0), then along the blue path to P'(0, p); psi_1'
prepared at O is carried along the lambda axis to P'(0, p), then back along the blue
path to P(p, 0).  Both energy curves are sampled along the blue path; E (psi_1 at P)
and E' (psi_1' after arriving at P) are printed next to the values quoted in the
hysteresis figure (dg = 1e-5, dt = 2e-2 per step, second-order Trotter, as stated for
the paper's runs), with the crossing points of the two curves.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

PRINTED = {0.12: (-9.16003, -9.15039), 0.50: (-14.06553, -14.06550)}


def _sample_every(n: int, samples: int = 48) -> int:
    """Steps between energy samples: a divisor of n close to n / samples."""
    d = max(1, n // samples)
    while n % d:
        d -= 1
    return d


def hysteresis(p: float, dg: float, dt: float, dtype: str = "c64", order: int = 2, renorm_every: int = 100,
               samples: int = 48, options: dict | None = None):
    """The history dependence of Sec. IV on the blue path, as two energy curves.

    psi_1 (Eq. (14)) is carried from O along the g axis to P(p, 0), then along the blue
    path to P'(0, p); psi_1' (Eq. (15)) is carried along the lambda axis to P'(0, p), then
    along the blue path back to P.  Both energies <H1> are sampled at the same lambda
    values (every few steps, both path ends included).  The printed pair is read at the
    same parameter point P: E is the energy of psi_1 as prepared at P (the start of its
    curve), E' the energy of psi_1' after it arrives at P (the end of its curve).  Reading
    the two path ends instead (psi_1 at P', psi_1' at P) compares mirror images: on the
    self-dual torus with J = h the two processes map onto each other, so those energies
    agree up to the Trotter ordering whatever the phase.

    Returns E, E', both curves (lambda, E(lambda), E'(lambda)), and the lambda values where
    E - E' changes sign (linear interpolation between samples).  renorm_every > 0
    renormalises the state every that many steps: over 10^5 steps the phase tables'
    residual modulus errors (~1e-10 each, correlated while the couplings change slowly)
    would otherwise move the norm by ~1e-5.  options: further {QS_OPT_*: value}."""
    import numpy as np
    from . import Simulator, QS_OPT_RENORM_EVERY
    from .protocol import prepare, blue, run_path
    out = {"p": p, "dtype": dtype, "renorm_every": renorm_every}
    t0 = time.perf_counter()
    sim = Simulator(3, 3, form="ug", dtype=dtype)
    sim.set_option(QS_OPT_RENORM_EVERY, renorm_every)
    for key, value in (options or {}).items():
        sim.set_option(key, value)
    fwd, back = blue(p, dg), blue(p, dg, reverse=True)
    every = _sample_every(len(fwd), samples)
    # psi_1: O -> P, then P -> P'
    sim.init_toric(0)
    sim.evolve_path(prepare(p, dg, "g"), dt, order)
    e1 = [float(sim.energy([(p, 0.0, 0.5, 0.5)])[0])]
    e1 += [e for _, e in run_path(sim, fwd, dt, order, measure_every=every)]
    # psi_1': O -> P', then P' -> P
    sim.init_toric(1)
    sim.evolve_path(prepare(p, dg, "lambda"), dt, order)
    e2 = [float(sim.energy([(0.0, p, 0.5, 0.5)])[0])]
    e2 += [e for _, e in run_path(sim, back, dt, order, measure_every=every)]
    lam = np.linspace(0.0, p, len(e1))
    E1 = np.array(e1)
    E2 = np.array(e2[::-1])                 # on the same lambda grid
    D = E1 - E2
    cross = []
    for i in range(len(D) - 1):
        if D[i] == 0.0 or D[i] * D[i + 1] < 0.0:
            cross.append(float(lam[i] + (lam[i + 1] - lam[i]) * D[i] / (D[i] - D[i + 1])))
    out.update({"E": float(E1[0]), "E_prime": float(E2[0]),
                "E_at_P_prime": float(E1[-1]), "E_prime_at_P_prime": float(E2[-1]),
                "crossings": cross, "max_abs_difference": float(np.max(np.abs(D))),
                "curve": {"lambda": lam.tolist(), "E": E1.tolist(), "E_prime": E2.tolist()},
                "steps_per_state": len(prepare(p, dg)) + len(fwd), "sample_every": every,
                "seconds": time.perf_counter() - t0})
    if p in PRINTED:
        out["printed_E"], out["printed_E_prime"] = PRINTED[p]
    return out


PRINTED_CURVATURE_MIN = {0.05: 0.1920, 0.15: 0.1916, 0.25: 0.2489}


def _curvature_minimum(g, e, k: int, h: float):
    """(g, value) at the smallest central second difference of e over k samples (h in g),
    evaluated at every sample and refined by a parabola through the smallest three."""
    import numpy as np
    d2 = (e[2 * k:] - 2 * e[k:-k] + e[:-2 * k]) / h ** 2          # at g[k:-k]
    gd = g[k:-k]
    i = int(np.argmin(d2[1:-1])) + 1
    y0, y1, y2 = d2[i - 1], d2[i], d2[i + 1]
    shift = 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    return float(gd[i] + shift * (gd[i + 1] - gd[i])), float(y1 + 0.25 * (y0 - y2) * shift)


PRINTED_DUAL_LINE_EXTREMUM = 0.1798


def dual_line_curvature(p: float = 0.5, dg: float = 1e-5, dt: float = 0.02, every: int = 100,
                        stencil: int = 10, dtype: str = "c64", order: int = 2, renorm_every: int = 100):
    """Energy on the dual line g = lambda (Sec. V) and the extremum of its second derivative.

    Reading of the path "from (0, p) through (p, p) to O": psi_1' is carried along the
    lambda axis O -> (0, p) (the state of Sec. IV prepared at P'), then to (p, p), then along
    g = lambda down to O with <H1(g, g)> measured every `every` steps; d^2E/dg^2 as in
    red_path_curvature.  3x3 torus, unitary gauge, J = h = 1/2."""
    import numpy as np
    from . import Simulator, QS_OPT_RENORM_EVERY
    from .protocol import prepare, segment, run_path
    t0 = time.perf_counter()
    sim = Simulator(3, 3, form="ug", dtype=dtype)
    sim.set_option(QS_OPT_RENORM_EVERY, renorm_every)
    sim.init_toric(1)
    sim.evolve_path(prepare(p, dg, "lambda"), dt, order)
    sim.evolve_path(segment((0.0, p), (p, p), dg), dt, order)
    meas = run_path(sim, segment((p, p), (0.0, 0.0), dg), dt, order, measure_every=every)
    g = np.array([c[0] for c, _ in meas])
    e = np.array([v for _, v in meas])
    h = stencil * every * dg
    g_min, d2_min = _curvature_minimum(g, e, stencil, h)
    return {"p": p, "dg": dg, "dt": dt, "dtype": dtype, "h": h, "points": len(g), "g_min": g_min,
            "d2E_min": d2_min, "E_end": float(e[-1]), "printed_g_extremum": PRINTED_DUAL_LINE_EXTREMUM,
            "steps": 3 * int(round(p / dg)), "seconds": time.perf_counter() - t0}


def red_path_curvature(r: float, p: float = 0.5, dg: float = 1e-5, dt: float = 0.02, every: int = 100,
                       stencil: int = 10, dtype: str = "c64", order: int = 2, renorm_every: int = 100,
                       curve: bool = False):
    """Energy along a broken red path of Sec. V and the minimum of its second derivative.

    psi_1 is carried O -> P(p, 0) -> R(p, r), then along R -> R'(0, r) the energy
    <H1(g, r)> is measured every `every` steps (g spacing every * dg).  d^2E/dg^2 is the
    central second difference over `stencil` samples (h = stencil * every * dg = 0.01 by
    default), evaluated at every sample; its minimum is refined by a parabola through the
    smallest three values.  A narrower stencil resolves the small non-adiabatic
    oscillations of E(g) (the same in complex64 and complex128) instead of the
    transition: at h = 0.001 the minimum moves by up to 0.007, from h = 0.005 on it is
    stable to 0.001.  3x3 torus, unitary gauge, J = h = 1/2."""
    import numpy as np
    from . import Simulator, QS_OPT_RENORM_EVERY
    from .protocol import prepare, segment, run_path
    t0 = time.perf_counter()
    sim = Simulator(3, 3, form="ug", dtype=dtype)
    sim.set_option(QS_OPT_RENORM_EVERY, renorm_every)
    sim.init_toric(0)
    sim.evolve_path(prepare(p, dg, "g"), dt, order)
    sim.evolve_path(segment((p, 0.0), (p, r), dg), dt, order)
    meas = run_path(sim, segment((p, r), (0.0, r), dg), dt, order, measure_every=every)
    g = np.array([c[0] for c, _ in meas])
    e = np.array([v for _, v in meas])
    h = stencil * every * dg
    g_min, d2_min = _curvature_minimum(g, e, stencil, h)
    out = {"r": r, "p": p, "dg": dg, "dt": dt, "dtype": dtype, "h": h, "points": len(g),
           "g_min": g_min, "d2E_min": d2_min,
           "E_end": float(e[-1]), "steps": int(round(p / dg)) + int(round(r / dg)) + int(round(p / dg)),
           "seconds": time.perf_counter() - t0}
    if r in PRINTED_CURVATURE_MIN:
        out["printed_g_min"] = PRINTED_CURVATURE_MIN[r]
    if curve:
        out["g"] = g.tolist()
        out["E"] = e.tolist()
    return out


def red_path_dos(r: float, g_points=(0.45, 0.35, 0.25, 0.15, 0.05), p: float = 0.5, dg: float = 1e-5,
                 dt: float = 0.02, dtype: str = "c64", order: int = 2, renorm_every: int = 100):
    """Density of states of Z~ = -sum_l sigma^z_l (Sec. V) along a broken red path.

    psi_1 is carried O -> P(p, 0) -> R(p, r) and then along R -> R'(0, r); when g reaches
    each value of g_points (descending) the histogram P(k) over the number k of links in
    sigma^z = -1 (Z~ = 2k - n_links) is taken with qs_dos.  Returns the histograms, the
    position of the largest bin and the number of maxima of each histogram (the paper
    reads a single maximum in each phase for r < 0.16 as a second-order transition).
    Reading of "maximum": in the deconfined phase the bins of even and odd k alternate
    (the toric-code parity structure), so maxima are counted on the even-k and the odd-k
    envelopes separately, each ignoring local maxima below 5% of its largest bin."""
    import numpy as np
    from . import Simulator, QS_OPT_RENORM_EVERY
    from .protocol import prepare, segment
    t0 = time.perf_counter()
    sim = Simulator(3, 3, form="ug", dtype=dtype)
    sim.set_option(QS_OPT_RENORM_EVERY, renorm_every)
    sim.init_toric(0)
    sim.evolve_path(prepare(p, dg, "g"), dt, order)
    sim.evolve_path(segment((p, 0.0), (p, r), dg), dt, order)
    g_now, out = p, []
    for g in sorted(g_points, reverse=True):
        if g < g_now:
            sim.evolve_path(segment((g_now, r), (g, r), dg), dt, order)
            g_now = g
        h = sim.dos()[0]
        maxima = []
        for par in (0, 1):
            v = h[par::2]
            top = float(v.max())
            maxima.append(sum(1 for i in range(len(v))
                              if v[i] >= 0.05 * top and (i == 0 or v[i] > v[i - 1])
                              and (i == len(v) - 1 or v[i] > v[i + 1])))
        out.append({"g": g, "dos": h.tolist(), "maxima_even": maxima[0], "maxima_odd": maxima[1],
                    "argmax_k": int(np.argmax(h)), "mean_k": float(np.dot(np.arange(len(h)), h)),
                    "sum": float(h.sum())})
    return {"r": r, "p": p, "dg": dg, "dt": dt, "dtype": dtype, "points": out,
            "seconds": time.perf_counter() - t0}


PRINTED_TABLE1 = {200: (0.03982, 4.79e-5), 500: (0.04009, 4.99e-5), 800: (0.04075, 4.98e-5)}


def trotter_error_study(ns=(10, 200, 500, 800), n0: int = 10, r: float = 0.05, p: float = 0.5,
                        grid: float = 1e-4, dtype: str = "c64", order: int = 2, renorm_every: int = 100):
    """The Trotter-error comparison of Sec. VI (Table I) on the subpath R(p, r) -> R'(0, r).

    Reading: the state is prepared once at R (psi_1 carried O -> P -> R with dg = 1e-5,
    dt = 0.02), then every run n takes the subpath with dg = 1e-4 / n and dt = 0.2 / n, so
    dg / dt is the same for all n (the same continuous adiabatic path) and the runs differ
    by their Trotter error only.  E_n(g) = <H1(g, r)> is sampled every `grid` in g (the
    same points for every n); delta_n = sum over the samples of |E_n0(g) - E_n(g)| and
    alpha_n = max over the samples.  3x3 torus, unitary gauge, J = h = 1/2.  The
    differences are ~1e-6: complex64 rounding (~3e-6 over these runs) hides them, so the
    comparison needs complex128."""
    import numpy as np
    from . import Simulator, QS_OPT_RENORM_EVERY
    from .protocol import prepare, segment
    t0 = time.perf_counter()
    sim = Simulator(3, 3, form="ug", dtype=dtype)
    sim.set_option(QS_OPT_RENORM_EVERY, renorm_every)
    sim.init_toric(0)
    sim.evolve_path(prepare(p, 1e-5, "g"), 0.02, order)
    sim.evolve_path(segment((p, 0.0), (p, r), 1e-5), 0.02, order)
    at_r = sim.state.clone()
    n_pts = int(round(p / grid))
    curves, runs = {}, []
    for n in ns:
        dg, dt = 1e-4 / n, 0.2 / n
        per = int(round(grid / dg))                 # steps between samples
        sim.state.copy_(at_r)
        t1 = time.perf_counter()
        e = np.empty(n_pts)
        for j in range(n_pts):
            k = j * per + np.arange(1, per + 1)     # global step indices of this piece
            a = np.empty((per, 4))
            a[:, 0] = p - dg * k                    # g_k = p - k dg
            a[:, 1] = r
            a[:, 2] = 0.5
            a[:, 3] = 0.5
            sim.evolve_path(a, dt, order)
            e[j] = float(sim.energy([(a[-1, 0], r, 0.5, 0.5)])[0])
        curves[n] = e
        runs.append({"n": n, "dg": dg, "dt": dt, "steps": per * n_pts, "seconds": time.perf_counter() - t1})
    for run in runs:
        d = np.abs(curves[n0] - curves[run["n"]])
        run["delta"] = float(d.sum())
        run["alpha"] = float(d.max())
        if run["n"] in PRINTED_TABLE1:
            run["printed_delta"], run["printed_alpha"] = PRINTED_TABLE1[run["n"]]
    return {"r": r, "p": p, "n0": n0, "grid": grid, "samples": n_pts, "dtype": dtype, "runs": runs,
            "seconds": time.perf_counter() - t0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--p", type=float, nargs="+", default=[0.12, 0.50])
    ap.add_argument("--dg", type=float, default=1e-5)
    ap.add_argument("--dt", type=float, default=0.02)
    ap.add_argument("--dtype", default="c64")
    ap.add_argument("--renorm-every", type=int, default=100)
    ap.add_argument("--red", type=float, nargs="*", default=[],
                    help="also the second-derivative minima along the red paths at these r")
    ap.add_argument("--table1", action="store_true",
                    help="also the Trotter-error comparison of Sec. VI (n = 10, 200, 500, 800; complex128)")
    a = ap.parse_args()
    out = {"hysteresis": [hysteresis(p, a.dg, a.dt, a.dtype, renorm_every=a.renorm_every) for p in a.p],
           "dg": a.dg, "dt": a.dt, "dtype": a.dtype}
    if a.red:
        out["red_paths"] = [red_path_curvature(r, dg=a.dg, dt=a.dt, dtype=a.dtype, renorm_every=a.renorm_every)
                            for r in a.red]
    if a.table1:
        out["table1"] = trotter_error_study(grid=1e-5, dtype="c128", renorm_every=0)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
