"""Reproduce the hysteresis energies of Sec. IV on the GPU.

    python -m paper_2108_13410_gb300.reproduce [--p 0.12 0.50] [--dg 1e-5] [--dt 0.02]

3x3 torus, unitary-gauge form (18 link qubits), J = h = 1/2.  E: psi_1 prepared at O is
carried along the g axis to P(p, 0), then along the blue path to P'(0, p); E': psi_1'
prepared at O is carried along the lambda axis to P'(0, p), then back along the blue
path to P(p, 0).  The energies at the path ends are printed next to the values quoted
in the hysteresis figure (dg = 1e-5, dt = 2e-2 per step, second-order Trotter, as stated
for the paper's runs).  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

PRINTED = {0.12: (-9.16003, -9.15039), 0.50: (-14.06553, -14.06550)}


def hysteresis(p: float, dg: float, dt: float, dtype: str = "c64", order: int = 2, renorm_every: int = 100,
               options: dict | None = None):
    """Energies at the ends of the two hysteresis paths.  renorm_every > 0 renormalises
    the state every that many steps: over 10^5 steps the phase tables' residual modulus
    errors (~1e-10 each, correlated while the couplings change slowly) would otherwise
    move the norm by ~1e-5.  options: further {QS_OPT_*: value} for the simulator."""
    from . import Simulator, QS_OPT_RENORM_EVERY
    from .protocol import prepare, blue
    out = {"p": p, "dtype": dtype, "renorm_every": renorm_every}
    t0 = time.perf_counter()
    sim = Simulator(3, 3, form="ug", dtype=dtype)
    sim.set_option(QS_OPT_RENORM_EVERY, renorm_every)
    for key, value in (options or {}).items():
        sim.set_option(key, value)
    sim.init_toric(0)
    sim.evolve_path(prepare(p, dg, "g"), dt, order)
    path = blue(p, dg)
    sim.evolve_path(path, dt, order)
    out["E"] = float(sim.energy([path[-1]])[0])
    sim.init_toric(1)
    sim.evolve_path(prepare(p, dg, "lambda"), dt, order)
    path = blue(p, dg, reverse=True)
    sim.evolve_path(path, dt, order)
    out["E_prime"] = float(sim.energy([path[-1]])[0])
    out["steps_per_state"] = len(prepare(p, dg)) + len(path)
    out["seconds"] = time.perf_counter() - t0
    if p in PRINTED:
        out["printed_E"], out["printed_E_prime"] = PRINTED[p]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--p", type=float, nargs="+", default=[0.12, 0.50])
    ap.add_argument("--dg", type=float, default=1e-5)
    ap.add_argument("--dt", type=float, default=0.02)
    ap.add_argument("--dtype", default="c64")
    ap.add_argument("--renorm-every", type=int, default=100)
    a = ap.parse_args()
    print(json.dumps({"hysteresis": [hysteresis(p, a.dg, a.dt, a.dtype, renorm_every=a.renorm_every) for p in a.p],
                      "dg": a.dg, "dt": a.dt, "dtype": a.dtype}))


if __name__ == "__main__":
    main()
