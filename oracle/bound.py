"""Trotter error-bound arithmetic of Sec. VI and the Appendix (test infrastructure only).

Along the sub-path lambda = r, g = n * dg (n = 1..N, N = p / dg), the Appendix
bounds each second-order step by dt^3/6 W_1 + dt^3/12 W_2 with
    W_1 = 162 g + 648 g lambda^2 + 648 g lambda + 324 lambda^2,
    W_2 = 324 g^2 + 648 g^2 lambda + 162 lambda,
from the norm estimates ||H_1|| ~ 18 g, ||H_3|| ~ 18 lambda, ||H_2|| ~ 9,
||[H_1,H_2]|| ~ 18 g, ||[H_1,H_3]|| ~ 36 g lambda, ||[H_2,H_3]|| ~ 18 lambda
(3x3 torus, 18 links).  Summing with sum g ~ pN/2 and sum g^2 ~ p^2 N/3 gives the
closed form of Sec. VI:
    eps <~ dt^3 N (13.5 p + 54 p r^2 + 54 p r + 54 r^2 + 9 p^2 + 18 p^2 r + 13.5 r).
The stray Delta_m factor in the W_2 sum of the Appendix is read as a typo (the
closed form only follows without it).
"""
from __future__ import annotations


def w1(g: float, lam: float) -> float:
    # ||H2|| (||[H2,H1]|| + ||[H3,H1]||) + ||H3|| (||[H2,H1]|| + ||[H3,H1]|| + ||[H3,H2]||)
    return 9.0 * (18.0 * g + 36.0 * g * lam) + 18.0 * lam * (18.0 * g + 36.0 * g * lam + 18.0 * lam)


def w2(g: float, lam: float) -> float:
    # ||H1|| (||[H1,H2]|| + ||[H1,H3]||) + ||H2|| ||[H2,H3]||
    return 18.0 * g * (18.0 * g + 36.0 * g * lam) + 9.0 * (18.0 * lam)


def eps_sum(p: float, r: float, dg: float, dt: float) -> float:
    """Step-by-step sum of the per-step bound along g = n dg, n = 1..N."""
    N = int(round(p / dg))
    tot = 0.0
    for n in range(1, N + 1):
        g = n * dg
        tot += dt ** 3 / 6.0 * w1(g, r) + dt ** 3 / 12.0 * w2(g, r)
    return tot


def eps_closed(p: float, r: float, dg: float, dt: float) -> float:
    """Closed form of Sec. VI."""
    N = p / dg
    return dt ** 3 * N * (13.5 * p + 54 * p * r * r + 54 * p * r + 54 * r * r
                          + 9 * p * p + 18 * p * p * r + 13.5 * r)


def table1_row(n: int, p: float = 0.5, r: float = 0.05):
    """(dg, dt, eps) for Table I: dg = 1e-4 / n, dt = 0.2 / n."""
    dg = 1e-4 / n
    dt = 0.2 / n
    return dg, dt, eps_closed(p, r, dg, dt)
