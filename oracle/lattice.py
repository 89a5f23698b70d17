"""Oracle lattice: qubit numbering and Pauli-string term lists (test infrastructure).

Follows the model of Sec. II:
  * gauge-Higgs form, Eq. (1): sigma qubits on links, tau qubits on vertices;
    terms -J tau^x_v, -h B_p (B_p = product of the four sigma^z around p, Eq. (2)),
    -g sigma^x_l, -lambda tau^z_j sigma^z_<jk> tau^z_k;
    Gauss-law generators Q_v = tau^x_v A^x_v (Eq. (3)).
  * unitary-gauge (toric code in two transverse fields) form, Eq. (4): links only;
    terms -J A^x_v, -h B_p, -g sigma^x_l, -lambda sigma^z_l.

The paper's lattice figure is not available, so the numbering below is this
project's own (layout-independent observables only):
  periodic Lx x Ly torus, N = Lx*Ly vertices, v = y*Lx + x:
      horizontal link (x,y)->(x+1,y): qubit v
      vertical   link (x,y)->(x,y+1): qubit N + v
      vertex tau_v (gauge-Higgs form only): qubit 2N + v
  open Lx x Ly plaquettes, (Lx+1) x (Ly+1) vertices, v = y*(Lx+1) + x:
      existing horizontal links ordered by v, then vertical links by v, then
      vertex qubits (gauge-Higgs form only).
  plaquette (x,y) = {h(x,y), h(x,y+1), u(x,y), u(x+1,y)}
  star A_v        = the existing links among {h(x,y), h(x-1,y), u(x,y), u(x,y-1)}
  bond on link l = <j,k>: {tau_j, sigma_l, tau_k}
Bit value 0 of a qubit is the Z = +1 eigenstate.

This file is the oracle's own copy of the layout; the CUDA path builds its term
tables independently.
"""
from __future__ import annotations

from dataclasses import dataclass, field


def mask_of(qubits) -> int:
    m = 0
    for q in qubits:
        m |= 1 << q
    return m


@dataclass
class OracleLattice:
    Lx: int
    Ly: int
    periodic: bool
    form: str  # "gh" (gauge-Higgs) or "ug" (unitary gauge)
    n_qubits: int = 0
    hlink: dict = field(default_factory=dict)   # (x, y) -> qubit
    ulink: dict = field(default_factory=dict)   # (x, y) -> qubit
    site: dict = field(default_factory=dict)    # (x, y) -> qubit (gh only)
    links: list = field(default_factory=list)   # [(qubit, (x,y), (x2,y2))]
    plaquettes: list = field(default_factory=list)  # lists of 4 qubits
    stars: list = field(default_factory=list)       # lists of link qubits per vertex
    bonds: list = field(default_factory=list)       # [tau_j, sigma_l, tau_k] (gh)
    vertices: list = field(default_factory=list)    # [(x, y)] in v order

    def __post_init__(self):
        if self.form not in ("gh", "ug"):
            raise ValueError("form must be 'gh' or 'ug'")
        Lx, Ly = self.Lx, self.Ly
        if self.periodic:
            if Lx < 2 or Ly < 2:
                raise ValueError("periodic lattice needs Lx, Ly >= 2")
            vx, vy = Lx, Ly
            N = Lx * Ly
            self.vertices = [(x, y) for y in range(vy) for x in range(vx)]
            for y in range(vy):
                for x in range(vx):
                    v = y * Lx + x
                    self.hlink[(x, y)] = v
                    self.ulink[(x, y)] = N + v
            nl = 2 * N
        else:
            if Lx < 1 or Ly < 1:
                raise ValueError("open lattice needs Lx, Ly >= 1")
            vx, vy = Lx + 1, Ly + 1
            self.vertices = [(x, y) for y in range(vy) for x in range(vx)]
            q = 0
            for y in range(vy):
                for x in range(vx - 1):
                    self.hlink[(x, y)] = q
                    q += 1
            for y in range(vy - 1):
                for x in range(vx):
                    self.ulink[(x, y)] = q
                    q += 1
            nl = q
        self.n_links = nl
        self.n_sites = vx * vy
        self._vx, self._vy = vx, vy
        if self.form == "gh":
            for i, (x, y) in enumerate(self.vertices):
                self.site[(x, y)] = nl + i
            self.n_qubits = nl + self.n_sites
        else:
            self.n_qubits = nl

        def H(x, y):
            if self.periodic:
                return self.hlink[(x % vx, y % vy)]
            return self.hlink.get((x, y))

        def U(x, y):
            if self.periodic:
                return self.ulink[(x % vx, y % vy)]
            return self.ulink.get((x, y))

        # links with their end points
        for (x, y), q in self.hlink.items():
            self.links.append((q, (x, y), ((x + 1) % vx, y)))
        for (x, y), q in self.ulink.items():
            self.links.append((q, (x, y), (x, (y + 1) % vy)))
        self.links.sort()

        for y in range(Ly):
            for x in range(Lx):
                self.plaquettes.append([H(x, y), H(x, y + 1), U(x, y), U(x + 1, y)])
        for (x, y) in self.vertices:
            cand = [H(x, y), H(x - 1, y) if (self.periodic or x >= 1) else None,
                    U(x, y), U(x, y - 1) if (self.periodic or y >= 1) else None]
            self.stars.append([q for q in cand if q is not None])
        if self.form == "gh":
            for q, a, b in self.links:
                self.bonds.append([self.site[a], q, self.site[b]])

    # ---- term lists -------------------------------------------------------
    @property
    def link_qubits(self):
        return [q for q, _, _ in self.links]

    @property
    def site_qubits(self):
        return [self.site[v] for v in self.vertices] if self.form == "gh" else []

    def x_single(self):
        """(qubit, kind) for single-qubit X terms: kind 's' = sigma^x, 't' = tau^x."""
        out = [(q, "s") for q in self.link_qubits]
        out += [(q, "t") for q in self.site_qubits]
        return out

    def x_strings(self):
        """X-string terms of the unitary-gauge form: the star operators A_v."""
        return [mask_of(s) for s in self.stars] if self.form == "ug" else []

    def z_plaquettes(self):
        return [mask_of(p) for p in self.plaquettes]

    def z_second(self):
        """Second Z class: bonds tau^z sigma^z tau^z (gh) or sigma^z_l (ug)."""
        if self.form == "gh":
            return [mask_of(b) for b in self.bonds]
        return [1 << q for q in self.link_qubits]

    def gauss(self):
        """Q_v = tau^x_v A^x_v as X-string masks (gh form only)."""
        if self.form != "gh":
            return []
        return [mask_of([self.site[v]] + s) for v, s in zip(self.vertices, self.stars)]

    def wilson(self):
        """Non-contractible Wilson loops W_x (along x at y=0) and W_y (along y at x=0)."""
        if not self.periodic:
            return []
        wx = mask_of([self.hlink[(x, 0)] for x in range(self._vx)])
        wy = mask_of([self.ulink[(0, y)] for y in range(self._vy)])
        return [wx, wy]

    def thooft(self):
        """'t Hooft loops V_1 = prod_y X_h(0,y), V_2 = prod_x X_u(x,0) (X-string masks)."""
        if not self.periodic:
            return []
        v1 = mask_of([self.hlink[(0, y)] for y in range(self._vy)])
        v2 = mask_of([self.ulink[(x, 0)] for x in range(self._vx)])
        return [v1, v2]
