// lattice.h -- term tables of the Z2 gauge-Higgs model for the CUDA path.
//
// Sec. II: sigma qubits on links, tau qubits on vertices (gauge-Higgs form,
// Eq. (1)); links only in the unitary-gauge form (Eq. (4)).  Terms are kept as
// 64-bit qubit masks:
//   X type:  sigma^x_l, tau^x_v (single qubit), A_v (X string, unitary gauge)
//   Z type:  B_p (4 links), bond tau^z_j sigma^z_l tau^z_k (gauge-Higgs),
//            sigma^z_l (unitary gauge)
// The numbering is documented in include/qsim.h.
#pragma once
#include <cstdint>
#include <stdexcept>
#include <vector>

namespace qsim {

struct Lattice {
    int Lx = 0, Ly = 0;
    bool periodic = true;
    bool gauge_higgs = true;
    int n_links = 0, n_vertices = 0, n_qubits = 0;
    std::vector<uint64_t> plaquettes;   // B_p masks
    std::vector<uint64_t> second;       // bonds (gh) or sigma^z_l (ug)
    std::vector<uint64_t> stars;        // A_v link masks, one per vertex
    std::vector<uint64_t> gauss;        // Q_v = tau^x_v A_v (gh)
    std::vector<uint64_t> wilson;       // W_x, W_y (periodic)
    std::vector<uint64_t> thooft;       // V_1, V_2 (periodic)
    std::vector<int> x_class;           // per qubit: 0 = sigma^x (link), 1 = tau^x (vertex)
};

inline Lattice make_lattice(int Lx, int Ly, bool periodic, bool gauge_higgs) {
    Lattice L;
    L.Lx = Lx; L.Ly = Ly; L.periodic = periodic; L.gauge_higgs = gauge_higgs;
    int vx = periodic ? Lx : Lx + 1;
    int vy = periodic ? Ly : Ly + 1;
    if (periodic ? (Lx < 2 || Ly < 2) : (Lx < 1 || Ly < 1))
        throw std::invalid_argument("lattice too small");
    L.n_vertices = vx * vy;
    // link numbering
    std::vector<int> H(vx * vy, -1), U(vx * vy, -1);
    int q = 0;
    if (periodic) {
        int N = vx * vy;
        for (int v = 0; v < N; ++v) { H[v] = v; U[v] = N + v; }
        q = 2 * N;
    } else {
        for (int y = 0; y < vy; ++y)
            for (int x = 0; x + 1 < vx; ++x) H[y * vx + x] = q++;
        for (int y = 0; y + 1 < vy; ++y)
            for (int x = 0; x < vx; ++x) U[y * vx + x] = q++;
    }
    L.n_links = q;
    L.n_qubits = gauge_higgs ? q + L.n_vertices : q;
    if (L.n_qubits > 63) throw std::invalid_argument("too many qubits");
    auto h = [&](int x, int y) -> int {
        if (periodic) { x = (x % vx + vx) % vx; y = (y % vy + vy) % vy; }
        else if (x < 0 || y < 0 || x >= vx || y >= vy) return -1;
        return H[y * vx + x];
    };
    auto u = [&](int x, int y) -> int {
        if (periodic) { x = (x % vx + vx) % vx; y = (y % vy + vy) % vy; }
        else if (x < 0 || y < 0 || x >= vx || y >= vy) return -1;
        return U[y * vx + x];
    };
    auto bit = [](int qq) -> uint64_t { return qq < 0 ? 0ull : (1ull << qq); };
    auto site = [&](int x, int y) -> int { return L.n_links + y * vx + x; };

    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x)
            L.plaquettes.push_back(bit(h(x, y)) | bit(h(x, y + 1)) | bit(u(x, y)) | bit(u(x + 1, y)));
    for (int y = 0; y < vy; ++y)
        for (int x = 0; x < vx; ++x) {
            uint64_t m = bit(h(x, y)) | bit(u(x, y));
            if (periodic || x >= 1) m |= bit(h(x - 1, y));
            if (periodic || y >= 1) m |= bit(u(x, y - 1));
            L.stars.push_back(m);
            if (gauge_higgs) L.gauss.push_back(m | bit(site(x, y)));
        }
    // second Z class, in link-qubit order
    std::vector<uint64_t> sec(L.n_links, 0);
    for (int y = 0; y < vy; ++y)
        for (int x = 0; x < vx; ++x) {
            int hq = H[y * vx + x], uq = U[y * vx + x];
            if (hq >= 0) {
                int x2 = (x + 1) % vx;
                sec[hq] = gauge_higgs ? (bit(site(x, y)) | bit(hq) | bit(site(x2, y))) : bit(hq);
            }
            if (uq >= 0) {
                int y2 = (y + 1) % vy;
                sec[uq] = gauge_higgs ? (bit(site(x, y)) | bit(uq) | bit(site(x, y2))) : bit(uq);
            }
        }
    L.second = sec;
    if (periodic) {
        uint64_t wx = 0, wy = 0, v1 = 0, v2 = 0;
        for (int x = 0; x < vx; ++x) { wx |= bit(h(x, 0)); v2 |= bit(u(x, 0)); }
        for (int y = 0; y < vy; ++y) { wy |= bit(u(0, y)); v1 |= bit(h(0, y)); }
        L.wilson = {wx, wy};
        L.thooft = {v1, v2};
    }
    L.x_class.assign(L.n_qubits, 0);
    for (int k = L.n_links; k < L.n_qubits; ++k) L.x_class[k] = 1;
    return L;
}

}  // namespace qsim
