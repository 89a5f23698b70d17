// scan_mixed.cuh -- the phase-diagram scan of two lattices in one persistent launch.
//
// Every coupling point is an independent adiabatic run (Sec. III).  One launch takes the
// points of a 12-qubit gauge-Higgs lattice (the 2x2 torus) and of a 13..20-qubit lattice
// in the unitary gauge (the 3x2 open lattice has 17 link qubits), CTAs pulling points
// from a work queue (one atomic counter; no CTA ever waits for another):
//   * a 12-qubit point runs on chip in the CTA's shared memory (scan12_point);
//   * a larger unitary-gauge point runs on the CTA's own slot of a scratch state in global
//     memory (the slot, 2^n complex64 amplitudes, stays in L2 while the CTA works on it),
//     as the Walsh-Hadamard form of every Trotter factor group: two TMA-pipelined passes
//     over the slot's 2^(n-12) tiles of 4096 amplitudes,
//         pass 1 (qubits 12..n-1):  H, the Hadamard-basis X table D_X (and 2^-n), H
//         pass 0 (qubits 0..11):    H, the Z layer, H of the next factor group
//     (all Walsh-Hadamard butterflies on different qubits commute, and the leading H of
//     the first group is a pass of its own).  The observables follow from the final
//     state: the diagonal ones in the last pass, sigma^x and the stars A_v from one more
//     Walsh-Hadamard transform (diagonal in the Hadamard basis).
// Diagonal factors are products of two small tables, exp(i alpha (nA - 2a)) exp(i beta
// (nB - 2b)) for a odd terms of class A and b of class B, rebuilt every factor group with
// dev_unit_pair_fast.
#pragma once
#include "scan.cuh"
#include "xpass_tma.cuh"

namespace qsim {

struct ScanUGParams {
    int n_points, n_ops;          // points of the unitary-gauge lattice, factor groups per point
    RecGeom G;                    // schedule geometry (batch 1)
    int n;                        // qubits (13..20)
    int nP, nL, nS;               // plaquettes, links, stars
    int tiles_shift;              // n - 12: tiles per state = 2^tiles_shift
    float scale;                  // 2^-n
    TmaPass p0;                   // pass 0: qubits 0..11, Z-layer classes (plaquettes, links)
    TmaPass p1;                   // pass 1: the other qubits, Hadamard-basis classes (stars, links)
};

// unnormalised Walsh-Hadamard butterflies on the register bits of mask
__device__ __forceinline__ void had_w(u64 (&w)[NR], unsigned mask) { hadamard_w(w, mask); }

// Diagonal factor of an amplitude from its odd-term counts (tables ta[a], tb[b] of
// (u, s) pairs) and, when measuring, |v|^2 weighted by (nA - 2a) and (nB - 2b).
struct DiagOps {
    const float2 *ta, *tb;        // null: no phase
    float scale;                  // applied with the phase (1: none)
    bool measure;
    float wscale;                 // factor of the measured weights
};

// One tile in shared memory (swizzled, 4096 amplitudes): round 1 of Walsh-Hadamard
// butterflies (stages A, B, C on P.rot), the diagonal factor in the stage-C layout,
// optionally round 2 (stages C, B, A); the result is left in shared memory in the layout
// of the last stage.  pa, pb: parity words of this thread's stage-C position and tile.
__device__ void ug_tile(u64 *tb, const TmaPass &P, uint32_t pa, uint32_t pb, const DiagOps &D, bool round2,
                        float (&m)[3]) {
    const int t = threadIdx.x;
    const int tlo = t & 15, thi = t >> 4;
    const int a_base = swz128(t);
    const int b_base = t << 3, b_x = t & 7;
    auto c_idx = [&](int r) { return ((tlo ^ ((r & 7) << 1)) | (thi << 8)) + (r << 4); };
    u64 w[NR];
    // ---- round 1: stage A ----
#pragma unroll
    for (int r = 0; r < NR; ++r) w[r] = tb[a_base + (r << TB)];
    had_w(w, P.rot[0]);
#pragma unroll
    for (int r = 0; r < NR; ++r) tb[a_base + (r << TB)] = w[r];
    __syncthreads();
    if (P.stage_b) {
        ulonglong2 *t2 = reinterpret_cast<ulonglong2 *>(tb);
#pragma unroll
        for (int q = 0; q < NR / 2; ++q) { const ulonglong2 x = t2[b_base + (q ^ b_x)]; w[2 * q] = x.x; w[2 * q + 1] = x.y; }
        had_w(w, P.rot[1]);
#pragma unroll
        for (int q = 0; q < NR / 2; ++q) t2[b_base + (q ^ b_x)] = make_ulonglong2(w[2 * q], w[2 * q + 1]);
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) w[r] = tb[c_idx(r)];
    had_w(w, P.rot[2]);
    // ---- diagonal factor and measurement in the stage-C layout ----
    if (D.ta || D.measure) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int oa = __popc(pa ^ P.pa_reg[r]), ob = __popc(pb ^ P.pb_reg[r]);
            float2 v = unpk(w[r]);
            if (D.ta) {
                v = cphase(cphase(v, D.ta[oa]), D.tb[ob]);
                v.x *= D.scale; v.y *= D.scale;
            }
            if (D.measure) {
                const float q = (v.x * v.x + v.y * v.y) * D.wscale;
                m[0] += q;
                m[1] += q * (float)(P.nA - 2 * oa);
                m[2] += q * (float)(P.nB - 2 * ob);
            }
            w[r] = pk(v.x, v.y);
        }
    }
    if (!round2) {
#pragma unroll
        for (int r = 0; r < NR; ++r) tb[c_idx(r)] = w[r];
        return;
    }
    // ---- round 2: stages C (in registers), B, A ----
    had_w(w, P.rot[2]);
#pragma unroll
    for (int r = 0; r < NR; ++r) tb[c_idx(r)] = w[r];
    __syncthreads();
    if (P.stage_b) {
        ulonglong2 *t2 = reinterpret_cast<ulonglong2 *>(tb);
#pragma unroll
        for (int q = 0; q < NR / 2; ++q) { const ulonglong2 x = t2[b_base + (q ^ b_x)]; w[2 * q] = x.x; w[2 * q + 1] = x.y; }
        had_w(w, P.rot[1]);
#pragma unroll
        for (int q = 0; q < NR / 2; ++q) t2[b_base + (q ^ b_x)] = make_ulonglong2(w[2 * q], w[2 * q + 1]);
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) w[r] = tb[a_base + (r << TB)];
    had_w(w, P.rot[0]);
#pragma unroll
    for (int r = 0; r < NR; ++r) tb[a_base + (r << TB)] = w[r];
}

// The same for a pass whose butterflies sit on tile bits 8..11 and 7 only (the 17-qubit
// lattice's second pass, 5 new qubits): one layout L holds the whole round, registers =
// bits 8..11, lanes = bits 0..3 and 7, warps = bits 4..6.  Bit 7's butterflies exchange
// through a warp shuffle (partner lane ^ 16), so the tile is read and written once, with
// no block barrier inside the tile.  With the 128-byte swizzle a half-warp reads one whole
// 128-byte row (bits 0..3), free of bank conflicts.  pa, pb: parity words of the tile.
__device__ void ug_tile_l(u64 *tb, const TmaPass &P, uint32_t pa, uint32_t pb, const DiagOps &D, bool round2,
                          float (&m)[3]) {
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    // slot of register r: l = (lane & 15) | warp << 4 | (lane >> 4) << 7 | r << 8,
    // swizzled l ^ (((l >> 4) & 7) << 1) = l ^ (warp << 1)
    const int base = ((lane & 15) ^ (warp << 1)) | (warp << 4) | ((lane >> 4) << 7);
    // parity of this thread's local bits (0..3 and 7 from the lane, 4..6 from the warp)
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if ((lane >> j) & 1) { pa ^= P.paA_thr[j]; pb ^= P.pbA_thr[j]; }
    if (lane & 16) { pa ^= P.paA_thr[7]; pb ^= P.pbA_thr[7]; }
#pragma unroll
    for (int j = 0; j < 3; ++j)
        if ((warp >> j) & 1) { pa ^= P.paA_thr[4 + j]; pb ^= P.pbA_thr[4 + j]; }
    const bool bit7 = (P.rot[2] & 8u) != 0;
    const float sg = (lane & 16) ? -1.f : 1.f;
    const u64 sgn = pk(sg, sg);
    // butterflies on bit 7: the lane with the bit clear keeps self + partner, the other
    // partner - self
    auto shfl_round = [&](u64 (&w)[NR]) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const unsigned lo = (unsigned)w[r], hi = (unsigned)(w[r] >> 32);
            const u64 other = ((u64)__shfl_xor_sync(0xffffffffu, hi, 16) << 32) | __shfl_xor_sync(0xffffffffu, lo, 16);
            w[r] = fma2p(sgn, w[r], other);
        }
    };
    u64 w[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) w[r] = tb[base + (r << 8)];
    had_w(w, P.rot[0]);
    if (bit7) shfl_round(w);
    if (D.ta || D.measure) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int oa = __popc(pa ^ P.paA_reg[r]), ob = __popc(pb ^ P.pbA_reg[r]);
            float2 v = unpk(w[r]);
            if (D.ta) {
                v = cphase(cphase(v, D.ta[oa]), D.tb[ob]);
                v.x *= D.scale; v.y *= D.scale;
            }
            if (D.measure) {
                const float q = (v.x * v.x + v.y * v.y) * D.wscale;
                m[0] += q;
                m[1] += q * (float)(P.nA - 2 * oa);
                m[2] += q * (float)(P.nB - 2 * ob);
            }
            w[r] = pk(v.x, v.y);
        }
    }
    if (round2) {
        if (bit7) shfl_round(w);
        had_w(w, P.rot[0]);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) tb[base + (r << 8)] = w[r];
}

// Persistent scan of both lattices.  Shared memory (dynamic, 1024-byte aligned): NBUF
// 32 KB tile buffers (the 12-qubit points use the first as their state); a pass keeps
// NBUF - 1 tile loads in flight ahead of the tile being processed.
template <int NBUF>
__global__ void __launch_bounds__(NT, NBUF <= 3 ? 2 : 1) k_scan_mixed(const DevCouplings *__restrict__ cpl12,
                                                      const DevCouplings *__restrict__ cpl17,
                                                      const double *__restrict__ sv,
                                                      double *__restrict__ out12, double *__restrict__ out17,
                                                      int *__restrict__ queue, int *__restrict__ err_flag,
                                                      const __grid_constant__ CUtensorMap tmap0,
                                                      const __grid_constant__ CUtensorMap tmap1,
                                                      const __grid_constant__ ScanParams P12,
                                                      const __grid_constant__ ScanUGParams U) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base_ptr = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float2 *buf = reinterpret_cast<float2 *>(base_ptr);            // NBUF x 4096
    __shared__ uint64_t bars[NBUF];
    __shared__ int s_item, s_ok;
    __shared__ float2 lut12[64];
    __shared__ float xus12[4];
    __shared__ double red[NT / 32][SCAN_NOBS];
    __shared__ float2 tXa[33], tXb[33], tZa[33], tZb[33];           // per-step factor tables
    __shared__ double mred[NT / 32][6];

    const int t = threadIdx.x;
    const long long max_wait = 2000000000ll;
    if (t == 0) {
        for (int b = 0; b < NBUF; ++b) mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
    __syncthreads();
    const int n_items = U.n_points + P12.n_points;
    long long gi = 0;                  // tiles loaded by this CTA: buffer gi % NBUF, parity (gi / NBUF) & 1
    const long long slot = blockIdx.x;
    // parity words of this thread's stage-C position in a pass
    auto thread_par = [&](const TmaPass &P, uint32_t &a, uint32_t &b) {
        a = 0; b = 0;
        const int tlo = t & 15, thi = t >> 4;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if ((tlo >> j) & 1) { a ^= P.pa_thr[j]; b ^= P.pb_thr[j]; }
            if ((thi >> j) & 1) { a ^= P.pa_thr[4 + j]; b ^= P.pb_thr[4 + j]; }
        }
    };
    auto tile_par = [&](const TmaPass &P, int tt, uint32_t &a, uint32_t &b) {
        a = 0; b = 0;
        for (int i = 0; i < U.tiles_shift; ++i)
            if ((tt >> i) & 1) { a ^= P.pa_tile[i]; b ^= P.pb_tile[i]; }
    };
    auto issue = [&](const CUtensorMap *map, const TmaPass &P, long long g, int tt) {
        const int b = (int)(g % NBUF);
        const long long tile = (slot << U.tiles_shift) | tt;
        const int x2 = (int)(tile & ((1ll << P.mid_bits) - 1));
        const int x4 = (int)(tile >> P.mid_bits);
        bulk_wait_read_all();                      // a store may still be reading the buffer
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&bars[b], TMA_TILE_BYTES);
        tma_load_5d(buf + (size_t)b * (1 << LT), map, &bars[b], 0, 0, x2, 0, x4);
    };
    // One pass over the slot's tiles: TMA load (next tile prefetched), ug_tile, TMA store.
    // Returns false if a load timed out (error flag set).
    auto pass = [&](const CUtensorMap *map, const TmaPass &P, const DiagOps &D, bool round2, bool store,
                    float (&m)[3]) -> bool {
        const int tiles = 1 << U.tiles_shift;
        uint32_t pa_t, pb_t;
        thread_par(P, pa_t, pb_t);
        if (t == 0) {
            bulk_wait_all();                       // the previous pass's stores are written
            asm volatile("fence.proxy.async.global;" ::: "memory");
            for (int j = 0; j < NBUF - 1 && j < tiles; ++j) issue(map, P, gi + j, j);
        }
        for (int tt = 0; tt < tiles; ++tt, ++gi) {
            const int b = (int)(gi % NBUF);
            const uint32_t par = (uint32_t)((gi / NBUF) & 1);
            if (t == 0 && !mbar_wait_bounded(&bars[b], par, max_wait)) {
                atomicOr(err_flag, 1);
                s_ok = 0;
                // wait (bounded) for this load and the ones issued after it
                for (int j = 0; j < NBUF - 1 && tt + j < tiles; ++j)
                    mbar_wait_bounded(&bars[(gi + j) % NBUF], (uint32_t)(((gi + j) / NBUF) & 1), max_wait);
                bulk_wait_all();
            }
            __syncthreads();
            if (!s_ok) return false;
            if (t == 0 && tt + NBUF - 1 < tiles) issue(map, P, gi + NBUF - 1, tt + NBUF - 1);
            u64 *tb = reinterpret_cast<u64 *>(buf + (size_t)b * (1 << LT));
            uint32_t pa, pb;
            tile_par(P, tt, pa, pb);
            if (P.rot[1] == 0 && (P.rot[2] & ~8u) == 0) ug_tile_l(tb, P, pa, pb, D, round2, m);
            else ug_tile(tb, P, pa ^ pa_t, pb ^ pb_t, D, round2, m);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (store && t == 0) {
                const long long tile = (slot << U.tiles_shift) | tt;
                tma_store_5d(map, tb, 0, 0, (int)(tile & ((1ll << P.mid_bits) - 1)), 0, (int)(tile >> P.mid_bits));
                bulk_commit();
            }
        }
        return true;
    };
    // block sums of the measured weights, FP64 per warp
    auto reduce3 = [&](float (&m)[3], double *dst) {
        for (int v = 0; v < 3; ++v) {
            double x = warp_sum((double)m[v]);
            if ((t & 31) == 0) mred[t >> 5][v] = x;
        }
        __syncthreads();
        if (t < 3) {
            double sum = 0.0;
            for (int w = 0; w < NT / 32; ++w) sum += mred[w][t];
            dst[t] = sum;
        }
        __syncthreads();
    };

    for (;;) {
        if (t == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        if (item >= U.n_points) {
            // ---- a 12-qubit point, on chip ----
            scan12_point<float>(item - U.n_points, buf, lut12, xus12, red, cpl12, sv, out12, P12);
            continue;
        }
        // ---- a unitary-gauge point on this CTA's slot ----
        const int pt = item;
        const DevCouplings c = cpl17[pt];
        // |+>^n: one tile of 2^-n/2, stored to every tile of the slot (pass-0 geometry)
        {
            float2 *tb = buf;
            const float a0 = rsqrtf((float)(1ll << U.n));
            if (t == 0) bulk_wait_all();
            __syncthreads();
            for (int i = t; i < (1 << LT); i += NT) tb[i] = make_float2(a0, 0.f);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (t == 0) {
                for (int tt = 0; tt < (1 << U.tiles_shift); ++tt) {
                    const long long tile = (slot << U.tiles_shift) | tt;
                    tma_store_5d(&tmap0, tb, 0, 0, (int)(tile & ((1ll << U.p0.mid_bits) - 1)), 0,
                                 (int)(tile >> U.p0.mid_bits));
                }
                bulk_commit();
            }
        }
        float mz[3] = {0.f, 0.f, 0.f}, mx[3] = {0.f, 0.f, 0.f}, dummy[3] = {0.f, 0.f, 0.f};
        bool ok = true;
        const DiagOps none{nullptr, nullptr, 1.f, false, 1.f};
        for (int op = 0; op < U.n_ops && ok; ++op) {
            // factor tables of this group
            double thx[2], zA, zB;
            bool has_z;
            dev_op_angles(U.G, &c, 0, sv, op, thx, &zA, &zB, &has_z);
            __syncthreads();                       // the previous group's tables are no longer read
            if (t <= U.nS) {                       // stars: exp(i th_tau (nS - 2a))
                float u, s; dev_unit_pair_fast<float>(thx[1] * (double)(U.nS - 2 * t), &u, &s); tXa[t] = make_float2(u, s);
            } else if (t >= 64 && t - 64 <= U.nL) {   // links: exp(i th_sigma (nL - 2b))
                const int k = t - 64;
                float u, s; dev_unit_pair_fast<float>(thx[0] * (double)(U.nL - 2 * k), &u, &s); tXb[k] = make_float2(u, s);
            } else if (t >= 128 && t - 128 <= U.nP) { // plaquettes: exp(i zA (nP - 2a))
                const int k = t - 128;
                float u, s; dev_unit_pair_fast<float>(has_z ? zA * (double)(U.nP - 2 * k) : 0.0, &u, &s);
                tZa[k] = make_float2(u, s);
            } else if (t >= 192 && t - 192 <= U.nL) { // sigma^z: exp(i zB (nL - 2b))
                const int k = t - 192;
                float u, s; dev_unit_pair_fast<float>(has_z ? zB * (double)(U.nL - 2 * k) : 0.0, &u, &s);
                tZb[k] = make_float2(u, s);
            }
            __syncthreads();
            if (op == 0) ok = ok && pass(&tmap0, U.p0, none, false, true, dummy);              // H(0..11)
            const DiagOps dx{tXa, tXb, U.scale, false, 1.f};
            ok = ok && pass(&tmap1, U.p1, dx, true, true, dummy);                          // H D_X H
            const bool last = op + 1 == U.n_ops;
            const DiagOps dz{has_z ? tZa : nullptr, tZb, 1.f, last, 1.f};
            ok = ok && pass(&tmap0, U.p0, dz, !last, true, mz);                            // H Z H'
        }
        // sigma^x and A_v: one more Walsh-Hadamard transform, weights 2^-n
        ok = ok && pass(&tmap0, U.p0, none, false, true, dummy);
        const DiagOps meas{nullptr, nullptr, 1.f, true, U.scale};
        ok = ok && pass(&tmap1, U.p1, meas, false, false, mx);
        if (!ok) return;
        __shared__ double sz[3], sx[3];
        reduce3(mz, sz);
        reduce3(mx, sx);
        if (t == 0) {
            // sz: norm, sum <B_p>, sum <sigma^z>; sx: norm, sum <A_v>, sum <sigma^x>
            const double e = -c.J * sx[1] - c.h * sz[1] - c.g * sx[2] - c.lambda * sz[2];
            double *o = out17 + (long long)pt * SCAN_NOBS;
            o[0] = e;
            o[1] = U.nP ? sz[1] / U.nP : 0.0;
            o[2] = 0.0;
            o[3] = 0.0;
            o[4] = sz[0];
            o[5] = U.nL ? sx[2] / U.nL : 0.0;
            o[6] = 0.0;
            o[7] = 0.0;
        }
    }
    if (t == 0) bulk_wait_all();          // the CTA's shared memory must outlive its stores
}

}  // namespace qsim
