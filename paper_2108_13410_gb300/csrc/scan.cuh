// scan.cuh -- phase-diagram scan of 12-qubit lattices in one persistent launch.
//
// Every (g, lambda) point is an independent adiabatic run (Sec. III) on a lattice
// of exactly 12 qubits (the 2x2 torus in the gauge-Higgs form).  A 4096-amplitude
// state fits one CTA's shared memory, so a CTA evolves a whole point on chip: the
// X layer as three register stages of four qubits (radix-16 butterflies, swizzled
// shared-memory transposes), the Z layer from a per-op phase table, all Trotter
// factor groups of the schedule, then the observables -- HBM is touched only for
// the couplings, the schedule and the results.  CTAs walk points
// blockIdx.x, +gridDim.x, ...
#pragma once
#include "kernels.cuh"

namespace qsim {

constexpr int SCAN_NOBS = 8;   // energy, <B_p> average, W_x, W_y, norm, <X> link avg, <X> vertex avg, 0

struct ScanParams {
    int n_points, n_ops;
    RecGeom G;                    // schedule geometry (batch = 1, tables sized nA x nB)
    int nA, nB;
    uint32_t colA[LT], colB[LT];  // parity columns of the 12 qubits
    unsigned cls_mask;            // bit q set: qubit q is a vertex (tau^x class)
    uint32_t wx, wy;              // Wilson-loop masks (0 if none)
    int n_link, n_vertex;
};

template <typename V, typename R>
__device__ __forceinline__ void scan_measure_pairs(const V (&v)[NR], int stage_base, unsigned cls_mask,
                                                   R &x0, R &x1) {
    // Re(conj(a) b) summed over the pairs of each register bit: half of <X_q>
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        R acc = 0;
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (!((r >> k) & 1)) acc += v[r].x * v[r | (1 << k)].x + v[r].y * v[r | (1 << k)].y;
        if ((cls_mask >> (stage_base + k)) & 1) x1 += acc; else x0 += acc;
    }
}

// One 12-qubit point for the whole schedule, on chip: `tile` is a 4096-amplitude
// shared-memory buffer (16-byte aligned), `lut` (at least nA + nB + 2 entries), `xus`,
// `red` small shared scratch.  The Z layer of a step is the product of two factors,
// exp(i zA (nA - 2 a)) exp(i zB (nB - 2 b)) for a odd plaquettes and b odd bonds, one
// table of nA + 1 and one of nB + 1 careful unit pairs, rebuilt every step with
// dev_unit_pair_fast (a table of (nA + 1)(nB + 1) entries with the 7 x 7 search took
// more FP64 time than the butterflies).
template <typename R>
__device__ void scan12_point(int pt, typename C2<R>::T *tile, typename C2<R>::T *lut, R *xus,
                             double (*red)[SCAN_NOBS], const DevCouplings *__restrict__ cpl,
                             const double *__restrict__ sv, double *__restrict__ out, const ScanParams &P) {
    using V = typename C2<R>::T;
    const int t = threadIdx.x;
    const int nB1 = P.nB + 1;
    const int tlo = t & 15, thi = t >> 4;
    // per-thread odd-term counts of the stage-C amplitudes (fixed for every op)
    uint8_t codeA[NR], codeB[NR];
    uint8_t wpar[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int l = tlo | (r << 4) | (thi << 8);
        uint32_t a = 0, b = 0;
#pragma unroll
        for (int q = 0; q < LT; ++q)
            if ((l >> q) & 1) { a ^= P.colA[q]; b ^= P.colB[q]; }
        codeA[r] = (uint8_t)__popc(a);
        codeB[r] = (uint8_t)(nB1 > 0 ? __popc(b) : 0);
        wpar[r] = (uint8_t)((__popc(l & P.wx) & 1) | ((__popc(l & P.wy) & 1) << 1));
    }
    V *lutA = lut, *lutB = lut + (P.nA + 1);
    int cls0[RB], cls1[RB], cls2[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        cls0[k] = (P.cls_mask >> (8 + k)) & 1;
        cls1[k] = (P.cls_mask >> k) & 1;
        cls2[k] = (P.cls_mask >> (4 + k)) & 1;
    }
    const R amp0 = (R)0.015625;   // 2^-6 = 1/sqrt(4096)

    const DevCouplings c = cpl[pt];
    __syncthreads();   // the caller's previous use of the shared buffers is over
    for (int i = t; i < (1 << LT); i += NT) tile[i] = mk<R>(amp0, (R)0);
    for (int op = 0; op < P.n_ops; ++op) {
        __syncthreads();   // previous op's tables and tile writes are done
        double thx[2], zA, zB;
        bool has_z;
        dev_op_angles(P.G, &c, 0, sv, op, thx, &zA, &zB, &has_z);
        if (t < 2) {
            R u, s;
            dev_unit_pair_fast<R>(thx[t], &u, &s);
            xus[2 * t] = u; xus[2 * t + 1] = s;
        } else if (has_z && t - 2 < P.nA + 1 + nB1) {
            const int k = t - 2;
            R u, s;
            if (k <= P.nA) {
                dev_unit_pair_fast<R>(zA * (double)(P.nA - 2 * k), &u, &s);
                lutA[k] = mk<R>(u, s);
            } else {
                dev_unit_pair_fast<R>(zB * (double)(P.nB - 2 * (k - P.nA - 1)), &u, &s);
                lutB[k - P.nA - 1] = mk<R>(u, s);
            }
        }
        __syncthreads();
        const R u0 = xus[0], s0 = xus[1], u1 = xus[2], s1 = xus[3];
        V v[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) v[r] = tile[swz(t | (r << TB))];
        rotate_regs<R>(v, 0xFu, cls0, u0, s0, u1, s1);
#pragma unroll
        for (int r = 0; r < NR; ++r) tile[swz(t | (r << TB))] = v[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < NR; ++r) v[r] = tile[swz(r | (t << RB))];
        rotate_regs<R>(v, 0xFu, cls1, u0, s0, u1, s1);
#pragma unroll
        for (int r = 0; r < NR; ++r) tile[swz(r | (t << RB))] = v[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < NR; ++r) v[r] = tile[swz(tlo | (r << 4) | (thi << 8))];
        rotate_regs<R>(v, 0xFu, cls2, u0, s0, u1, s1);
        if (has_z) {
#pragma unroll
            for (int r = 0; r < NR; ++r) v[r] = cphase(cphase(v[r], lutA[codeA[r]]), lutB[codeB[r]]);
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) tile[swz(tlo | (r << 4) | (thi << 8))] = v[r];
    }
    __syncthreads();
    // ---- observables: diagonal sums in stage-C layout, X pairs in all three ----
    R acc[SCAN_NOBS];
#pragma unroll
    for (int k = 0; k < SCAN_NOBS; ++k) acc[k] = 0;
    V v[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) v[r] = tile[swz(tlo | (r << 4) | (thi << 8))];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const R p = v[r].x * v[r].x + v[r].y * v[r].y;
        const int a = codeA[r], b = codeB[r];
        acc[1] += p * (R)(P.nA - 2 * a);
        acc[2] += (wpar[r] & 1) ? -p : p;
        acc[3] += (wpar[r] & 2) ? -p : p;
        acc[4] += p;
        acc[7] += p * (R)(P.nB - 2 * b);
    }
    scan_measure_pairs<V, R>(v, 4, P.cls_mask, acc[5], acc[6]);
#pragma unroll
    for (int r = 0; r < NR; ++r) v[r] = tile[swz(t | (r << TB))];
    scan_measure_pairs<V, R>(v, 8, P.cls_mask, acc[5], acc[6]);
#pragma unroll
    for (int r = 0; r < NR; ++r) v[r] = tile[swz(r | (t << RB))];
    scan_measure_pairs<V, R>(v, 0, P.cls_mask, acc[5], acc[6]);
    const int w = t >> 5;
#pragma unroll
    for (int k = 0; k < SCAN_NOBS; ++k) {
        double x = warp_sum((double)acc[k]);
        if ((t & 31) == 0) red[w][k] = x;
    }
    __syncthreads();
    if (t == 0) {
        double sum[SCAN_NOBS];
        for (int k = 0; k < SCAN_NOBS; ++k) {
            sum[k] = 0.0;
            for (int j = 0; j < NT / 32; ++j) sum[k] += red[j][k];
        }
        // sum[5], sum[6]: sum over pairs of Re(conj(a) b) = <X_q> / 2 summed per class
        const double xs = 2.0 * sum[5], xt = 2.0 * sum[6];
        const double e = -c.h * sum[1] - c.lambda * sum[7] - c.g * xs - c.J * xt;
        double *o = out + (long long)pt * SCAN_NOBS;
        o[0] = e;
        o[1] = P.nA ? sum[1] / P.nA : 0.0;
        o[2] = sum[2];
        o[3] = sum[3];
        o[4] = sum[4];
        o[5] = P.n_link ? xs / P.n_link : 0.0;
        o[6] = P.n_vertex ? xt / P.n_vertex : 0.0;
        o[7] = 0.0;
    }
}

template <typename R>
__global__ void __launch_bounds__(NT, 2) k_scan12(const DevCouplings *__restrict__ cpl, const double *__restrict__ sv,
                                               double *__restrict__ out, const __grid_constant__ ScanParams P) {
    using V = typename C2<R>::T;
    __shared__ __align__(16) V tile[1 << LT];
    __shared__ V lut[64];
    __shared__ R xus[4];
    __shared__ double red[NT / 32][SCAN_NOBS];
    for (int pt = blockIdx.x; pt < P.n_points; pt += gridDim.x)
        scan12_point<R>(pt, tile, lut, xus, red, cpl, sv, out, P);
}

}  // namespace qsim
