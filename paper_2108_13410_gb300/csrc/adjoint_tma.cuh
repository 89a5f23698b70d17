// adjoint_tma.cuh -- persistent, TMA-fed reverse pass of the adjoint gradient (complex64).
//
// The reverse sweep of adjoint.cuh with both states streamed by TMA: each tile buffer
// holds the psi tile and the lambda tile (two 5-D tensor-map loads, one mbarrier).  The
// sweep runs in the real-rotation frame phi = i^popc psi (both states converted on the
// first reverse pass, psi converted back on the last), where the inverse factor is the
// real rotation [[c, -s], [s, c]] (packed FP32x2 FMAs) and the X-group derivative term
//     Im<lambda|X_q|psi> = Im<lambda_phi|Y_q|psi_phi> = sum_pairs Re(conj(l_b) p_a) - Re(conj(l_a) p_b).
// The first reverse pass of a factor group undoes the Z layer in stage A (before any
// X term of the group is read) and accumulates the Z-group terms
//     Im(conj(lambda_i) psi_i) (nA - 2 oddA(i)),  ... (nB - 2 oddB(i)).
#pragma once
#include "xpass_tma.cuh"

namespace qsim {

__device__ __forceinline__ float rdot(u64 a, u64 b) {   // Re(conj(a) b) for packed complex
    const float2 x = unpk(a), y = unpk(b);
    return x.x * y.x + x.y * y.y;
}

__device__ __forceinline__ float warp_sum_f(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ float idot(u64 l, u64 p) {   // Im(conj(l) p)
    const float2 x = unpk(l), y = unpk(p);
    return x.x * y.y - x.y * y.x;
}

// reverse real-frame rotations on psi and lambda with the X-group terms read first
__device__ __forceinline__ void adj_rotate_w(u64 (&p)[NR], u64 (&l)[NR], unsigned mask, const int (&cls)[RB],
                                             const RotConst &C, float &g0, float &g1) {
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        if (!((mask >> k) & 1u)) continue;
        const bool c = cls[k] != 0;
        // inverse rotation: s -> -s
        const u64 nu = c ? C.nu[1] : C.nu[0], ps = c ? C.ns[1] : C.ns[0], ns = c ? C.ps[1] : C.ps[0];
        float g = 0.f;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if ((r >> k) & 1) continue;
            const int q = r | (1 << k);
            g += rdot(l[q], p[r]) - rdot(l[r], p[q]);
            rrotp(p[r], p[q], nu, ps, ns);
            rrotp(l[r], l[q], nu, ps, ns);
        }
        if (c) g1 += g; else g0 += g;
    }
}

// Tangent form (records from dev_tan_triple): the inverse factor is cos th [[1, -t],
// [t, 1]]; C = prod cos th is applied first (with the inverse Z layer, through the
// conjugated scaled table, or alone for a group without Z), so when stage s reads its
// terms psi and lambda both still carry prod cos th over the X qubits not yet
// un-rotated; corr = prod (1 + t^2) over those qubits (= 1 / that product squared)
// restores the terms.  corr is the value at the start of the stage and drops by
// qi = 1 / (1 + t^2) of each qubit the stage un-rotates before reading the next one.
// The pair products are accumulated as packed FP32x2 FMAs.
__device__ __forceinline__ void adj_rotate_t(u64 (&p)[NR], u64 (&l)[NR], unsigned mask, const int (&cls)[RB],
                                             const TanConst &C, float corr, float qi0, float qi1, float &g0,
                                             float &g1) {
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        if (!((mask >> k) & 1u)) continue;
        const bool c = cls[k] != 0;
        const u64 pt = c ? C.pt[1] : C.pt[0], nt = c ? C.nt[1] : C.nt[0];
        u64 accp = 0ull, accm = 0ull;   // (+0.0f, +0.0f)
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if ((r >> k) & 1) continue;
            const int q = r | (1 << k);
            accp = fma2p(l[q], p[r], accp);
            accm = fma2p(l[r], p[q], accm);
            const u64 pa = p[r], pb = p[q], la = l[r], lb = l[q];
            p[r] = fma2p(nt, pb, pa);
            p[q] = fma2p(pt, pa, pb);
            l[r] = fma2p(nt, lb, la);
            l[q] = fma2p(pt, la, lb);
        }
        const float2 sp = unpk(accp), sm = unpk(accm);
        const float g = ((sp.x + sp.y) - (sm.x + sm.y)) * corr;
        if (c) g1 += g; else g0 += g;
        corr *= c ? qi1 : qi0;
    }
}

// Tangent form with the constants of each register bit read from a shared-memory table:
// tc[k] = {(t, t), (-t, -t)} of the class of bit k, qi[k] = 1 / (1 + t^2) of that class;
// corr is the scale correction at the start of the stage.  Terms of bits of class 1
// (cls bit k set) go to g1, the others to g0.
__device__ __forceinline__ void adj_rotate_ts(u64 (&p)[NR], u64 (&l)[NR], unsigned mask, unsigned cls,
                                              const u64 (*tc)[2], const float *qi, float corr, float &g0,
                                              float &g1) {
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        if (!((mask >> k) & 1u)) continue;
        const u64 pt = tc[k][0], nt = tc[k][1];
        u64 accp = 0ull, accm = 0ull;   // (+0.0f, +0.0f)
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if ((r >> k) & 1) continue;
            const int q = r | (1 << k);
            accp = fma2p(l[q], p[r], accp);
            accm = fma2p(l[r], p[q], accm);
            const u64 pa = p[r], pb = p[q], la = l[r], lb = l[q];
            p[r] = fma2p(nt, pb, pa);
            p[q] = fma2p(pt, pa, pb);
            l[r] = fma2p(nt, lb, la);
            l[q] = fma2p(pt, la, lb);
        }
        const float2 sp = unpk(accp), sm = unpk(accm);
        const float g = ((sp.x + sp.y) - (sm.x + sm.y)) * corr;
        if ((cls >> k) & 1u) g1 += g; else g0 += g;
        corr *= qi[k];
    }
}

__device__ __forceinline__ void adj_rotate(u64 (&p)[NR], u64 (&l)[NR], unsigned mask, const int (&cls)[RB],
                                           const RotConst &C, float, float, float, float &g0, float &g1) {
    adj_rotate_w(p, l, mask, cls, C, g0, g1);
}
__device__ __forceinline__ void adj_rotate(u64 (&p)[NR], u64 (&l)[NR], unsigned mask, const int (&cls)[RB],
                                           const TanConst &C, float corr, float qi0, float qi1, float &g0,
                                           float &g1) {
    adj_rotate_t(p, l, mask, cls, C, corr, qi0, qi1, g0, g1);
}

// MERGED (tangent form only): a shared reverse pass over one qubit group G.  Round 1
// un-rotates X(G) of factor group j (terms to partials at slot0), then the Z layer of
// group j-1 is undone in the stage-C layout (its terms and its scaled table, recs2), and
// round 2 un-rotates X(G) of group j-1 in stages C, B, A (terms to partials2 at slot0b)
// and stores from the stage-A layout.  Mirrors the shared passes of the forward sweep.
// Both tiles go back to HBM by bulk tensor stores from shared memory.  In the tangent
// form the per-bit constants (t, -t), the 1 / (1 + t^2) factors and the per-stage scale
// corrections of both rounds sit in a small shared-memory table (broadcast reads), which
// keeps the kernel within 128 registers: two CTAs per SM with one tile-pair buffer each.
template <int NBUF, bool TAN, bool MERGED, bool EARLY>
__global__ void __launch_bounds__(NT, NBUF == 1 ? 2 : 1) k_adj_tma(float2 *__restrict__ psi, float2 *__restrict__ lam,
                                                   const double *__restrict__ recs, int rec_stride, int tiles_shift,
                                                   int *__restrict__ err_flag, double *__restrict__ partials,
                                                   int nblk, int slot0, int zinv,
                                                   const double *__restrict__ recs2,
                                                   double *__restrict__ partials2, int slot0b,
                                                   const __grid_constant__ CUtensorMap tmap_p,
                                                   const __grid_constant__ CUtensorMap tmap_l,
                                                   const __grid_constant__ TmaPass P) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base_ptr = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float2 *buf = reinterpret_cast<float2 *>(base_ptr);                       // NBUF x (psi, lambda) tiles
    float2 *lut = buf + 2 * NBUF * (1 << LT);
    uint2 *ptab = reinterpret_cast<uint2 *>(lut + (P.nA + 1) * (P.nB + 1));  // 3 x 256
    __shared__ uint64_t bars[NBUF];
    __shared__ int s_ok;
    __shared__ double red[NT / 32][8];
    __shared__ u64 s_tc[2][3][RB][2];     // TAN: per round, stage and register bit: (t,t), (-t,-t)
    __shared__ float s_qi[2][3][RB];      // TAN: 1 / (1 + t^2) of that bit's class
    __shared__ float s_corr[2][3];        // TAN: scale correction at the start of each stage
    __shared__ float s_xs;                // TAN: C of the factor group (groups without Z layer)

    const int t = threadIdx.x;
    const long long G = gridDim.x;
    const long long T = P.total_tiles;
    const long long first = blockIdx.x;
    const long long max_wait = 2000000000ll;

    if (t == 0) {
        for (int b = 0; b < NBUF; ++b) mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
    for (int e = t; e < 3 * 256; e += NT) {
        int byte = e >> 8, val = e & 255;
        uint32_t a = 0, b = 0;
        for (int j = 0; j < 8; ++j) {
            int bit = 8 * byte + j;
            if (bit < P.tile_bits && ((val >> j) & 1)) { a ^= P.pa_tile[bit]; b ^= P.pb_tile[bit]; }
        }
        ptab[e] = make_uint2(a, b);
    }
    __syncthreads();

    auto issue = [&](int it) {
        long long tile = first + (long long)it * G;
        int b = it % NBUF;
        int x2 = (int)(tile & ((1ll << P.mid_bits) - 1));
        int x4 = (int)(tile >> P.mid_bits);
        bulk_wait_read_all();                // a store may still be reading this buffer
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&bars[b], 2 * TMA_TILE_BYTES);
        tma_load_5d(buf + (size_t)(2 * b) * (1 << LT), &tmap_p, &bars[b], 0, 0, x2, 0, x4);
        tma_load_5d(buf + (size_t)(2 * b + 1) * (1 << LT), &tmap_l, &bars[b], 0, 0, x2, 0, x4);
    };
    const int n_my = first < T ? (int)((T - first + G - 1) / G) : 0;
    if (t == 0)
        for (int it = 0; it < NBUF - 1 && it < n_my; ++it) issue(it);

    const int tlo = t & 15, thi = t >> 4;
    const int a_base = swz128(t);
    const int b_base = t << 3, b_x = t & 7;
    uint32_t paA_t = 0, pbA_t = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        if ((t >> j) & 1) { paA_t ^= P.paA_thr[j]; pbA_t ^= P.pbA_thr[j]; }
    const int nB1 = P.nB + 1, nlut = (P.nA + 1) * nB1;
    uint32_t paC_t = 0, pbC_t = 0;                   // MERGED: stage-C thread parity columns
    if (MERGED) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if ((tlo >> j) & 1) { paC_t ^= P.pa_thr[j]; pbC_t ^= P.pb_thr[j]; }
            if ((thi >> j) & 1) { paC_t ^= P.pa_thr[4 + j]; pbC_t ^= P.pb_thr[4 + j]; }
        }
    }
    // stage-C shared-memory index of register r (128-byte swizzle)
    auto c_idx = [&](int r) { return ((tlo ^ ((r & 7) << 1)) | (thi << 8)) + (r << 4); };
    const long long tmask = (1ll << tiles_shift) - 1;
    long long cur_batch = -1;
    RotConst RC;                     // !TAN: (u, s) constants in registers
    int cls0[RB], cls1[RB], cls2[RB];
#pragma unroll
    for (int kk = 0; kk < RB; ++kk) {
        cls0[kk] = (P.cls[0] >> kk) & 1; cls1[kk] = (P.cls[1] >> kk) & 1; cls2[kk] = (P.cls[2] >> kk) & 1;
    }
    constexpr int NV = MERGED ? 8 : 4;
    // FP64 block sums of one batch element accumulate in per-warp shared-memory slots
    // (red[w][v], lane 0 of warp w adds the warp's per-tile float sum), so no FP64
    // accumulator occupies registers across tiles
    for (int e = t; e < (NT / 32) * 8; e += NT) red[e / 8][e % 8] = 0.0;
    auto add_tile = [&](int v, float x) {
        x = warp_sum_f(x);
        if ((t & 31) == 0) red[t >> 5][v] += (double)x;
    };
    // plain reverse passes: each lane keeps float sums of its four terms over eight tiles,
    // then the warp sums them into its FP64 slots (one FP64 add per value per eight tiles)
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    int n_acc = 0;
    auto flush_acc = [&]() {
#pragma unroll
        for (int v = 0; v < 4; ++v) { add_tile(v, acc[v]); acc[v] = 0.f; }
        n_acc = 0;
    };
    // values 0..3 to partials, 4..7 (MERGED) to partials2
    auto flush = [&](long long bat) {
        __syncthreads();
        if (t < NV) {
            double sum = 0.0;
            for (int w = 0; w < NT / 32; ++w) sum += red[w][t];
            if (t < 4) partials[(bat * nblk + slot0 + blockIdx.x) * RED_NV + t] = sum;
            else partials2[(bat * nblk + slot0b + blockIdx.x) * RED_NV + (t - 4)] = sum;
        }
        __syncthreads();
        for (int e = t; e < (NT / 32) * 8; e += NT) red[e / 8][e % 8] = 0.0;
    };
    // one un-rotation stage on both tiles (table-driven in the tangent form)
    auto unrot = [&](int round, int st, const int (&cls)[RB], float &g0, float &g1, u64 (&p)[NR], u64 (&l)[NR]) {
        if (TAN) adj_rotate_ts(p, l, P.rot[st], P.cls[st], s_tc[round][st], s_qi[round][st], s_corr[round][st], g0, g1);
        else adj_rotate_w(p, l, P.rot[st], cls, RC, g0, g1);
    };

    // EARLY (one buffer): the next tile pair is loaded as soon as every thread has read the
    // last stage of the current one from shared memory; both tiles then go back to HBM by
    // per-thread stores from registers while the load is in flight
    auto issue_next = [&](int it) {
        if (EARLY) {
            __syncthreads();
            if (t == 0 && it + 1 < n_my) issue(it + 1);
        }
    };
    long long toff_c = 0, toff_a = 0;   // EARLY: stage-C and stage-A global offsets of this thread
    if (EARLY) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if ((tlo >> j) & 1) toff_c += P.toff_c[j];
            if ((thi >> j) & 1) toff_c += P.toff_c[4 + j];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if ((t >> j) & 1) toff_a += P.toff_a[j];
    }
    long long tile = first;
    for (int it = 0; it < n_my; ++it, tile += G) {
        const int b = it % NBUF;
        const uint32_t parity = (uint32_t)((it / NBUF) & 1);
        const long long batch = tile >> tiles_shift;
        if (batch != cur_batch) {
            if (!MERGED && n_acc) flush_acc();
            if (cur_batch >= 0) flush(cur_batch);   // the previous batch element's sums
            __syncthreads();
            const double *rec = recs + batch * rec_stride;
            if (!TAN) load_xconst(RC, rec, P.tan_off);
            if (TAN && t < 2 * 3 * RB) {
                // round 0: this factor group (stages A, B, C), round 1 (MERGED): the
                // previous one (stages C, B, A); inverse factor: a' = a - t b, b' = b + t a
                const int round = t / (3 * RB), st = (t / RB) % 3, k = t % RB;
                if (round == 0 || MERGED) {
                    const double *rr = round ? recs2 + batch * rec_stride : rec;
                    const int c = (P.cls[st] >> k) & 1;
                    const double tv = rr[P.tan_off + c];
                    s_tc[round][st][k][0] = pk((float)tv, (float)tv);
                    s_tc[round][st][k][1] = pk(-(float)tv, -(float)tv);
                    s_qi[round][st][k] = (float)(1.0 / (1.0 + tv * tv));
                    if (k == 0) {
                        const double q0 = 1.0 + rr[P.tan_off] * rr[P.tan_off];
                        const double q1 = 1.0 + rr[P.tan_off + 1] * rr[P.tan_off + 1];
                        const int *u = round ? P.adj_u2[st] : P.adj_u[st];
                        s_corr[round][st] = (float)(pow(q0, (double)u[0]) * pow(q1, (double)u[1]));
                    }
                }
            }
            if (TAN && t == 0) s_xs = (float)rec[P.tan_off + 2];
            if (zinv) {   // inverse Z layer: conjugated phase table (tangent form: scaled by C)
                const int loff = TAN ? P.tan_off + 4 : 4;
                for (int i = t; i < nlut; i += NT)
                    lut[i] = make_float2((float)rec[loff + 2 * i], -(float)rec[loff + 2 * i + 1]);
            }
            if (MERGED) {   // the previous factor group's scaled Z table
                const double *rec2 = recs2 + batch * rec_stride;
                for (int i = t; i < nlut; i += NT)
                    lut[i] = make_float2((float)rec2[P.tan_off + 4 + 2 * i], -(float)rec2[P.tan_off + 5 + 2 * i]);
            }
            cur_batch = batch;
            __syncthreads();
        }
        if (NBUF == 1 && !(EARLY && it > 0)) {
            __syncthreads();                 // the single buffer is free again
            if (t == 0) issue(it);
        }
        if (t == 0) {
            if (!mbar_wait_bounded(&bars[b], parity, max_wait)) {
                atomicOr(err_flag, 1);
                s_ok = 0;
                for (int j = it + 1; j < it + NBUF - 1 && j < n_my; ++j)
                    mbar_wait_bounded(&bars[j % NBUF], (uint32_t)((j / NBUF) & 1), max_wait);
                bulk_wait_all();
            }
        }
        __syncthreads();
        if (!s_ok) return;
        if (NBUF > 1 && t == 0 && it + NBUF - 1 < n_my) issue(it + NBUF - 1);

        u64 *tp = reinterpret_cast<u64 *>(buf + (size_t)(2 * b) * (1 << LT));
        u64 *tl = reinterpret_cast<u64 *>(buf + (size_t)(2 * b + 1) * (1 << LT));
        u64 p[NR], l[NR];
        float g0 = 0.f, g1 = 0.f, ga = 0.f, gb = 0.f;
        const long long tin = tile & tmask;
        const int pc_tile = __popcll(tin);
        // ---- stage A ----
#pragma unroll
        for (int r = 0; r < NR; ++r) { p[r] = tp[a_base + (r << TB)]; l[r] = tl[a_base + (r << TB)]; }
        if (zinv) {
            const uint2 e0 = ptab[tin & 255], e1 = ptab[256 + ((tin >> 8) & 255)], e2 = ptab[512 + ((tin >> 16) & 255)];
            const uint32_t pa = paA_t ^ e0.x ^ e1.x ^ e2.x, pb = pbA_t ^ e0.y ^ e1.y ^ e2.y;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int oa = __popc(pa ^ P.paA_reg[r]), ob = __popc(pb ^ P.pbA_reg[r]);
                const float im = idot(l[r], p[r]);
                ga += im * (float)(P.nA - 2 * oa);
                gb += im * (float)(P.nB - 2 * ob);
                const float2 ph = lut[oa * nB1 + ob];
                const float2 vp = cphase(unpk(p[r]), ph), vl = cphase(unpk(l[r]), ph);
                p[r] = pk(vp.x, vp.y);
                l[r] = pk(vl.x, vl.y);
            }
        }
        if (TAN && !zinv && P.xscale) {   // C of a factor group without Z layer
            const float xs = s_xs;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float2 vp = unpk(p[r]), vl = unpk(l[r]);
                p[r] = pk(vp.x * xs, vp.y * xs);
                l[r] = pk(vl.x * xs, vl.y * xs);
            }
        }
        if (P.frame & 2) {
            const int k0 = __popc(t) + pc_tile;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float2 vp = mul_ipow(unpk(p[r]), k0 + __popc(r)), vl = mul_ipow(unpk(l[r]), k0 + __popc(r));
                p[r] = pk(vp.x, vp.y);
                l[r] = pk(vl.x, vl.y);
            }
        }
        unrot(0, 0, cls0, g0, g1, p, l);
#pragma unroll
        for (int r = 0; r < NR; ++r) { tp[a_base + (r << TB)] = p[r]; tl[a_base + (r << TB)] = l[r]; }
        __syncthreads();
        // ---- stage B ----
        if (P.stage_b) {
            ulonglong2 *tp2 = reinterpret_cast<ulonglong2 *>(tp), *tl2 = reinterpret_cast<ulonglong2 *>(tl);
#pragma unroll
            for (int m = 0; m < NR / 2; ++m) {
                const ulonglong2 qp = tp2[b_base + (m ^ b_x)], ql = tl2[b_base + (m ^ b_x)];
                p[2 * m] = qp.x; p[2 * m + 1] = qp.y;
                l[2 * m] = ql.x; l[2 * m + 1] = ql.y;
            }
            unrot(0, 1, cls1, g0, g1, p, l);
#pragma unroll
            for (int m = 0; m < NR / 2; ++m) {
                tp2[b_base + (m ^ b_x)] = make_ulonglong2(p[2 * m], p[2 * m + 1]);
                tl2[b_base + (m ^ b_x)] = make_ulonglong2(l[2 * m], l[2 * m + 1]);
            }
            __syncthreads();
        }
        // ---- stage C ----
#pragma unroll
        for (int r = 0; r < NR; ++r) { p[r] = tp[c_idx(r)]; l[r] = tl[c_idx(r)]; }
        if (!MERGED) issue_next(it);
        unrot(0, 2, cls2, g0, g1, p, l);
        if (P.frame & 4) {
            const int k0 = -(__popc(tlo) + __popc(thi) + pc_tile);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int kk = (k0 - __popc(r)) & 3;
                const float2 vp = mul_ipow(unpk(p[r]), kk), vl = mul_ipow(unpk(l[r]), kk);
                p[r] = pk(vp.x, vp.y);
                l[r] = pk(vl.x, vl.y);
            }
        }
        if (MERGED) {
            // ---- the previous factor group's Z layer, undone in the stage-C layout ----
            float g0b = 0.f, g1b = 0.f, ga2 = 0.f, gb2 = 0.f;
            {
                const uint2 e0 = ptab[tin & 255], e1 = ptab[256 + ((tin >> 8) & 255)], e2 = ptab[512 + ((tin >> 16) & 255)];
                const uint32_t pa = paC_t ^ e0.x ^ e1.x ^ e2.x, pb = pbC_t ^ e0.y ^ e1.y ^ e2.y;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int oa = __popc(pa ^ P.pa_reg[r]), ob = __popc(pb ^ P.pb_reg[r]);
                    const float im = idot(l[r], p[r]);
                    ga2 += im * (float)(P.nA - 2 * oa);
                    gb2 += im * (float)(P.nB - 2 * ob);
                    const float2 ph = lut[oa * nB1 + ob];
                    const float2 vp = cphase(unpk(p[r]), ph), vl = cphase(unpk(l[r]), ph);
                    p[r] = pk(vp.x, vp.y);
                    l[r] = pk(vl.x, vl.y);
                }
            }
            // ---- round 2: the previous factor group's X on the same qubits, stages C, B, A ----
            unrot(1, 2, cls2, g0b, g1b, p, l);
#pragma unroll
            for (int r = 0; r < NR; ++r) { tp[c_idx(r)] = p[r]; tl[c_idx(r)] = l[r]; }
            __syncthreads();
            if (P.stage_b) {
                ulonglong2 *tp2 = reinterpret_cast<ulonglong2 *>(tp), *tl2 = reinterpret_cast<ulonglong2 *>(tl);
#pragma unroll
                for (int m = 0; m < NR / 2; ++m) {
                    const ulonglong2 qp = tp2[b_base + (m ^ b_x)], ql = tl2[b_base + (m ^ b_x)];
                    p[2 * m] = qp.x; p[2 * m + 1] = qp.y;
                    l[2 * m] = ql.x; l[2 * m + 1] = ql.y;
                }
                unrot(1, 1, cls1, g0b, g1b, p, l);
#pragma unroll
                for (int m = 0; m < NR / 2; ++m) {
                    tp2[b_base + (m ^ b_x)] = make_ulonglong2(p[2 * m], p[2 * m + 1]);
                    tl2[b_base + (m ^ b_x)] = make_ulonglong2(l[2 * m], l[2 * m + 1]);
                }
                __syncthreads();
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) { p[r] = tp[a_base + (r << TB)]; l[r] = tl[a_base + (r << TB)]; }
            issue_next(it);
            unrot(1, 0, cls0, g0b, g1b, p, l);
            if (EARLY) {
                const long long mid = tile & ((1ll << P.mid_bits) - 1), up = tile >> P.mid_bits;
                const long long gbase = (mid << P.c) + (up << (P.next + P.k)) + toff_a;
                u64 *dp = reinterpret_cast<u64 *>(psi + gbase);
                u64 *dl = reinterpret_cast<u64 *>(lam + gbase);
#pragma unroll
                for (int r = 0; r < NR; ++r) { dp[P.roff_a[r]] = p[r]; dl[P.roff_a[r]] = l[r]; }
            } else {
                // back into the stage-A positions of the swizzled tiles
#pragma unroll
                for (int r = 0; r < NR; ++r) { tp[a_base + (r << TB)] = p[r]; tl[a_base + (r << TB)] = l[r]; }
            }
            add_tile(0, g0); add_tile(1, g1);
            add_tile(4, g0b); add_tile(5, g1b); add_tile(6, ga2); add_tile(7, gb2);
        } else {
            if (EARLY) {
                const long long mid = tile & ((1ll << P.mid_bits) - 1), up = tile >> P.mid_bits;
                const long long gbase = (mid << P.c) + (up << (P.next + P.k)) + toff_c;
                u64 *dp = reinterpret_cast<u64 *>(psi + gbase);
                u64 *dl = reinterpret_cast<u64 *>(lam + gbase);
#pragma unroll
                for (int r = 0; r < NR; ++r) { dp[P.roff_c[r]] = p[r]; dl[P.roff_c[r]] = l[r]; }
            } else {
#pragma unroll
                for (int r = 0; r < NR; ++r) { tp[c_idx(r)] = p[r]; tl[c_idx(r)] = l[r]; }
            }
            acc[0] += g0; acc[1] += g1; acc[2] += ga; acc[3] += gb;
            if (++n_acc == 8) flush_acc();
        }
        if (EARLY) continue;
        // both tiles back to HBM by bulk tensor stores (same maps and boxes as the loads)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            const int x2 = (int)(tile & ((1ll << P.mid_bits) - 1));
            const int x4 = (int)(tile >> P.mid_bits);
            tma_store_5d(&tmap_p, tp, 0, 0, x2, 0, x4);
            tma_store_5d(&tmap_l, tl, 0, 0, x2, 0, x4);
            bulk_commit();
        }
    }
    if (!MERGED && n_acc) flush_acc();
    if (cur_batch >= 0) flush(cur_batch);   // the last batch element's sums
    if (t == 0) bulk_wait_all();            // the CTA's shared memory must outlive its stores
}

}  // namespace qsim
