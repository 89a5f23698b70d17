// adjoint_wl.cuh -- shared reverse pass of the adjoint gradient with warp-local slices
// (complex64, tangent form; sm_103a).
//
// Same operator and terms as k_adj_tma<.., TAN = true, MERGED = true, ..>: on the pass's
// qubit group G, round 1 un-rotates X(G) of factor group j (derivative terms of its two
// X classes), then the Z layer of group j-1 is undone (its two Z-class terms), and round
// 2 un-rotates X(G) of group j-1 (its X terms), on psi and lambda together.  As in the
// warp-local forward pass (xpass_wl.cuh), when every rotated qubit sits on tile bits
// 4..11 a tile splits into eight 512-amplitude slices that never exchange data: one warp
// takes the psi and lambda slices of one item through both rounds (registers local
// {8..11} in layout L1, {4..7} in layout L2, passing through the slice's own shared-
// memory slots), a producer thread issues the TMA loads and bulk stores of both tiles of
// a pair over NBUF pooled pair buffers.  Each lane keeps float sums of the six terms
// over its amplitudes of eight consecutive items (one tile's worth, 4096 amplitudes per
// warp); then the warp sums them (shuffles) and lane 0 adds them to the warp's FP64
// slots, so FP64 work is one add per value per eight items.  The CTA's FP64 sums go to
// the same partial-sum slots as k_adj_tma's.
#pragma once
#include "adjoint_tma.cuh"
#include "xpass_wl.cuh"

namespace qsim {

// NBUF pair buffers, NW warps (NW - 1 consumers), MINB CTAs per SM; DEFER 1: a buffer
// is reloaded when the tile after its own has completed, 0: once its own store has read it.
template <int NBUF, int NW, int MINB, int DEFER>
__global__ void __launch_bounds__(32 * NW, MINB) k_adj_wl(float2 *__restrict__ psi, float2 *__restrict__ lam,
                                                        const double *__restrict__ recs, int rec_stride,
                                                        int tiles_shift, int *__restrict__ err_flag,
                                                        double *__restrict__ partials, int nblk, int slot0,
                                                        int zinv, const double *__restrict__ recs2,
                                                        double *__restrict__ partials2, int slot0b,
                                                        const __grid_constant__ CUtensorMap tmap_p,
                                                        const __grid_constant__ CUtensorMap tmap_l,
                                                        const __grid_constant__ TmaPass P) {
    (void)psi; (void)lam; (void)rec_stride; (void)tiles_shift; (void)zinv;
    constexpr int NTH = 32 * NW, NC = NW - 1;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base_ptr = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    float2 *buf = reinterpret_cast<float2 *>(base_ptr);                       // NBUF x (psi, lambda) tiles
    float2 *lut = buf + 2 * NBUF * (1 << LT);
    uint2 *ptab = reinterpret_cast<uint2 *>(lut + (P.nA + 1) * (P.nB + 1));  // 3 x 256
    __shared__ uint64_t full[NBUF], done[NBUF];
    __shared__ int s_stamp[NBUF];
    __shared__ int s_abort;
    __shared__ double red[NW][8];
    __shared__ u64 s_tc[2][3][RB][2];
    __shared__ float s_qi[2][3][RB];
    __shared__ float s_corr[2][3];

    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const int G = (int)gridDim.x;
    const int T = (int)P.total_tiles;
    const int first = (int)blockIdx.x;
    const long long max_wait = 2000000000ll;
    volatile int *abort_flag = &s_abort;
    volatile int *stamp = s_stamp;

    if (t == 0) {
        for (int b = 0; b < NBUF; ++b) { mbar_init(&full[b], 1); mbar_init(&done[b], 8); s_stamp[b] = -1; }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    for (int e = t; e < 3 * 256; e += NTH) {
        int byte = e >> 8, val = e & 255;
        uint32_t a = 0, b = 0;
        for (int j = 0; j < 8; ++j) {
            int bit = 8 * byte + j;
            if (bit < P.tile_bits && ((val >> j) & 1)) { a ^= P.pa_tile[bit]; b ^= P.pb_tile[bit]; }
        }
        ptab[e] = make_uint2(a, b);
    }
    for (int e = t; e < NW * 8; e += NTH) red[e / 8][e % 8] = 0.0;
    // records of the single batch element: round 0 this factor group (stages A, C),
    // round 1 the previous one (stages C, A); inverse factor a' = a - t b, b' = b + t a
    if (t < 2 * 3 * RB) {
        const int round = t / (3 * RB), st = (t / RB) % 3, k = t % RB;
        const double *rr = round ? recs2 : recs;
        const double tv = rr[P.tan_off + ((P.cls[st] >> k) & 1)];
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
    const int nB1 = P.nB + 1, nlut = (P.nA + 1) * nB1;
    for (int i = t; i < nlut; i += NTH)   // the previous factor group's scaled Z table, conjugated
        lut[i] = make_float2((float)recs2[P.tan_off + 4 + 2 * i], -(float)recs2[P.tan_off + 5 + 2 * i]);
    __syncthreads();

    const int n_my = first < T ? (T - first + G - 1) / G : 0;
    const int mid_mask = (1 << P.mid_bits) - 1;
    auto issue_load = [&](int j) {
        const int tile = first + j * G;
        const int b = j % NBUF;
        stamp[b] = j;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&full[b], 2 * TMA_TILE_BYTES);
        tma_load_5d(buf + (size_t)(2 * b) * (1 << LT), &tmap_p, &full[b], 0, 0, tile & mid_mask, 0, tile >> P.mid_bits);
        tma_load_5d(buf + (size_t)(2 * b + 1) * (1 << LT), &tmap_l, &full[b], 0, 0, tile & mid_mask, 0,
                    tile >> P.mid_bits);
    };

    if (warp == NC) {
        // ---------------- producer ----------------
        if (lane == 0) {
            int issued = 0;
            for (; issued < NBUF && issued < n_my; ++issued) issue_load(issued);
            for (int j = 0; j < n_my; ++j) {
                const int b = j % NBUF;
                if (!mbar_wait_or_abort(&done[b], (uint32_t)((j / NBUF) & 1), max_wait, abort_flag)) {
                    atomicOr(err_flag, 1);
                    *abort_flag = 1;
                    break;
                }
                const int tile = first + j * G;
                tma_store_5d(&tmap_p, buf + (size_t)(2 * b) * (1 << LT), 0, 0, tile & mid_mask, 0, tile >> P.mid_bits);
                tma_store_5d(&tmap_l, buf + (size_t)(2 * b + 1) * (1 << LT), 0, 0, tile & mid_mask, 0,
                             tile >> P.mid_bits);
                bulk_commit();
                if (j >= DEFER && j - DEFER + NBUF < n_my) {
                    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(DEFER) : "memory");
                    issue_load(j - DEFER + NBUF);
                    ++issued;
                }
            }
            for (int j = issued - NBUF < 0 ? 0 : issued - NBUF; j < issued; ++j)
                mbar_wait_bounded(&full[j % NBUF], (uint32_t)((j / NBUF) & 1), max_wait);
            bulk_wait_all();
        }
        __syncwarp();
    } else {
        // ---------------- consumers ----------------
        const int l0 = lane & 1, lh = lane >> 1;
        uint32_t pa_lane = 0, pb_lane = 0;   // stage-C parity columns of the L2 lane bits
        if (l0) { pa_lane ^= P.pa_thr[0]; pb_lane ^= P.pb_thr[0]; }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if ((lh >> j) & 1) { pa_lane ^= P.pa_thr[4 + j]; pb_lane ^= P.pb_thr[4 + j]; }
        const int n_items = 8 * n_my;
        float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // g0, g1, g0b, g1b, ga2, gb2
        int since_flush = 0;
        auto flush_terms = [&]() {
            const int slot[6] = {0, 1, 4, 5, 6, 7};
#pragma unroll
            for (int v = 0; v < 6; ++v) {
                const float x = warp_sum_f(acc[v]);
                if (lane == 0) red[warp][slot[v]] += (double)x;
                acc[v] = 0.f;
            }
        };
        for (int item = warp; item < n_items; item += NC) {
            const int j = item >> 3, w = item & 7;
            const int b = j % NBUF;
            const uint32_t par = (uint32_t)((j / NBUF) & 1);
            int ok = 1;
            if (lane == 0) {
                const long long t0 = clock64();
                while (stamp[b] != j) {
                    if (*abort_flag || clock64() - t0 > max_wait) { ok = 0; break; }
                }
                if (ok) ok = mbar_wait_or_abort(&full[b], par, max_wait, abort_flag) ? 1 : 0;
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) { atomicOr(err_flag, 1); *abort_flag = 1; }
                break;
            }
            (void)mbar_try_wait(&full[b], par);
            const int tile = first + j * G;
            unsigned char *tp = reinterpret_cast<unsigned char *>(buf + (size_t)(2 * b) * (1 << LT));
            unsigned char *tl = tp + TMA_TILE_BYTES;
            const int wl = w ^ (lh & 7);
            const int base_t = (l0 | (wl << 1) | (lh << 4)) << 3;
            const int base_2 = (l0 | (wl << 1) | ((lh & 7) << 4) | (lh << 8)) << 3;
            u64 p[NR], l[NR];
            float &g0 = acc[0], &g1 = acc[1], &g0b = acc[2], &g1b = acc[3], &ga2 = acc[4], &gb2 = acc[5];
            // ---- L1 (stage A) from the tile layout: round 1 on local 8..11 ----
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                p[r] = *reinterpret_cast<const u64 *>(tp + base_t + (r << 11));
                l[r] = *reinterpret_cast<const u64 *>(tl + base_t + (r << 11));
            }
            adj_rotate_ts(p, l, P.rot[0], P.cls[0], s_tc[0][0], s_qi[0][0], s_corr[0][0], g0, g1);
            __syncwarp();
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int o = (base_t ^ ((r & 7) * 0x90)) + ((r >> 3) << 14) + ((r & 7) << 11);
                *reinterpret_cast<u64 *>(tp + o) = p[r];
                *reinterpret_cast<u64 *>(tl + o) = l[r];
            }
            __syncwarp();
            // ---- L2 (stage C): round 1 on local 4..7, the previous group's Z layer, round 2 ----
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int o = (base_2 ^ ((r & 7) * 0x90)) + ((r >> 3) << 10);
                p[r] = *reinterpret_cast<const u64 *>(tp + o);
                l[r] = *reinterpret_cast<const u64 *>(tl + o);
            }
            adj_rotate_ts(p, l, P.rot[2], P.cls[2], s_tc[0][2], s_qi[0][2], s_corr[0][2], g0, g1);
            {
                const uint2 e0 = ptab[tile & 255], e1 = ptab[256 + ((tile >> 8) & 255)],
                            e2 = ptab[512 + ((tile >> 16) & 255)];
                uint32_t pa = pa_lane ^ e0.x ^ e1.x ^ e2.x;
                uint32_t pb = pb_lane ^ e0.y ^ e1.y ^ e2.y;
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    if ((w >> q) & 1) { pa ^= P.pa_thr[1 + q]; pb ^= P.pb_thr[1 + q]; }
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
            adj_rotate_ts(p, l, P.rot[2], P.cls[2], s_tc[1][2], s_qi[1][2], s_corr[1][2], g0b, g1b);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int o = (base_2 ^ ((r & 7) * 0x90)) + ((r >> 3) << 10);
                *reinterpret_cast<u64 *>(tp + o) = p[r];
                *reinterpret_cast<u64 *>(tl + o) = l[r];
            }
            __syncwarp();
            // ---- L1 (stage A) from the exchange layout: round 2 on local 8..11; back to the tile ----
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int o = (base_t ^ ((r & 7) * 0x90)) + ((r >> 3) << 14) + ((r & 7) << 11);
                p[r] = *reinterpret_cast<const u64 *>(tp + o);
                l[r] = *reinterpret_cast<const u64 *>(tl + o);
            }
            adj_rotate_ts(p, l, P.rot[0], P.cls[0], s_tc[1][0], s_qi[1][0], s_corr[1][0], g0b, g1b);
            __syncwarp();
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                *reinterpret_cast<u64 *>(tp + base_t + (r << 11)) = p[r];
                *reinterpret_cast<u64 *>(tl + base_t + (r << 11)) = l[r];
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&done[b]);
            if (++since_flush == 8) { flush_terms(); since_flush = 0; }
        }
        if (since_flush) flush_terms();
    }
    __syncthreads();
    // the CTA's FP64 sums: values 0..3 (round 1; 2 and 3 stay zero, no Z layer of this
    // group in a shared pass) to partials, 4..7 to partials2
    if (t < 8) {
        double sum = 0.0;
        for (int w = 0; w < NC; ++w) sum += red[w][t];
        if (t < 4) partials[((long long)slot0 + blockIdx.x) * RED_NV + t] = sum;
        else partials2[((long long)slot0b + blockIdx.x) * RED_NV + (t - 4)] = sum;
    }
    (void)nblk;
}

}  // namespace qsim
