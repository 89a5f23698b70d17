// xpass_wl.cuh -- shared X pass with warp-local slices (complex64; sm_103a).
//
// Same operator as k_xpass_tma<.., MERGED = true, ..>.  Gauge-Higgs (tangent-form
// rotations): X of one factor group on the pass's new qubits, the whole diagonal Z
// layer, X of the next factor group on the same qubits (Eq. (8): all X-type factors
// commute).  Unitary gauge (HAD: unnormalised Walsh-Hadamard butterflies): H on the
// pass's qubits, a diagonal table (the Hadamard-basis X layer D_X, or the Z layer), H
// again, with the table's scale (2^-n after the two transforms of D_X).  It applies to
// passes whose
// rotated qubits all sit on local bits 4..11 of the 4096-amplitude tile (a pass fusing
// k <= 8 new qubits keeps a chunk of 12 - k >= 4 unrotated low bits).  Then local bits
// 1..3 never take part in a butterfly, and the tile splits into eight slices of 512
// amplitudes (local bits 1..3 fixed) that never exchange data:
//   * one slice is one warp's work item: 16 amplitudes per lane, two register layouts
//       L1: registers local {8..11}, lanes local {0, 4, 5, 6, 7}
//       L2: registers local {4..7},  lanes local {0, 8, 9, 10, 11}
//     and the passage between them goes through the slice's own shared-memory slots,
//     so a slice needs __syncwarp only and no CTA-wide barrier;
//   * the CTA's warps but the last take work items (tile, slice) in turn, item i ->
//     warp i mod (NW - 1); the last warp's lane 0 is the producer: it issues the TMA
//     load of each tile into one of NBUF buffers, waits (mbarrier, 8 arrivals) until
//     the eight slices of a tile are done, issues its bulk tensor store, and reloads
//     a buffer once its store has read it (with four or more buffers the buffer of the
//     tile before, whose store has had a tile's time to read it);
//   * before a consumer waits on a buffer's load barrier it waits for the buffer's
//     stamp (the tile the producer last issued into it) to name its tile, so the
//     barrier's phase parity it then tests is never one or two phases stale, whatever
//     the number of consumer warps.
// Default geometry: one CTA per SM, 24 warps, six buffers (a tile pool of 192 KB).
// Shared-memory slots (8-byte units) of amplitude l with the TMA 128-byte swizzle:
//   tile layout:     s = l ^ (((l >> 4) & 7) << 1)
//   exchange layout: the row R = (l >> 4) ^ ((l >> 8) & 7), s = l0 | ((w ^ (R & 7)) << 1) | (R << 4)
//     (w = local bits 1..3), a permutation of the same slice's slots in which both L1
//     and L2 accesses hit 16 distinct 8-byte bank pairs per half-warp, as L1 accesses
//     of the tile layout do.
#pragma once
#include "xpass_tma.cuh"

namespace qsim {

// Bounded mbarrier wait that also gives up when another warp has flagged an abort.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *bar, uint32_t parity, long long max_cycles,
                                                   volatile int *abort_flag) {
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > max_cycles) return false;
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// NBUF tile buffers, NW warps (NW - 1 consumers), MINB resident CTAs per SM; HAD:
// Walsh-Hadamard butterflies instead of tangent-form rotations.
template <int NBUF, int NW, int MINB, bool HAD>
__global__ void __launch_bounds__(32 * NW, MINB) k_xpass_wl(float2 *__restrict__ psi,
                                                                   const double *__restrict__ recs,
                                                                   const double *__restrict__ recs2,
                                                                   int rec_stride, int tiles_shift,
                                                                   int *__restrict__ err_flag,
                                                                   const __grid_constant__ CUtensorMap tmap,
                                                                   const __grid_constant__ TmaPass P) {
    (void)psi; (void)rec_stride;
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment for the 128-byte swizzle, as an offset from the shared array
    // (keeps the accesses below in the shared window, 32-bit addressed)
    unsigned char *base_ptr = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    float2 *buf = reinterpret_cast<float2 *>(base_ptr);                       // NBUF x 4096
    float2 *lut = buf + NBUF * (1 << LT);                                       // (nA+1)(nB+1)
    uint2 *ptab = reinterpret_cast<uint2 *>(lut + (P.nA + 1) * (P.nB + 1));     // 3 x 256
    constexpr int NTH = 32 * NW, NC = NW - 1;
    constexpr int DEFER = NBUF >= 4 ? 1 : 0;
    __shared__ uint64_t full[NBUF], done[NBUF];
    __shared__ int s_stamp[NBUF];       // tile (CTA-local index) last issued into each buffer
    __shared__ int s_abort;
    __shared__ u64 s_tc[2][3][RB][2];   // per round, stage (A: local 8..11, C: local 4..7), bit

    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    // tile indices fit 32 bits: one state of at most 2^34 amplitudes (host-checked)
    const int G = (int)gridDim.x;
    const int T = (int)P.total_tiles;
    const int first = (int)blockIdx.x;
    const long long max_wait = 2000000000ll;   // SM cycles (~1 s)
    volatile int *abort_flag = &s_abort;

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
    // the next pass may start its set-up; wait for the previous kernel's writes (state,
    // operator records) before the first read of global memory
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // operator records of the single batch element: tangent constants of both rounds,
    // phase table scaled by the cos factors of the X layer (Walsh-Hadamard passes: the
    // record's table as it is)
    if (!HAD && t < 2 * 3 * RB) {
        const int round = t / (3 * RB), st = (t / RB) % 3, k = t % RB;
        const double *rr = round ? recs2 : recs;
        const float tv = (float)rr[P.tan_off + ((P.cls[st] >> k) & 1)];
        s_tc[round][st][k][0] = pk(tv, tv);
        s_tc[round][st][k][1] = pk(-tv, -tv);
    }
    const int nB1 = P.nB + 1;
    const int nlut = (P.nA + 1) * nB1;
    const int loff = HAD ? P.lut_off : P.tan_off + 4;
    for (int i = t; i < nlut; i += NTH)
        lut[i] = make_float2((float)recs[loff + 2 * i], (float)recs[loff + 2 * i + 1]);
    __syncthreads();

    const int n_my = first < T ? (T - first + G - 1) / G : 0;   // tiles of this CTA
    const int mid_mask = (1 << P.mid_bits) - 1;
    volatile int *stamp = s_stamp;
    auto issue_load = [&](int j) {
        const int tile = first + j * G;
        const int b = j % NBUF;
        stamp[b] = j;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&full[b], TMA_TILE_BYTES);
        tma_load_5d(buf + (size_t)b * (1 << LT), &tmap, &full[b], 0, 0, tile & mid_mask, 0, tile >> P.mid_bits);
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
                tma_store_5d(&tmap, buf + (size_t)b * (1 << LT), 0, 0, tile & mid_mask, 0, tile >> P.mid_bits);
                bulk_commit();
                // reload the buffer of tile j - DEFER once its store has read it (every
                // bulk group but the DEFER newest is read).  With four or more buffers
                // the reload waits a tile (the store of tile j is not waited for); with
                // two or three it follows the tile's own store.
                if (j >= DEFER && j - DEFER + NBUF < n_my) {
                    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(DEFER) : "memory");
                    issue_load(j - DEFER + NBUF);
                    ++issued;
                }
            }
            // leave no copy in flight: loads that no slice consumed (abort), then stores
            for (int j = issued - NBUF < 0 ? 0 : issued - NBUF; j < issued; ++j)
                mbar_wait_bounded(&full[j % NBUF], (uint32_t)((j / NBUF) & 1), max_wait);
            bulk_wait_all();
        }
        __syncwarp();
    } else {
        // ---------------- consumers ----------------
        const int l0 = lane & 1, lh = lane >> 1;            // lane bits: l0, then four more
        (void)tiles_shift;   // one state: the tile index carries no batch bits
        // parity columns of the L2 lane bits (local 0 and 8..11)
        uint32_t pa_lane = 0, pb_lane = 0;
        if (l0) { pa_lane ^= P.pa_thr[0]; pb_lane ^= P.pb_thr[0]; }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if ((lh >> j) & 1) { pa_lane ^= P.pa_thr[4 + j]; pb_lane ^= P.pb_thr[4 + j]; }
        const int n_items = 8 * n_my;
        for (int item = warp; item < n_items; item += NC) {
            const int j = item >> 3, w = item & 7;
            const int b = j % NBUF;
            const uint32_t par = (uint32_t)((j / NBUF) & 1);
            // lane 0 waits for the buffer's stamp, then for the load; the other lanes then
            // observe the completed phase themselves
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
            unsigned char *tb = reinterpret_cast<unsigned char *>(buf + (size_t)b * (1 << LT));
            // byte offsets of the lane's slots (see the header)
            const int wl = w ^ (lh & 7);
            const int base_t = (l0 | (wl << 1) | (lh << 4)) << 3;                       // tile, L1
            const int base_2 = (l0 | (wl << 1) | ((lh & 7) << 4) | (lh << 8)) << 3;     // exchange, L2
            const int pc_tile = __popc(tile);
            u64 v[NR];
            // ---- L1 from the tile layout; round 1 on local 8..11 ----
#pragma unroll
            for (int r = 0; r < NR; ++r) v[r] = *reinterpret_cast<const u64 *>(tb + base_t + (r << 11));
            if (P.frame & 2) {
                const int k0 = __popc(lane) + __popc(w) + pc_tile;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const float2 x = mul_ipow(unpk(v[r]), k0 + __popc(r));
                    v[r] = pk(x.x, x.y);
                }
            }
            if (P.rot[2] == 0) {
                // every rotated qubit on tile bits 8..11: both rounds and the Z layer in
                // layout L1, each lane writing back the slots it read (no exchange)
                if (HAD) hadamard_w(v, P.rot[0]); else rotate_ts(v, P.rot[0], s_tc[0][0]);
                const uint2 e0 = ptab[tile & 255], e1 = ptab[256 + ((tile >> 8) & 255)],
                            e2 = ptab[512 + ((tile >> 16) & 255)];
                uint32_t pa = e0.x ^ e1.x ^ e2.x, pb = e0.y ^ e1.y ^ e2.y;
                if (l0) { pa ^= P.paA_thr[0]; pb ^= P.pbA_thr[0]; }
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    if ((w >> q) & 1) { pa ^= P.paA_thr[1 + q]; pb ^= P.pbA_thr[1 + q]; }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if ((lh >> q) & 1) { pa ^= P.paA_thr[4 + q]; pb ^= P.pbA_thr[4 + q]; }
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const float2 x = cphase(unpk(v[r]), lut[__popc(pa ^ P.paA_reg[r]) * nB1 + __popc(pb ^ P.pbA_reg[r])]);
                    v[r] = pk(x.x, x.y);
                }
                if (P.scale != 1.0f) {
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        float2 x = unpk(v[r]);
                        x.x *= P.scale; x.y *= P.scale;
                        v[r] = pk(x.x, x.y);
                    }
                }
                if (HAD) hadamard_w(v, P.rot[0]); else rotate_ts(v, P.rot[0], s_tc[1][0]);
                if (P.frame & 4) {
                    const int k0 = -(__popc(lane) + __popc(w) + pc_tile);
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const float2 x = mul_ipow(unpk(v[r]), (k0 - __popc(r)) & 3);
                        v[r] = pk(x.x, x.y);
                    }
                }
#pragma unroll
                for (int r = 0; r < NR; ++r) *reinterpret_cast<u64 *>(tb + base_t + (r << 11)) = v[r];
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&done[b]);
                continue;
            }
            if (HAD) hadamard_w(v, P.rot[0]); else rotate_ts(v, P.rot[0], s_tc[0][0]);
            __syncwarp();
#pragma unroll
            for (int r = 0; r < NR; ++r)
                *reinterpret_cast<u64 *>(tb + ((base_t ^ ((r & 7) * 0x90)) + ((r >> 3) << 14) + ((r & 7) << 11))) = v[r];
            __syncwarp();
            // ---- L2 from the exchange layout; round 1 on local 4..7, Z layer, round 2 ----
#pragma unroll
            for (int r = 0; r < NR; ++r) v[r] = *reinterpret_cast<const u64 *>(tb + ((base_2 ^ ((r & 7) * 0x90)) + ((r >> 3) << 10)));
            if (HAD) hadamard_w(v, P.rot[2]); else rotate_ts(v, P.rot[2], s_tc[0][2]);
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
                    const float2 x = cphase(unpk(v[r]), lut[__popc(pa ^ P.pa_reg[r]) * nB1 + __popc(pb ^ P.pb_reg[r])]);
                    v[r] = pk(x.x, x.y);
                }
                if (P.scale != 1.0f) {
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        float2 x = unpk(v[r]);
                        x.x *= P.scale; x.y *= P.scale;
                        v[r] = pk(x.x, x.y);
                    }
                }
            }
            if (HAD) hadamard_w(v, P.rot[2]); else rotate_ts(v, P.rot[2], s_tc[1][2]);
#pragma unroll
            for (int r = 0; r < NR; ++r)
                *reinterpret_cast<u64 *>(tb + ((base_2 ^ ((r & 7) * 0x90)) + ((r >> 3) << 10))) = v[r];
            __syncwarp();
            // ---- L1 from the exchange layout; round 2 on local 8..11; back to the tile ----
#pragma unroll
            for (int r = 0; r < NR; ++r)
                v[r] = *reinterpret_cast<const u64 *>(tb + ((base_t ^ ((r & 7) * 0x90)) + ((r >> 3) << 14) + ((r & 7) << 11)));
            if (HAD) hadamard_w(v, P.rot[0]); else rotate_ts(v, P.rot[0], s_tc[1][0]);
            if (P.frame & 4) {
                const int k0 = -(__popc(lane) + __popc(w) + pc_tile);
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const float2 x = mul_ipow(unpk(v[r]), (k0 - __popc(r)) & 3);
                    v[r] = pk(x.x, x.y);
                }
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < NR; ++r) *reinterpret_cast<u64 *>(tb + base_t + (r << 11)) = v[r];
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&done[b]);
        }
    }
    __syncthreads();
}

}  // namespace qsim
