// xpass_tma.cuh -- persistent, TMA-fed X pass for complex64 states (sm_103a).
//
// Same operator as k_xpass (exp(i theta_q X_q) on the 12 local qubits of a
// 4096-amplitude tile, optionally followed by the whole diagonal Z layer), but:
//   * tiles arrive by cp.async.bulk.tensor (TMA) into shared memory, described by a
//     5-D tensor map whose box is the tile (16 contiguous amplitudes x the chunk and
//     new-qubit dimensions), with the 128-byte swizzle;
//   * the grid is persistent: each CTA walks tiles blockIdx.x, +gridDim.x, ... with
//     NBUF shared-memory buffers, so the TMA load of the next tiles overlaps the
//     butterflies of the current one (mbarrier-tracked, bounded waits);
//   * every per-pass constant (offsets, parity columns, rotation masks) is a
//     __grid_constant__ kernel parameter, read from the constant bank.
// Stage layouts (local bit -> register / thread), as in k_xpass:
//   A: registers local {8..11}, threads local {0..7}           (8-byte smem access)
//   B: registers local {0..3},  threads local {4..11}          (16-byte smem access)
//   C: registers local {4..7},  threads local {0..3, 8..11}    (global store)
// With the 128-byte swizzle, amplitude l sits at l ^ (((l >> 4) & 7) << 1): every
// stage then hits 16 distinct banks per half-warp (8-byte) or 8 distinct 16-byte
// units per quarter-warp (16-byte).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

#include "kernels.cuh"

namespace qsim {

struct TmaPass {
    int c;                      // chunk bits (global bits 0..c-1 stay local bits 0..c-1)
    int next;                   // first new global bit (local bit c)
    int k;                      // new bits in this pass
    int mid_bits;               // next - c: tile-index bits that land on global bits c..next-1
    long long total_tiles;      // batch * 2^(n - 12)
    long long toff_c[8];        // stage C: global offset of thread bit j (local 0,1,2,3,8,9,10,11)
    long long roff_c[NR];       // stage C: global offset of register r (local bits 4..7)
    unsigned rot[3];            // register bits to rotate in stages A, B, C
    unsigned cls[3];            // register bit k of stage s uses class (cls[s] >> k) & 1
    int stage_b;                // run stage B
    int apply_z, nA, nB;
    uint32_t pa_thr[8], pb_thr[8];    // parity columns of the stage-C thread bits
    uint32_t pa_reg[NR], pb_reg[NR];  // parity of stage-C register r
    uint32_t pa_tile[32], pb_tile[32];// parity columns of tile-index bits (bit order of tau)
    int tile_bits;              // tile-index bits that carry parity (not batch)
    int hadamard;               // butterflies (a + b, a - b) instead of rotations
    int lut_off;                // offset (doubles) of the phase table in the operator record
    float scale;                // factor applied with the phase (a power of two)
    int frame;                  // bit 0: rotations in the frame phi_i = i^popc(i) psi_i;
                                // bit 1: convert psi -> phi at stage A; bit 2: phi -> psi at stage C
    uint32_t paA_thr[8], pbA_thr[8];  // parity columns of the stage-A thread bits (local 0..7)
    uint32_t paA_reg[NR], pbA_reg[NR];// parity of stage-A register r (local bits 8..11)
    long long toff_a[8];        // stage A: global offset of thread bit j (local 0..7)
    long long roff_a[NR];       // stage A: global offset of register r (local bits 8..11)
    int tan_off;                // offset (doubles) of the tangent triple in the record
    int xscale;                 // tangent form: multiply by the record's C before the
                                // store (set on the last pass of a group without Z;
                                // with a Z layer C is in the scaled table)
    int adj_u[3][2];            // adjoint, tangent form: X qubits of the factor group per
                                // class not yet un-rotated when stage s reads its terms
    int adj_u2[3][2];           // the same for the second round of a shared reverse pass
                                // (the previous factor group; stages run C, B, A)
};

constexpr int TMA_TILE_BYTES = (1 << LT) * 8;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after ~max_cycles SM clocks (about a second) and reports it.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long max_cycles) {
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > max_cycles) return false;
    return true;
}

__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ int swz128(int l) { return l ^ (((l >> 4) & 7) << 1); }

// TMA bulk tensor store of a shared-memory tile (same map and box as the load)
__device__ __forceinline__ void tma_store_5d(const CUtensorMap *map, const void *src, int c0, int c1, int c2,
                                             int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5, %6}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(smem_addr(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// packed FP32x2 fused multiply-add: (a.x * b.x + c.x, a.y * b.y + c.y)
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

typedef unsigned long long u64;

__device__ __forceinline__ u64 pk(float x, float y) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}

// packed FP32x2 FMA on register pairs
__device__ __forceinline__ u64 fma2p(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ void rrotp(u64 &a, u64 &b, u64 nu, u64 ps, u64 ns) {
    const u64 ta = fma2p(nu, a, a);
    const u64 tb = fma2p(nu, b, b);
    const u64 na = fma2p(ps, b, ta);
    const u64 nb = fma2p(ns, a, tb);
    a = na;
    b = nb;
}

// In the frame phi_i = i^{popcount(i)} psi_i, exp(i theta X_q) becomes the real rotation
// [[cos, sin], [-sin, cos]] (S X S^dagger = Y with S = diag(1, i)), which treats the real
// and imaginary parts alike:  a' = a - u a + s b,  b' = b - u b - s a  (cos = 1 - u).
__device__ __forceinline__ void rrot(float2 &a, float2 &b, float2 nu, float2 ps, float2 ns) {
    const float2 ta = fma2(nu, a, a);
    const float2 tb = fma2(nu, b, b);
    const float2 na = fma2(ps, b, ta);
    const float2 nb = fma2(ns, a, tb);
    a = na;
    b = nb;
}

__device__ __forceinline__ void rotate_regs_phi(float2 (&v)[NR], unsigned mask, const int (&cls)[RB], float u0,
                                                float s0, float u1, float s1) {
    u64 w[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) w[r] = pk(v[r].x, v[r].y);
    const u64 nu0 = pk(-u0, -u0), ps0 = pk(s0, s0), ns0 = pk(-s0, -s0);
    const u64 nu1 = pk(-u1, -u1), ps1 = pk(s1, s1), ns1 = pk(-s1, -s1);
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        if (!((mask >> k) & 1u)) continue;
        const bool c = cls[k] != 0;
        const u64 nu = c ? nu1 : nu0, ps = c ? ps1 : ps0, ns = c ? ns1 : ns0;
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (!((r >> k) & 1)) rrotp(w[r], w[r | (1 << k)], nu, ps, ns);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) asm("mov.b64 {%0, %1}, %2;" : "=f"(v[r].x), "=f"(v[r].y) : "l"(w[r]));
}

// unnormalised Hadamard butterflies with packed FP32x2: (a, b) <- (a + b, a - b)
__device__ __forceinline__ void hadamard_regs2(float2 (&v)[NR], unsigned mask) {
    const float2 one = make_float2(1.f, 1.f), mone = make_float2(-1.f, -1.f);
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        if (!((mask >> k) & 1u)) continue;
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (!((r >> k) & 1)) {
                const int q = r | (1 << k);
                const float2 a = v[r], b = v[q];
                v[r] = fma2(one, a, b);
                v[q] = fma2(mone, b, a);
            }
    }
}

__device__ __forceinline__ float2 unpk(u64 w) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(w));
    return v;
}

// Real-frame rotations on packed register pairs; per class the constants
// (-u, -u), (s, s), (-s, -s) are prepared once per operator record.
struct RotConst { u64 nu[2], ps[2], ns[2]; };

__device__ __forceinline__ void rotate_w(u64 (&w)[NR], unsigned mask, const int (&cls)[RB], const RotConst &C) {
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        if (!((mask >> k) & 1u)) continue;
        const bool c = cls[k] != 0;
        const u64 nu = c ? C.nu[1] : C.nu[0], ps = c ? C.ps[1] : C.ps[0], ns = c ? C.ns[1] : C.ns[0];
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (!((r >> k) & 1)) rrotp(w[r], w[r | (1 << k)], nu, ps, ns);
    }
}

// Tangent form (dev_tan_triple): butterflies a' = a + t b, b' = b - t a on packed
// register pairs, constants (t, t) and (-t, -t) per class; the cos factors of the whole
// X layer are applied once, as the record's scalar C.
struct TanConst { u64 pt[2], nt[2]; };

__device__ __forceinline__ void rotate_t(u64 (&w)[NR], unsigned mask, const int (&cls)[RB], const TanConst &C) {
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        if (!((mask >> k) & 1u)) continue;
        const bool c = cls[k] != 0;
        const u64 pt = c ? C.pt[1] : C.pt[0], nt = c ? C.nt[1] : C.nt[0];
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (!((r >> k) & 1)) {
                const int q = r | (1 << k);
                const u64 a = w[r], b = w[q];
                w[r] = fma2p(pt, b, a);
                w[q] = fma2p(nt, a, b);
            }
    }
}

// Tangent form with the constants of each register bit read from shared memory
// (tc[k] = {(t, t), (-t, -t)} for the class of that bit), so no registers hold them
// between stages and no selects pick them.
__device__ __forceinline__ void rotate_ts(u64 (&w)[NR], unsigned mask, const u64 (*tc)[2]) {
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        if (!((mask >> k) & 1u)) continue;
        const u64 pt = tc[k][0], nt = tc[k][1];
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (!((r >> k) & 1)) {
                const int q = r | (1 << k);
                const u64 a = w[r], b = w[q];
                w[r] = fma2p(pt, b, a);
                w[q] = fma2p(nt, a, b);
            }
    }
}

__device__ __forceinline__ void rot_apply(u64 (&w)[NR], unsigned mask, const int (&cls)[RB], const RotConst &C) {
    rotate_w(w, mask, cls, C);
}
__device__ __forceinline__ void rot_apply(u64 (&w)[NR], unsigned mask, const int (&cls)[RB], const TanConst &C) {
    rotate_t(w, mask, cls, C);
}

// rotation constants of one operator record, (u, s) or tangent form
__device__ __forceinline__ void load_xconst(RotConst &C, const double *rec, int) {
    const float u0 = (float)rec[0], s0 = (float)rec[1], u1 = (float)rec[2], s1 = (float)rec[3];
    C.nu[0] = pk(-u0, -u0); C.ps[0] = pk(s0, s0); C.ns[0] = pk(-s0, -s0);
    C.nu[1] = pk(-u1, -u1); C.ps[1] = pk(s1, s1); C.ns[1] = pk(-s1, -s1);
}
__device__ __forceinline__ void load_xconst(TanConst &C, const double *rec, int tan_off) {
    const float t0 = (float)rec[tan_off], t1 = (float)rec[tan_off + 1];
    C.pt[0] = pk(t0, t0); C.nt[0] = pk(-t0, -t0);
    C.pt[1] = pk(t1, t1); C.nt[1] = pk(-t1, -t1);
}

__device__ __forceinline__ void hadamard_w(u64 (&w)[NR], unsigned mask) {
    const u64 one = pk(1.f, 1.f), mone = pk(-1.f, -1.f);
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        if (!((mask >> k) & 1u)) continue;
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (!((r >> k) & 1)) {
                const int q = r | (1 << k);
                const u64 a = w[r], b = w[q];
                w[r] = fma2p(one, a, b);
                w[q] = fma2p(mone, b, a);
            }
    }
}

// v * i^k
__device__ __forceinline__ float2 mul_ipow(float2 v, int k) {
    float2 r = (k & 1) ? make_float2(-v.y, v.x) : v;
    if (k & 2) { r.x = -r.x; r.y = -r.y; }
    return r;
}

// MERGED: the pass applies X(G) of one factor group, the Z layer, then X(G) of the
// next factor group (recs2), for the same tile qubits G.  All X-type factors commute,
// so consecutive factor groups that take their qubit groups in opposite orders share
// the pass that holds G (one HBM round trip fewer per Trotter step).  With Hadamard
// butterflies (unitary gauge) both rounds are Walsh-Hadamard butterflies on G around
// the diagonal table (the Hadamard-basis X layer or the Z layer).  The second round
// runs stages C, B, A and stores from the stage-A layout.
// TAN: rotations in the tangent form (records carry the triple at P.tan_off).
template <int NBUF, bool STORE_TMA, bool MERGED, bool TAN>
__global__ void __launch_bounds__(NT, NBUF == 2 ? 3 : 2) k_xpass_tma(float2 *__restrict__ psi, const double *__restrict__ recs,
                                                  const double *__restrict__ recs2,
                                                  int rec_stride, int tiles_shift,
                                                  int *__restrict__ err_flag,
                                                  const __grid_constant__ CUtensorMap tmap,
                                                  const __grid_constant__ TmaPass P) {
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment for the 128-byte swizzle pattern
    unsigned char *base_ptr = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float2 *buf = reinterpret_cast<float2 *>(base_ptr);                       // NBUF x 4096
    float2 *lut = buf + NBUF * (1 << LT);                                       // (nA+1)(nB+1)
    uint2 *ptab = reinterpret_cast<uint2 *>(lut + (P.apply_z ? (P.nA + 1) * (P.nB + 1) : 0));  // 3 x 256
    __shared__ uint64_t bars[NBUF];
    __shared__ int s_ok;
    typedef typename std::conditional<TAN, TanConst, RotConst>::type XC;
    __shared__ XC s_rc2;           // MERGED: rotation constants of the second round
    __shared__ u64 s_tc[2][3][RB][2];   // TAN and MERGED: per round, stage and register bit:
                                        // (t,t), (-t,-t); plain passes keep them in registers

    const int t = threadIdx.x;
    const long long G = gridDim.x;
    const long long T = P.total_tiles;
    const long long first = blockIdx.x;
    const long long max_wait = 2000000000ll;   // SM cycles (~1 s)

    if (t == 0) {
        for (int b = 0; b < NBUF; ++b) mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
    // per-CTA tables: parity of tile-index bytes, Z phase table (batch 0 record; the
    // record of other batch elements is loaded when the batch index changes)
    if (P.apply_z) {
        for (int e = t; e < 3 * 256; e += NT) {
            int byte = e >> 8, val = e & 255;
            uint32_t a = 0, b = 0;
            for (int j = 0; j < 8; ++j) {
                int bit = 8 * byte + j;
                if (bit < P.tile_bits && ((val >> j) & 1)) { a ^= P.pa_tile[bit]; b ^= P.pb_tile[bit]; }
            }
            ptab[e] = make_uint2(a, b);
        }
    }
    __syncthreads();
    // Programmatic dependent launch: the next pass may start its set-up (everything above
    // reads only kernel parameters), and this one waits for the previous kernel's writes
    // (the state, the operator records) before its first read of global memory.  Both
    // instructions do nothing when the launch carries no programmatic dependency.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    auto coords_of = [&](long long tile, int &x1, int &x2, int &x4) {
        x1 = 0;
        x2 = (int)(tile & ((1ll << P.mid_bits) - 1));
        x4 = (int)(tile >> P.mid_bits);
    };
    auto issue = [&](long long it) {
        long long tile = first + it * G;
        int b = (int)(it % NBUF);
        int x1, x2, x4;
        coords_of(tile, x1, x2, x4);
        if (STORE_TMA) bulk_wait_read_all();   // a store may still be reading this buffer
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&bars[b], TMA_TILE_BYTES);
        tma_load_5d(buf + (size_t)b * (1 << LT), &tmap, &bars[b], 0, x1, x2, 0, x4);
    };

    const int n_my = first < T ? (int)((T - first + G - 1) / G) : 0;   // tiles this CTA processes
    if (t == 0)
        for (int it = 0; it < NBUF - 1 && it < n_my; ++it) issue(it);

    // per-thread constants: shared-memory bases of the three stages (the 128-byte
    // swizzle touches amplitude bits 1..3 only, from bits 4..6), stage-C offsets
    const int tlo = t & 15, thi = t >> 4;
    const int a_base = swz128(t);                     // stage A: + (r << 8)
    int c_base[8];                                    // stage C: c_base[r & 7] + (r << 4)
#pragma unroll
    for (int j = 0; j < 8; ++j) c_base[j] = (tlo ^ (j << 1)) | (thi << 8);
    const int b_base = t << 3;                        // stage B, float4 index
    const int b_x = t & 7;                            // stage B swizzle of the float4 slot
    long long toff = 0;
    uint32_t pa_t = 0, pb_t = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if ((tlo >> j) & 1) { toff += P.toff_c[j]; pa_t ^= P.pa_thr[j]; pb_t ^= P.pb_thr[j]; }
        if ((thi >> j) & 1) { toff += P.toff_c[4 + j]; pa_t ^= P.pa_thr[4 + j]; pb_t ^= P.pb_thr[4 + j]; }
    }
    long long toff_a = 0;                             // MERGED: stage-A store offset
    if (MERGED) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if ((t >> j) & 1) toff_a += P.toff_a[j];
    }
    const int nB1 = P.nB + 1;
    const int nlut = (P.nA + 1) * nB1;
    long long cur_batch = -1;
    XC RC;
    float xs = 1.f;                                   // tangent form: scalar C of the record
    int cls0[RB], cls1[RB], cls2[RB];
#pragma unroll
    for (int kk = 0; kk < RB; ++kk) {
        cls0[kk] = (P.cls[0] >> kk) & 1; cls1[kk] = (P.cls[1] >> kk) & 1; cls2[kk] = (P.cls[2] >> kk) & 1;
    }
    const long long tmask = (1ll << tiles_shift) - 1;

    long long tile = first;
    for (int it = 0; it < n_my; ++it, tile += G) {
        const int b = it % NBUF;
        const uint32_t parity = (uint32_t)((it / NBUF) & 1);
        const long long batch = tile >> tiles_shift;
        if (batch != cur_batch) {
            // operator record of this batch element (angles, phase table)
            __syncthreads();
            const double *rec = recs + batch * rec_stride;
            if (TAN && !MERGED) load_xconst(RC, rec, P.tan_off);
            if (TAN) {
                xs = (float)rec[P.tan_off + 2];
                if (MERGED && t < 2 * 3 * RB) {
                    const int round = t / (3 * RB), st = (t / RB) % 3, k = t % RB;
                    const double *rr = round ? recs2 + batch * rec_stride : rec;
                    const float tv = (float)rr[P.tan_off + ((P.cls[st] >> k) & 1)];
                    s_tc[round][st][k][0] = pk(tv, tv);
                    s_tc[round][st][k][1] = pk(-tv, -tv);
                }
            } else {
                load_xconst(RC, rec, P.tan_off);
            }
            if (P.apply_z) {
                const int loff = TAN ? P.tan_off + 4 : P.lut_off;   // tangent form: table scaled by C
                for (int i = t; i < nlut; i += NT)
                    lut[i] = make_float2((float)rec[loff + 2 * i], (float)rec[loff + 2 * i + 1]);
            }
            if (!TAN && MERGED && t == 0) load_xconst(s_rc2, recs2 + batch * rec_stride, P.tan_off);
            cur_batch = batch;
        }
        if (t == 0) {
            if (!mbar_wait_bounded(&bars[b], parity, max_wait)) {
                atomicOr(err_flag, 1);
                s_ok = 0;
                // wait (bounded) for every load this CTA still has in flight before leaving
                for (int j = it; j < it + NBUF - 1 && j < n_my; ++j)
                    mbar_wait_bounded(&bars[j % NBUF], (uint32_t)((j / NBUF) & 1), max_wait);
                if (STORE_TMA) bulk_wait_all();
            }
        }
        __syncthreads();
        if (!s_ok) return;
        if (t == 0 && it + NBUF - 1 < n_my) issue(it + NBUF - 1);

        u64 *tb = reinterpret_cast<u64 *>(buf + (size_t)b * (1 << LT));
        u64 w[NR];
        // ---- stage A: registers = local 8..11 ----
#pragma unroll
        for (int r = 0; r < NR; ++r) w[r] = tb[a_base + (r << TB)];
        const int pc_tile = __popcll(tile & tmask);
        if (P.frame & 2) {
            const int k0 = __popc(t) + pc_tile;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float2 v = mul_ipow(unpk(w[r]), k0 + __popc(r));
                w[r] = pk(v.x, v.y);
            }
        }
        if (P.frame & 1) { if (TAN && MERGED) rotate_ts(w, P.rot[0], s_tc[0][0]); else rot_apply(w, P.rot[0], cls0, RC); }
        else hadamard_w(w, P.rot[0]);
#pragma unroll
        for (int r = 0; r < NR; ++r) tb[a_base + (r << TB)] = w[r];
        __syncthreads();
        // ---- stage B: registers = local 0..3 (16-byte accesses) ----
        if (P.stage_b) {
            ulonglong2 *tb2 = reinterpret_cast<ulonglong2 *>(tb);
#pragma unroll
            for (int m = 0; m < NR / 2; ++m) {
                const ulonglong2 q = tb2[b_base + (m ^ b_x)];
                w[2 * m] = q.x;
                w[2 * m + 1] = q.y;
            }
            if (P.frame & 1) { if (TAN && MERGED) rotate_ts(w, P.rot[1], s_tc[0][1]); else rot_apply(w, P.rot[1], cls1, RC); }
            else hadamard_w(w, P.rot[1]);
#pragma unroll
            for (int m = 0; m < NR / 2; ++m) tb2[b_base + (m ^ b_x)] = make_ulonglong2(w[2 * m], w[2 * m + 1]);
            __syncthreads();
        }
        // ---- stage C: registers = local 4..7; diagonal phase; store ----
#pragma unroll
        for (int r = 0; r < NR; ++r) w[r] = tb[c_base[r & 7] + (r << 4)];
        if (P.frame & 1) { if (TAN && MERGED) rotate_ts(w, P.rot[2], s_tc[0][2]); else rot_apply(w, P.rot[2], cls2, RC); }
        else hadamard_w(w, P.rot[2]);
        // global base of the tile: mid bits -> global c.., upper bits (and batch) -> next+k..
        const long long mid = tile & ((1ll << P.mid_bits) - 1);
        const long long up = tile >> P.mid_bits;
        const long long gbase = (mid << P.c) + (up << (P.next + P.k));
        if (P.apply_z || (P.frame & 4) || (TAN && P.xscale)) {
            float2 v[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) v[r] = unpk(w[r]);
            if (P.apply_z) {
                const long long tin = tile & tmask;                       // parity ignores batch
                uint2 e0 = ptab[tin & 255], e1 = ptab[256 + ((tin >> 8) & 255)], e2 = ptab[512 + ((tin >> 16) & 255)];
                const uint32_t pa = pa_t ^ e0.x ^ e1.x ^ e2.x;
                const uint32_t pb = pb_t ^ e0.y ^ e1.y ^ e2.y;
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    v[r] = cphase(v[r], lut[__popc(pa ^ P.pa_reg[r]) * nB1 + __popc(pb ^ P.pb_reg[r])]);
                if (P.scale != 1.0f) {
#pragma unroll
                    for (int r = 0; r < NR; ++r) { v[r].x *= P.scale; v[r].y *= P.scale; }
                }
            }
            if (TAN && !P.apply_z && P.xscale) {
                // the cos factors of a factor group without Z layer (with a Z layer they
                // are in its table)
#pragma unroll
                for (int r = 0; r < NR; ++r) { v[r].x *= xs; v[r].y *= xs; }
            }
            if (!MERGED && (P.frame & 4)) {
                const int k0 = -(__popc(tlo) + __popc(thi) + pc_tile);
#pragma unroll
                for (int r = 0; r < NR; ++r) v[r] = mul_ipow(v[r], (k0 - __popc(r)) & 3);
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) w[r] = pk(v[r].x, v[r].y);
        }
        if (MERGED) {
            // ---- second round: stage C (still in registers), B, A; store from A ----
            if (P.frame & 1) {
                if (TAN) {
                    rotate_ts(w, P.rot[2], s_tc[1][2]);
                } else {
                    const XC R2 = s_rc2;
                    rot_apply(w, P.rot[2], cls2, R2);
                }
            } else {
                hadamard_w(w, P.rot[2]);
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) tb[c_base[r & 7] + (r << 4)] = w[r];
            __syncthreads();
            if (P.stage_b) {
                ulonglong2 *tb2 = reinterpret_cast<ulonglong2 *>(tb);
#pragma unroll
                for (int m = 0; m < NR / 2; ++m) {
                    const ulonglong2 q = tb2[b_base + (m ^ b_x)];
                    w[2 * m] = q.x;
                    w[2 * m + 1] = q.y;
                }
                if (P.frame & 1) {
                    if (TAN) {
                        rotate_ts(w, P.rot[1], s_tc[1][1]);
                    } else {
                        const XC R2 = s_rc2;
                        rot_apply(w, P.rot[1], cls1, R2);
                    }
                } else {
                    hadamard_w(w, P.rot[1]);
                }
#pragma unroll
                for (int m = 0; m < NR / 2; ++m) tb2[b_base + (m ^ b_x)] = make_ulonglong2(w[2 * m], w[2 * m + 1]);
                __syncthreads();
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) w[r] = tb[a_base + (r << TB)];
            if (P.frame & 1) {
                if (TAN) {
                    rotate_ts(w, P.rot[0], s_tc[1][0]);
                } else {
                    const XC R2 = s_rc2;
                    rot_apply(w, P.rot[0], cls0, R2);
                }
            } else {
                hadamard_w(w, P.rot[0]);
            }
            if (P.frame & 4) {
                const int k0 = -(__popc(t) + pc_tile);
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const float2 v = mul_ipow(unpk(w[r]), (k0 - __popc(r)) & 3);
                    w[r] = pk(v.x, v.y);
                }
            }
            if (STORE_TMA) {
#pragma unroll
                for (int r = 0; r < NR; ++r) tb[a_base + (r << TB)] = w[r];
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
                if (t == 0) {
                    const int x2 = (int)(tile & ((1ll << P.mid_bits) - 1));
                    const int x4 = (int)(tile >> P.mid_bits);
                    tma_store_5d(&tmap, tb, 0, 0, x2, 0, x4);
                    bulk_commit();
                }
            } else {
                u64 *dst = reinterpret_cast<u64 *>(psi + gbase + toff_a);
#pragma unroll
                for (int r = 0; r < NR; ++r) dst[P.roff_a[r]] = w[r];
            }
        } else if (STORE_TMA) {
            // back into the swizzled tile, then one bulk tensor store of the whole tile
#pragma unroll
            for (int r = 0; r < NR; ++r) tb[c_base[r & 7] + (r << 4)] = w[r];
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (t == 0) {
                const int x2 = (int)(tile & ((1ll << P.mid_bits) - 1));
                const int x4 = (int)(tile >> P.mid_bits);
                tma_store_5d(&tmap, tb, 0, 0, x2, 0, x4);
                bulk_commit();
            }
        } else {
            u64 *dst = reinterpret_cast<u64 *>(psi + gbase + toff);
#pragma unroll
            for (int r = 0; r < NR; ++r) dst[P.roff_c[r]] = w[r];
        }
    }
    if (STORE_TMA && t == 0) bulk_wait_all();   // the CTA's shared memory must outlive its stores
}

}  // namespace qsim

namespace qsim {

// Self-test of the bounded wait: an mbarrier that expects one arrival which never
// comes.  mbar_wait_bounded gives up after max_cycles, the kernel records the
// timeout in err_flag (bit 1) and returns; nothing faults and the context stays usable.
__global__ void k_wait_probe(int *__restrict__ err_flag, long long max_cycles) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!mbar_wait_bounded(&bar, 0, max_cycles)) atomicOr(err_flag, 2);
    }
}

}  // namespace qsim
