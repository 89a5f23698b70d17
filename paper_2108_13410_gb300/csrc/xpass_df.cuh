// xpass_df.cuh -- complex128 Walsh-Hadamard passes in double-float arithmetic (sm_103a).
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so a complex128 pass written with
// FP64 butterflies is bound by the FP64 pipe far below the HBM roofline.  Here each real
// number of the state is carried as an unevaluated sum hi + lo of two floats (|lo| <=
// ulp(hi) / 2, 48 significand bits), and the passes run on the FP32 pipes with packed
// f32x2 instructions, (re, im) in one 64-bit register:
//   * sum and difference: Knuth's two-sum (two-diff) of the high parts (exact), the
//     error and the low parts summed into the low part (8 packed operations per output).
//     Within a pass the pairs are not renormalised after every butterfly (the low part
//     grows by at most the pass's number of stages times an ulp of the high part, about
//     2^-43 relative); one fast renormalisation runs before the table product and before
//     the store;
//   * product with a table entry (cos phi, sin phi) held in double-float: the rounding
//     error of the high product recovered exactly by scalar FMA (fmaf, one rounding),
//     the cross terms by packed FMA, renormalisation.  (A packed f32x2 FMA in that role
//     left the products at float precision, ~5e-8 per phase, so the exact term is not
//     taken from it.)
// Layout in HBM while a call runs ("blocked double-float"): every block of 16 amplitudes
// (256 bytes of complex128) holds the 16 high (re, im) float pairs, then the 16 low pairs.
// A block converts in place, and the high (low) halves of a tile form an ordinary
// complex64-like tile under a tensor map with doubled strides (base, base + 128 bytes), so
// the pass loads a tile pair by two TMA copies and reuses the stage layouts of the
// complex64 kernel (xpass_tma.cuh).  The pass applies unnormalised Walsh-Hadamard
// butterflies on the pass's qubits (the unitary-gauge X layer H^n D_X H^n and the Z layer
// between transforms, Sec. II), optionally the diagonal table with its scale, and (MERGED)
// a second round of butterflies on the same qubits.  ROT: the gauge-Higgs form instead:
// tangent-form rotations in the real frame phi = i^popc psi (a' = a + t b, b' = b - t a,
// t = tan theta of the qubit's class in double-float, Eq. (8)), the Z layer from the
// table scaled by the group's cos factors C, C alone for a group without Z layer, the
// frame conversions on the first and last pass of a call, and (MERGED) the next factor
// group's rotations on the same qubits.
#pragma once
#include "xpass_tma.cuh"

namespace qsim {

__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 swap2(u64 a) {   // (x, y) -> (y, x)
    u64 d;
    asm("{\n\t.reg .b32 x, y;\n\tmov.b64 {x, y}, %1;\n\tmov.b64 %0, {y, x};\n\t}" : "=l"(d) : "l"(a));
    return d;
}

// a * b - p per lane for p = RN(a * b): exact, by scalar FMA
__device__ __forceinline__ u64 prod_err(u64 a, u64 b, u64 p) {
    const float2 x = unpk(a), y = unpk(b), q = unpk(p);
    return pk(fmaf(x.x, y.x, -q.x), fmaf(x.y, y.y, -q.y));
}

// (vh, vl) * (ch, cl), both lanes: exact high product, cross terms, renormalisation.
__device__ __forceinline__ void df_mul(u64 vh, u64 vl, u64 ch, u64 cl, u64 &rh, u64 &rl) {
    const u64 p = mul2(vh, ch);
    u64 e = prod_err(vh, ch, p);
    e = fma2p(vh, cl, e);
    e = fma2p(vl, ch, e);
    rh = add2(p, e);
    rl = sub2(e, sub2(rh, p));
}

__device__ __forceinline__ void df_add(u64 ah, u64 al, u64 bh, u64 bl, u64 &rh, u64 &rl) {
    const u64 s = add2(ah, bh);
    const u64 sv = sub2(s, ah);
    u64 e = add2(sub2(ah, sub2(s, sv)), sub2(bh, sv));
    e = add2(e, add2(al, bl));
    rh = add2(s, e);
    rl = sub2(e, sub2(rh, s));
}

// sum and difference without renormalisation (see the header)
__device__ __forceinline__ void df_butterfly_lazy(u64 &ah, u64 &al, u64 &bh, u64 &bl) {
    const u64 s = add2(ah, bh);
    const u64 sv = sub2(s, ah);
    const u64 es = add2(sub2(ah, sub2(s, sv)), sub2(bh, sv));
    const u64 d = sub2(ah, bh);
    const u64 dv = sub2(d, ah);
    const u64 ed = sub2(sub2(ah, sub2(d, dv)), add2(bh, dv));
    const u64 ls = add2(es, add2(al, bl));
    const u64 ld = add2(ed, sub2(al, bl));
    ah = s; al = ls; bh = d; bl = ld;
}

// fast renormalisation of every pair: |l| <= ulp(h) / 2 afterwards
__device__ __forceinline__ void df_renorm(u64 (&h)[NR], u64 (&l)[NR]) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const u64 nh = add2(h[r], l[r]);
        l[r] = sub2(l[r], sub2(nh, h[r]));
        h[r] = nh;
    }
}

// unnormalised Walsh-Hadamard butterflies on the register bits of mask
__device__ __forceinline__ void df_hadamard(u64 (&h)[NR], u64 (&l)[NR], unsigned mask) {
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        if (!((mask >> k) & 1u)) continue;
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (!((r >> k) & 1)) df_butterfly_lazy(h[r], l[r], h[r | (1 << k)], l[r | (1 << k)]);
    }
}

// t * x for a double-float scalar t = (th, th) + (tl, tl) and pair x: unnormalised
// product (p, e), p = RN(th xh), e = its exact error plus the cross terms
__device__ __forceinline__ void df_scale_lazy(u64 th, u64 tl, u64 xh, u64 xl, u64 &p, u64 &e) {
    p = mul2(th, xh);
    e = prod_err(th, xh, p);
    e = fma2p(th, xl, e);
    e = fma2p(tl, xh, e);
}

// tangent-form rotation of a pair, without renormalisation: a' = a + t b, b' = b - t a
__device__ __forceinline__ void df_rot_lazy(u64 &ah, u64 &al, u64 &bh, u64 &bl, u64 th, u64 tl) {
    u64 pb, eb, pa, ea;
    df_scale_lazy(th, tl, bh, bl, pb, eb);
    df_scale_lazy(th, tl, ah, al, pa, ea);
    const u64 s = add2(ah, pb);
    const u64 sv = sub2(s, ah);
    const u64 es = add2(sub2(ah, sub2(s, sv)), sub2(pb, sv));
    const u64 ls = add2(es, add2(al, eb));
    const u64 d = sub2(bh, pa);
    const u64 dv = sub2(d, bh);
    const u64 ed = sub2(sub2(bh, sub2(d, dv)), add2(pa, dv));
    const u64 ld = add2(ed, sub2(bl, ea));
    ah = s; al = ls; bh = d; bl = ld;
}

// rotations on the register bits of mask; tc[k] = {(th, th), (tl, tl)} of bit k's class
__device__ __forceinline__ void df_rotate(u64 (&h)[NR], u64 (&l)[NR], unsigned mask, const u64 (*tc)[2]) {
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        if (!((mask >> k) & 1u)) continue;
        const u64 th = tc[k][0], tl = tc[k][1];
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (!((r >> k) & 1)) df_rot_lazy(h[r], l[r], h[r | (1 << k)], l[r | (1 << k)], th, tl);
    }
}

// v * i^k on both parts (exact)
__device__ __forceinline__ void df_ipow(u64 &h, u64 &l, int k) {
    const float2 a = mul_ipow(unpk(h), k), b = mul_ipow(unpk(l), k);
    h = pk(a.x, a.y);
    l = pk(b.x, b.y);
}

// Phase table entry in double-float, packed for the complex product
// v (c + i s) = (vr c - vi s, vi c + vr s) = v*(c, c) + swap(v*(s, -s)).
struct DfPhase { u64 ch, cl, sh, sl; };

__device__ __forceinline__ void df_phase(u64 &vh, u64 &vl, const DfPhase &q) {
    u64 ah, al, bh, bl;
    df_mul(vh, vl, q.ch, q.cl, ah, al);   // (vr c, vi c)
    df_mul(vh, vl, q.sh, q.sl, bh, bl);   // (vr s, -vi s)
    df_add(ah, al, swap2(bh), swap2(bl), vh, vl);
}

// Split of a double into two floats with integer operations (GB300's FP64 conversions
// run at the FP64 rate): hi = d with its binary fraction cut to 23 bits (truncation),
// lo = the 29 dropped fraction bits as a float (rounded to 24 bits), so hi + lo keeps 48
// significand bits.  |d| below 2^-126 (no normal float hi) maps to (0, 0): the state's
// amplitudes are at most 1, so that drops less than 2^-126 absolute.
__device__ __forceinline__ void split_double(double d, float &hi, float &lo) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned int top = (unsigned int)(u >> 32), bot = (unsigned int)u;
    const unsigned int sign = top & 0x80000000u;
    const int e = (int)((top >> 20) & 0x7ffu);          // biased double exponent
    const int E = e - 896;                               // biased float exponent of hi
    if (e == 0x7ff || E >= 255) { hi = __double2float_rn(d); lo = 0.f; return; }   // keeps inf / NaN
    if (E <= 0) { hi = 0.f; lo = 0.f; return; }
    hi = __uint_as_float(sign | ((unsigned int)E << 23) | ((top & 0xfffffu) << 3) | (bot >> 29));
    const unsigned int r = bot & 0x1fffffffu;            // dropped bits, units of 2^(e-1075)
    const int El = e - 948;                              // biased float exponent of 2^(e-1075)
    // below the normal range the power of two is applied in two factors (El + 64 > 12 here)
    const float v = El > 0 ? __uint2float_rn(r) * __uint_as_float((unsigned int)El << 23)
                           : __uint2float_rn(r) * __uint_as_float((unsigned int)(El + 64) << 23) * 0x1p-64f;
    lo = __uint_as_float(__float_as_uint(v) | sign);
}

// hi + lo as a double: exact conversions of both floats by bit assembly, one FP64 add
__device__ __forceinline__ double float_to_double_bits(float f) {
    const unsigned int b = __float_as_uint(f);
    const unsigned int E = (b >> 23) & 0xffu;
    if (E == 0 || E == 255) return (double)f;            // zero, subnormal, inf, NaN
    const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                                 ((unsigned long long)(E + 896u) << 52) |
                                 ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}

// In-place conversion of complex128 amplitudes to the blocked double-float layout and
// back: a warp takes four runs of two 16-amplitude blocks (one amplitude per lane and
// run, four loads in flight), reads them whole, and writes them after __syncwarp, so no
// block is read after another lane wrote to it.  n_amps is a multiple of 128.
constexpr int DF_RUNS = 4;

__global__ void k_df_split(double2 *__restrict__ state, long long n_amps) {
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    for (long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); 32 * DF_RUNS * w < n_amps;
         w += warps) {
        double2 v[DF_RUNS];
#pragma unroll
        for (int k = 0; k < DF_RUNS; ++k) v[k] = state[32 * (DF_RUNS * w + k) + lane];
        __syncwarp();
#pragma unroll
        for (int k = 0; k < DF_RUNS; ++k) {
            const long long g = 32 * (DF_RUNS * w + k) + lane;
            float rh, rl, ih, il;
            split_double(v[k].x, rh, rl);
            split_double(v[k].y, ih, il);
            float2 *blk = reinterpret_cast<float2 *>(state + (g & ~15ll));
            blk[g & 15] = make_float2(rh, ih);
            blk[16 + (g & 15)] = make_float2(rl, il);
        }
    }
}

__global__ void k_df_join(double2 *__restrict__ state, long long n_amps) {
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    for (long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); 32 * DF_RUNS * w < n_amps;
         w += warps) {
        float2 h[DF_RUNS], l[DF_RUNS];
#pragma unroll
        for (int k = 0; k < DF_RUNS; ++k) {
            const long long g = 32 * (DF_RUNS * w + k) + lane;
            const float2 *blk = reinterpret_cast<const float2 *>(state + (g & ~15ll));
            h[k] = blk[g & 15];
            l[k] = blk[16 + (g & 15)];
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < DF_RUNS; ++k)
            state[32 * (DF_RUNS * w + k) + lane] =
                make_double2(float_to_double_bits(h[k].x) + float_to_double_bits(l[k].x),
                             float_to_double_bits(h[k].y) + float_to_double_bits(l[k].y));
    }
}

// One Walsh-Hadamard pass over a state in the blocked double-float layout: tile pairs
// (high, low) by TMA into one buffer per CTA (two CTAs per SM); the next pair's load is
// issued as soon as the current pair's last stage has been read from shared memory, and
// both halves go back by per-thread stores from registers while that load is in flight.
template <bool MERGED, bool ROT>
__global__ void __launch_bounds__(NT, 2) k_xpass_df(float2 *__restrict__ state, const double *__restrict__ recs,
                                                    const double *__restrict__ recs2,
                                                    int rec_stride, int tiles_shift, int *__restrict__ err_flag,
                                                    const __grid_constant__ CUtensorMap tmap_h,
                                                    const __grid_constant__ CUtensorMap tmap_l,
                                                    const __grid_constant__ TmaPass P) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base_ptr = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    float2 *buf = reinterpret_cast<float2 *>(base_ptr);                  // (high, low) tile pair
    u64 *lut = reinterpret_cast<u64 *>(buf + 2 * (1 << LT));              // 4 u64 per entry
    uint2 *ptab = reinterpret_cast<uint2 *>(lut + 4 * (P.apply_z ? (P.nA + 1) * (P.nB + 1) : 0));
    __shared__ uint64_t bar;
    __shared__ int s_ok;
    __shared__ u64 s_tc[2][3][RB][2];   // ROT: per round, stage and register bit: (th, th), (tl, tl)
    __shared__ u64 s_xs[2];             // ROT: C of the group, (Ch, Ch), (Cl, Cl)

    const int t = threadIdx.x;
    const long long G = gridDim.x;
    const long long T = P.total_tiles;
    const long long first = blockIdx.x;
    const long long max_wait = 2000000000ll;
    if (t == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
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
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    auto issue = [&](long long tile) {
        const int x2 = (int)(tile & ((1ll << P.mid_bits) - 1));
        const int x4 = (int)(tile >> P.mid_bits);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&bar, 2 * TMA_TILE_BYTES);
        tma_load_5d(buf, &tmap_h, &bar, 0, 0, x2, 0, x4);
        tma_load_5d(buf + (1 << LT), &tmap_l, &bar, 0, 0, x2, 0, x4);
    };
    const int n_my = first < T ? (int)((T - first + G - 1) / G) : 0;
    if (t == 0 && n_my > 0) issue(first);

    const int tlo = t & 15, thi = t >> 4;
    const int a_base = swz128(t);
    int c_base[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) c_base[j] = (tlo ^ (j << 1)) | (thi << 8);
    const int b_base = t << 3, b_x = t & 7;
    // global amplitude offsets of this thread without its low four bits (global bits 0..3
    // are local bits 0..3 = tlo in the stage-C and stage-A layouts)
    long long toff_c = 0, toff_a = 0;
    uint32_t pa_t = 0, pb_t = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if ((thi >> j) & 1) toff_c += P.toff_c[4 + j];
        if ((tlo >> j) & 1) { pa_t ^= P.pa_thr[j]; pb_t ^= P.pb_thr[j]; }
        if ((thi >> j) & 1) { pa_t ^= P.pa_thr[4 + j]; pb_t ^= P.pb_thr[4 + j]; }
    }
#pragma unroll
    for (int j = 4; j < 8; ++j)
        if ((t >> j) & 1) toff_a += P.toff_a[j];
    const int nB1 = P.nB + 1;
    const int nlut = (P.nA + 1) * nB1;
    const u64 dscale = pk(P.scale, P.scale);
    const long long tmask = (1ll << tiles_shift) - 1;
    long long cur_batch = -1;

    long long tile = first;
    for (int it = 0; it < n_my; ++it, tile += G) {
        const long long batch = tile >> tiles_shift;
        if (batch != cur_batch) {
            // phase table of this batch element: (cos, sin) in double-float, packed
            __syncthreads();
            const double *rec = recs + batch * rec_stride;
            if (ROT && t < 2 * 3 * RB) {
                // round 0: this factor group (stages A, B, C); round 1 (MERGED): the next one
                const int round = t / (3 * RB), st = (t / RB) % 3, k = t % RB;
                if (round == 0 || MERGED) {
                    const double *rr = round ? recs2 + batch * rec_stride : rec;
                    const double tv = rr[P.tan_off + ((P.cls[st] >> k) & 1)];
                    const float a = __double2float_rn(tv), b = __double2float_rn(tv - (double)a);
                    s_tc[round][st][k][0] = pk(a, a);
                    s_tc[round][st][k][1] = pk(b, b);
                }
            }
            if (ROT && t == 0) {
                const double cv = rec[P.tan_off + 2];
                const float a = __double2float_rn(cv), b = __double2float_rn(cv - (double)a);
                s_xs[0] = pk(a, a);
                s_xs[1] = pk(b, b);
            }
            if (P.apply_z) {
                const int loff = ROT ? P.tan_off + 4 : P.lut_off;   // ROT: the table scaled by C
                for (int i = t; i < nlut; i += NT) {
                    const double c = 1.0 - rec[loff + 2 * i], s = rec[loff + 2 * i + 1];
                    const float ch = __double2float_rn(c), cl = __double2float_rn(c - (double)ch);
                    const float sh = __double2float_rn(s), sl = __double2float_rn(s - (double)sh);
                    u64 *q = lut + 4 * i;
                    q[0] = pk(ch, ch); q[1] = pk(cl, cl); q[2] = pk(sh, -sh); q[3] = pk(sl, -sl);
                }
            }
            cur_batch = batch;
            __syncthreads();
        }
        if (t == 0) {
            if (!mbar_wait_bounded(&bar, (uint32_t)(it & 1), max_wait)) {
                atomicOr(err_flag, 1);
                s_ok = 0;
            }
        }
        __syncthreads();
        if (!s_ok) return;

        u64 *th = reinterpret_cast<u64 *>(buf);
        u64 *tl = reinterpret_cast<u64 *>(buf + (1 << LT));
        u64 h[NR], l[NR];
        // ---- stage A: registers = local 8..11 ----
#pragma unroll
        for (int r = 0; r < NR; ++r) { h[r] = th[a_base + (r << TB)]; l[r] = tl[a_base + (r << TB)]; }
        const int pc_tile = __popcll(tile & tmask);
        if (ROT && (P.frame & 2)) {   // psi -> phi = i^popc psi
            const int k0 = __popc(t) + pc_tile;
#pragma unroll
            for (int r = 0; r < NR; ++r) df_ipow(h[r], l[r], k0 + __popc(r));
        }
        if (ROT) df_rotate(h, l, P.rot[0], s_tc[0][0]); else df_hadamard(h, l, P.rot[0]);
#pragma unroll
        for (int r = 0; r < NR; ++r) { th[a_base + (r << TB)] = h[r]; tl[a_base + (r << TB)] = l[r]; }
        __syncthreads();
        // ---- stage B: registers = local 0..3 ----
        if (P.stage_b) {
            ulonglong2 *th2 = reinterpret_cast<ulonglong2 *>(th), *tl2 = reinterpret_cast<ulonglong2 *>(tl);
#pragma unroll
            for (int m = 0; m < NR / 2; ++m) {
                const ulonglong2 qh = th2[b_base + (m ^ b_x)], ql = tl2[b_base + (m ^ b_x)];
                h[2 * m] = qh.x; h[2 * m + 1] = qh.y;
                l[2 * m] = ql.x; l[2 * m + 1] = ql.y;
            }
            if (ROT) df_rotate(h, l, P.rot[1], s_tc[0][1]); else df_hadamard(h, l, P.rot[1]);
#pragma unroll
            for (int m = 0; m < NR / 2; ++m) {
                th2[b_base + (m ^ b_x)] = make_ulonglong2(h[2 * m], h[2 * m + 1]);
                tl2[b_base + (m ^ b_x)] = make_ulonglong2(l[2 * m], l[2 * m + 1]);
            }
            __syncthreads();
        }
        // ---- stage C: registers = local 4..7; table, scale ----
#pragma unroll
        for (int r = 0; r < NR; ++r) { h[r] = th[c_base[r & 7] + (r << 4)]; l[r] = tl[c_base[r & 7] + (r << 4)]; }
        if (!MERGED) {
            // the pair's last shared-memory read: the next pair may load
            __syncthreads();
            if (t == 0 && it + 1 < n_my) issue(tile + G);
        }
        if (ROT) df_rotate(h, l, P.rot[2], s_tc[0][2]); else df_hadamard(h, l, P.rot[2]);
        const long long mid = tile & ((1ll << P.mid_bits) - 1);
        const long long up = tile >> P.mid_bits;
        const long long gbase = (mid << P.c) + (up << (P.next + P.k));
        if (P.apply_z) {
            df_renorm(h, l);
            const long long tin = tile & tmask;
            const uint2 e0 = ptab[tin & 255], e1 = ptab[256 + ((tin >> 8) & 255)], e2 = ptab[512 + ((tin >> 16) & 255)];
            const uint32_t pa = pa_t ^ e0.x ^ e1.x ^ e2.x;
            const uint32_t pb = pb_t ^ e0.y ^ e1.y ^ e2.y;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const u64 *q = lut + 4 * (__popc(pa ^ P.pa_reg[r]) * nB1 + __popc(pb ^ P.pb_reg[r]));
                DfPhase ph;
                ph.ch = q[0]; ph.cl = q[1]; ph.sh = q[2]; ph.sl = q[3];
                df_phase(h[r], l[r], ph);
            }
            if (P.scale != 1.0f) {   // a power of two: exact on both parts
#pragma unroll
                for (int r = 0; r < NR; ++r) { h[r] = mul2(h[r], dscale); l[r] = mul2(l[r], dscale); }
            }
        }
        if (ROT && !P.apply_z && P.xscale) {   // C of a factor group without Z layer
            const u64 ch = s_xs[0], cl = s_xs[1];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                u64 p, e;
                df_scale_lazy(ch, cl, h[r], l[r], p, e);
                h[r] = p; l[r] = e;
            }
        }
        if (ROT && !MERGED && (P.frame & 4)) {   // phi -> psi
            const int k0 = -(__popc(tlo) + __popc(thi) + pc_tile);
#pragma unroll
            for (int r = 0; r < NR; ++r) df_ipow(h[r], l[r], (k0 - __popc(r)) & 3);
        }
        u64 *dst;
        if (MERGED) {
            // ---- second round: stage C (in registers), B, A; store from stage A ----
            if (ROT) df_rotate(h, l, P.rot[2], s_tc[1][2]); else df_hadamard(h, l, P.rot[2]);
#pragma unroll
            for (int r = 0; r < NR; ++r) { th[c_base[r & 7] + (r << 4)] = h[r]; tl[c_base[r & 7] + (r << 4)] = l[r]; }
            __syncthreads();
            if (P.stage_b) {
                ulonglong2 *th2 = reinterpret_cast<ulonglong2 *>(th), *tl2 = reinterpret_cast<ulonglong2 *>(tl);
#pragma unroll
                for (int m = 0; m < NR / 2; ++m) {
                    const ulonglong2 qh = th2[b_base + (m ^ b_x)], ql = tl2[b_base + (m ^ b_x)];
                    h[2 * m] = qh.x; h[2 * m + 1] = qh.y;
                    l[2 * m] = ql.x; l[2 * m + 1] = ql.y;
                }
                if (ROT) df_rotate(h, l, P.rot[1], s_tc[1][1]); else df_hadamard(h, l, P.rot[1]);
#pragma unroll
                for (int m = 0; m < NR / 2; ++m) {
                    th2[b_base + (m ^ b_x)] = make_ulonglong2(h[2 * m], h[2 * m + 1]);
                    tl2[b_base + (m ^ b_x)] = make_ulonglong2(l[2 * m], l[2 * m + 1]);
                }
                __syncthreads();
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) { h[r] = th[a_base + (r << TB)]; l[r] = tl[a_base + (r << TB)]; }
            __syncthreads();
            if (t == 0 && it + 1 < n_my) issue(tile + G);
            if (ROT) df_rotate(h, l, P.rot[0], s_tc[1][0]); else df_hadamard(h, l, P.rot[0]);
            if (ROT && (P.frame & 4)) {   // phi -> psi
                const int k0 = -(__popc(t) + pc_tile);
#pragma unroll
                for (int r = 0; r < NR; ++r) df_ipow(h[r], l[r], (k0 - __popc(r)) & 3);
            }
            df_renorm(h, l);
            // blocked layout: amplitude g = 16 m + j has its high pair at float2 index
            // 32 m + j and its low pair at 32 m + 16 + j
            dst = reinterpret_cast<u64 *>(state) + 2 * (gbase + toff_a) + tlo;
#pragma unroll
            for (int r = 0; r < NR; ++r) { dst[2 * P.roff_a[r]] = h[r]; dst[2 * P.roff_a[r] + 16] = l[r]; }
        } else {
            df_renorm(h, l);
            dst = reinterpret_cast<u64 *>(state) + 2 * (gbase + toff_c) + tlo;
#pragma unroll
            for (int r = 0; r < NR; ++r) { dst[2 * P.roff_c[r]] = h[r]; dst[2 * P.roff_c[r] + 16] = l[r]; }
        }
    }
}

}  // namespace qsim
