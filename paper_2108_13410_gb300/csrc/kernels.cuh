// kernels.cuh -- sm_103a kernels of the Trotterised gauge-Higgs evolution.
//
// The hot path is a memory-bound butterfly over a 2^n-amplitude state vector:
//   * k_xpass   : exp(i theta_q X_q) on up to 12 qubits per HBM pass.  A CTA stages
//                 a 4096-amplitude tile (12 "local" bits chosen by the pass plan),
//                 applies 4 qubits per register stage (radix-16 butterflies in
//                 registers), transposes through shared memory between stages, and
//                 optionally applies the whole diagonal Z layer before storing
//                 (Eq. (8): all X-type factors commute, all Z-type factors commute).
//   * k_zdiag   : the Z layer alone: amplitude i gets exp(i dt s [h sum_p (-1)^{pi_p(i)}
//                 + lambda sum_b (-1)^{pi_b(i)}]), looked up from an FP64-built table
//                 indexed by the number of odd plaquettes and odd bonds of i.
//   * k_rx / k_zterm / k_xstring : one Pauli factor per launch (per-gate form).
//   * k_reduce_* / k_finish : FP64 block partials and a fixed-order final sum.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qsim {

constexpr int LT = 12;                 // tile bits (4096 amplitudes per CTA)
constexpr int RB = 4;                  // register bits per stage (16 amplitudes / thread)
constexpr int TB = LT - RB;            // thread bits
constexpr int NT = 1 << TB;            // 256 threads per CTA
constexpr int NR = 1 << RB;            // 16 registers (amplitudes) per thread
constexpr int MAXQ = 40;
constexpr int RED_THREADS = 256;
constexpr int RED_NV = 4;              // values per reduction record

// Fixed stage layouts (local bit -> register or thread):
//   stage 0: registers = local {8..11}, threads = local {0..7}       (global load)
//   stage 1: registers = local {0..3},  threads = local {4..11}      (shared memory)
//   stage 2: registers = local {4..7},  threads = local {0..3, 8..11} (global store)
struct PassDesc {
    int n;                      // qubits
    int nfixed;                 // n - LT tile-index bits
    int fixed_pos[MAXQ];        // global bit of tile-index bit k (increasing)
    int lmap[LT];               // global bit of local bit j
    int stage1_on;              // stage 1 has something to rotate
    unsigned rot_mask[3];       // per stage: register bits to rotate
    int reg_cls[3][RB];         // X class (0 link sigma^x, 1 vertex tau^x) per register bit
    int apply_z;                // multiply by a diagonal phase table before the store
    int nA, nB;                 // table dims (nA+1) x (nB+1): odd terms of the two classes
    uint32_t colA[MAXQ];        // per global qubit: class-A terms containing it (bit p)
    uint32_t colB[MAXQ];        // per global qubit: class-B terms containing it
    int hadamard;               // butterflies (a + b, a - b) instead of rotations
    int lut_off;                // offset (doubles) of the phase table in the operator record
    double scale;               // factor applied with the phase (a power of two)
};
// Diagonal tables: Z layer -- class A = plaquettes B_p, class B = bonds (gauge-Higgs)
// or sigma^z_l (unitary gauge).  In the Hadamard basis of the unitary-gauge X layer
// -- class A = stars A_v, class B = single links (X_l becomes Z_l).

// Operator record (doubles): [u_sigma, s_sigma, u_tau, s_tau, then (nA+1)(nB+1)
//   phase pairs (u, s) of exp(i phi(nA_odd, nB_odd))], where exp(i t) = (1 - u) + i s,
//   u = 1 - cos t, s = sin t (u keeps full relative precision for small angles);
//   then the Hadamard-basis X table (unitary gauge) and, at tan_off, the tangent form
//   (t_sigma, t_tau, C, 0) of the X layer (dev_tan_triple) followed by the Z table
//   scaled by C (dev_scaled_pair; same layout as the plain Z table).
__host__ __device__ inline int record_doubles(int nA, int nB) {
    int r = 4 + 2 * (nA + 1) * (nB + 1);
    return (r + 1) & ~1;
}

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

template <typename R>
__device__ __forceinline__ typename C2<R>::T mk(R x, R y) {
    typename C2<R>::T v; v.x = x; v.y = y; return v;
}

// (a, b) <- exp(i theta X) (a, b) with cos theta = 1 - u, sin theta = s:
//   a' = a - u a + i s b,  b' = b - u b + i s a
template <typename V, typename R>
__device__ __forceinline__ void xrot(V &a, V &b, R u, R s) {
    R ar = a.x, ai = a.y, br = b.x, bi = b.y;
    a.x = fma(-s, bi, fma(-u, ar, ar)); a.y = fma(s, br, fma(-u, ai, ai));
    b.x = fma(-s, ai, fma(-u, br, br)); b.y = fma(s, ar, fma(-u, bi, bi));
}

// v * exp(i t) with exp(i t) = (1 - p.x) + i p.y
template <typename V>
__device__ __forceinline__ V cphase(V v, V p) {
    V r;
    r.x = fma(-p.y, v.y, fma(-p.x, v.x, v.x));
    r.y = fma(p.y, v.x, fma(-p.x, v.y, v.y));
    return r;
}

__device__ __forceinline__ int swz(int l) { return l ^ ((l >> 4) & 15); }

// unnormalised Hadamard butterfly: (a, b) <- (a + b, a - b)
template <typename V>
__device__ __forceinline__ void hbfly(V &a, V &b) {
    V t = a;
    a.x = t.x + b.x; a.y = t.y + b.y;
    b.x = t.x - b.x; b.y = t.y - b.y;
}

template <typename R, typename V>
__device__ __forceinline__ void rotate_regs(V (&v)[NR], unsigned mask, const int (&cls)[RB],
                                            R u0, R s0, R u1, R s1, bool had = false) {
    if (had) {
#pragma unroll
        for (int k = 0; k < RB; ++k) {
            if (!((mask >> k) & 1u)) continue;
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if (!((r >> k) & 1)) hbfly(v[r], v[r | (1 << k)]);
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        if (!((mask >> k) & 1u)) continue;
        R u = cls[k] ? u1 : u0;
        R s = cls[k] ? s1 : s0;
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (!((r >> k) & 1)) xrot(v[r], v[r | (1 << k)], u, s);
    }
}

// ---------------------------------------------------------------------------
// Fused X pass (+ optional Z layer)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(NT) k_xpass(typename C2<R>::T *__restrict__ psi,
                                              long long state_stride,
                                              const double *__restrict__ recs, int rec_stride,
                                              const PassDesc *__restrict__ d) {
    using V = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *tile = reinterpret_cast<V *>(smem_raw);
    V *lut = tile + (1 << LT);
    const int t = threadIdx.x;
    psi += (long long)blockIdx.y * state_stride;
    const double *rec = recs + (long long)blockIdx.y * rec_stride;

    const long long tau = blockIdx.x;
    const int nfixed = d->nfixed;
    long long base = 0;
    for (int k = 0; k < nfixed; ++k)
        if ((tau >> k) & 1) base |= 1ll << d->fixed_pos[k];

    const R u0 = (R)rec[0], s0 = (R)rec[1], u1 = (R)rec[2], s1 = (R)rec[3];
    const int apply_z = d->apply_z;
    const bool had = d->hadamard != 0;
    const int nB1 = d->nB + 1;
    if (apply_z) {
        const int nl = (d->nA + 1) * nB1;
        const double *tab = rec + d->lut_off;
        for (int i = t; i < nl; i += NT) lut[i] = mk<R>((R)tab[2 * i], (R)tab[2 * i + 1]);
    }
    int lm[LT];
#pragma unroll
    for (int j = 0; j < LT; ++j) lm[j] = d->lmap[j];

    V v[NR];
    // ---- stage 0: global -> registers (lanes along local bits 0..4) ----
    {
        long long toff = base;
#pragma unroll
        for (int j = 0; j < TB; ++j)
            if ((t >> j) & 1) toff |= 1ll << lm[j];
        long long rs[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) rs[k] = 1ll << lm[TB + k];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            long long off = toff;
#pragma unroll
            for (int k = 0; k < RB; ++k)
                if ((r >> k) & 1) off |= rs[k];
            v[r] = psi[off];
        }
        int cls[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) cls[k] = d->reg_cls[0][k];
        rotate_regs<R>(v, d->rot_mask[0], cls, u0, s0, u1, s1, had);
#pragma unroll
        for (int r = 0; r < NR; ++r) tile[swz(t | (r << TB))] = v[r];
    }
    __syncthreads();
    // ---- stage 1: registers hold local bits 0..3 ----
    if (d->stage1_on) {
#pragma unroll
        for (int r = 0; r < NR; ++r) v[r] = tile[swz(r | (t << RB))];
        int cls[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) cls[k] = d->reg_cls[1][k];
        rotate_regs<R>(v, d->rot_mask[1], cls, u0, s0, u1, s1, had);
#pragma unroll
        for (int r = 0; r < NR; ++r) tile[swz(r | (t << RB))] = v[r];
        __syncthreads();
    }
    // ---- stage 2: registers hold local bits 4..7; store to global ----
    const int tlo = t & 15, thi = t >> 4;
#pragma unroll
    for (int r = 0; r < NR; ++r) v[r] = tile[swz(tlo | (r << 4) | (thi << 8))];
    {
        int cls[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) cls[k] = d->reg_cls[2][k];
        rotate_regs<R>(v, d->rot_mask[2], cls, u0, s0, u1, s1, had);
    }
    long long toff = base;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if ((tlo >> j) & 1) toff |= 1ll << lm[j];
        if ((thi >> j) & 1) toff |= 1ll << lm[8 + j];
    }
    long long rs[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) rs[k] = 1ll << lm[4 + k];
    if (apply_z) {
        // parity vectors: P(i) = xor of the columns of the set bits of i
        uint32_t pa = 0, pb = 0;
        for (int k = 0; k < nfixed; ++k)
            if ((tau >> k) & 1) { int g = d->fixed_pos[k]; pa ^= d->colA[g]; pb ^= d->colB[g]; }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if ((tlo >> j) & 1) { pa ^= d->colA[lm[j]]; pb ^= d->colB[lm[j]]; }
            if ((thi >> j) & 1) { pa ^= d->colA[lm[8 + j]]; pb ^= d->colB[lm[8 + j]]; }
        }
        uint32_t ra[RB], rb[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) { ra[k] = d->colA[lm[4 + k]]; rb[k] = d->colB[lm[4 + k]]; }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            uint32_t a = pa, b = pb;
#pragma unroll
            for (int k = 0; k < RB; ++k)
                if ((r >> k) & 1) { a ^= ra[k]; b ^= rb[k]; }
            v[r] = cphase(v[r], lut[__popc(a) * nB1 + __popc(b)]);
        }
        if (d->scale != 1.0) {
            const R sc = (R)d->scale;
#pragma unroll
            for (int r = 0; r < NR; ++r) { v[r].x *= sc; v[r].y *= sc; }
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        long long off = toff;
#pragma unroll
        for (int k = 0; k < RB; ++k)
            if ((r >> k) & 1) off |= rs[k];
        psi[off] = v[r];
    }
}

// ---------------------------------------------------------------------------
// Parity tables: P(i) = T[0][i & 255] ^ T[1][(i >> 8) & 255] ^ ...
// ---------------------------------------------------------------------------
constexpr int MAXBYTES = (MAXQ + 7) / 8;

__device__ __forceinline__ void build_parity_tables(uint2 *tab, const uint32_t *colA,
                                                    const uint32_t *colB, int n) {
    const int nbytes = (n + 7) / 8;
    for (int e = threadIdx.x; e < nbytes * 256; e += blockDim.x) {
        int k = e >> 8, val = e & 255;
        uint32_t a = 0, b = 0;
        for (int j = 0; j < 8; ++j) {
            int q = 8 * k + j;
            if (q < n && ((val >> j) & 1)) { a ^= colA[q]; b ^= colB[q]; }
        }
        tab[e] = make_uint2(a, b);
    }
}

__device__ __forceinline__ uint2 parity_of(const uint2 *tab, long long i, int nbytes) {
    uint32_t a = 0, b = 0;
    for (int k = 0; k < nbytes; ++k) {
        uint2 e = tab[(k << 8) | (int)((i >> (8 * k)) & 255)];
        a ^= e.x; b ^= e.y;
    }
    return make_uint2(a, b);
}

// Z layer alone, one HBM pass; grid-stride over amplitudes; blockIdx.y = batch.
template <typename R>
__global__ void __launch_bounds__(256) k_zdiag(typename C2<R>::T *__restrict__ psi, int n,
                                               long long state_stride,
                                               const double *__restrict__ recs, int rec_stride,
                                               const uint32_t *__restrict__ colA,
                                               const uint32_t *__restrict__ colB, int nA, int nB) {
    using V = typename C2<R>::T;
    __shared__ uint2 tab[MAXBYTES * 256];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *lut = reinterpret_cast<V *>(smem_raw);
    psi += (long long)blockIdx.y * state_stride;
    const double *rec = recs + (long long)blockIdx.y * rec_stride;
    build_parity_tables(tab, colA, colB, n);
    const int nB1 = nB + 1, nl = (nA + 1) * nB1;
    for (int i = threadIdx.x; i < nl; i += blockDim.x) lut[i] = mk<R>((R)rec[4 + 2 * i], (R)rec[5 + 2 * i]);
    __syncthreads();
    const int nbytes = (n + 7) / 8;
    const long long dim = 1ll << n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < dim;
         i += (long long)gridDim.x * blockDim.x) {
        uint2 p = parity_of(tab, i, nbytes);
        psi[i] = cphase(psi[i], lut[__popc(p.x) * nB1 + __popc(p.y)]);
    }
}

// ---------------------------------------------------------------------------
// Per-gate kernels (one Pauli factor per launch)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_rx(typename C2<R>::T *__restrict__ psi, int n, long long state_stride, int q,
                     R u, R s) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= (1ll << (n - 1))) return;
    psi += (long long)blockIdx.y * state_stride;
    long long lo = p & ((1ll << q) - 1);
    long long i0 = ((p >> q) << (q + 1)) | lo;
    long long i1 = i0 | (1ll << q);
    auto a = psi[i0], b = psi[i1];
    xrot(a, b, u, s);
    psi[i0] = a; psi[i1] = b;
}

template <typename R>
__global__ void k_xstring(typename C2<R>::T *__restrict__ psi, int n, long long state_stride,
                          unsigned long long mask, int top, R u, R s) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= (1ll << (n - 1))) return;
    psi += (long long)blockIdx.y * state_stride;
    long long lo = p & ((1ll << top) - 1);
    long long i0 = ((p >> top) << (top + 1)) | lo;   // bit `top` of i0 is 0
    long long i1 = i0 ^ (long long)mask;
    auto a = psi[i0], b = psi[i1];
    xrot(a, b, u, s);
    psi[i0] = a; psi[i1] = b;
}

// amplitude i <- exp(i theta (-1)^{popcount(i & mask)}) amplitude i, cos theta = 1 - u
template <typename R>
__global__ void k_zterm(typename C2<R>::T *__restrict__ psi, int n, long long state_stride,
                        unsigned long long mask, R u, R s) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (1ll << n)) return;
    psi += (long long)blockIdx.y * state_stride;
    R ss = (__popcll((unsigned long long)i & mask) & 1) ? -s : s;
    psi[i] = cphase(psi[i], mk<R>(u, ss));
}

template <typename R>
__global__ void k_fill(typename C2<R>::T *__restrict__ psi, long long count, R re) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        psi[i] = mk<R>(re, (R)0);
}

// psi_b <- psi_b / sqrt(norm_b), norm_b = res[b * RED_NV] (device, FP64)
template <typename R>
__global__ void k_scale_by_norm(typename C2<R>::T *__restrict__ psi, long long state_stride,
                                const double *__restrict__ res) {
    psi += (long long)blockIdx.y * state_stride;
    const double nrm = res[blockIdx.y * RED_NV];
    const R f = (R)(1.0 / sqrt(nrm));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < state_stride;
         i += (long long)gridDim.x * blockDim.x) {
        auto a = psi[i];
        a.x *= f; a.y *= f;
        psi[i] = a;
    }
}

// ---------------------------------------------------------------------------
// FP64 reductions: each block writes RED_NV partials; k_finish sums them in a
// fixed order (deterministic for a fixed grid).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <int NVAL>
__device__ __forceinline__ void block_store(double (&acc)[NVAL], double *out) {
    __shared__ double sh[RED_THREADS / 32][RED_NV];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int v = 0; v < NVAL; ++v) {
        double x = warp_sum(acc[v]);
        if (l == 0) sh[w][v] = x;
    }
    __syncthreads();
    if (threadIdx.x < NVAL) {
        double s = 0.0;
        for (int k = 0; k < RED_THREADS / 32; ++k) s += sh[k][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// values: [norm, sum_i p_i (nA - 2 oddA(i)), sum_i p_i (nB - 2 oddB(i)), <Z_zmask>],
// p_i = |psi_i|^2.  Products are summed in the state's precision over runs of
// RED_RUN amplitudes (exact enough: 8 terms of one sign-pattern), and the runs are
// accumulated in FP64.
constexpr int RED_RUN = 8;

template <typename R>
__global__ void __launch_bounds__(RED_THREADS) k_reduce_diag(
    const typename C2<R>::T *__restrict__ psi, int n, long long state_stride,
    const uint32_t *__restrict__ colA, const uint32_t *__restrict__ colB, int nA, int nB,
    unsigned long long zmask, double *__restrict__ partials) {
    __shared__ uint2 tab[MAXBYTES * 256];
    psi += (long long)blockIdx.y * state_stride;
    build_parity_tables(tab, colA, colB, n);
    __syncthreads();
    const int nbytes = (n + 7) / 8;
    const long long dim = 1ll << n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < dim; i0 += stride * RED_RUN) {
        R f[4] = {0, 0, 0, 0};
#pragma unroll
        for (int u = 0; u < RED_RUN; ++u) {
            long long i = i0 + u * stride;
            if (i < dim) {
                auto a = psi[i];
                R p = a.x * a.x + a.y * a.y;
                uint2 par = parity_of(tab, i, nbytes);
                f[0] += p;
                f[1] += p * (R)(nA - 2 * __popc(par.x));
                f[2] += p * (R)(nB - 2 * __popc(par.y));
                f[3] += (__popcll((unsigned long long)i & zmask) & 1) ? -p : p;
            }
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] += (double)f[v];
    }
    block_store<4>(acc, partials + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * RED_NV);
}

// sum_i conj(a_i) b_{i ^ mask} (re, im); with a == b this is <X_mask>
template <typename R>
__global__ void __launch_bounds__(RED_THREADS) k_reduce_xmask(
    const typename C2<R>::T *__restrict__ a, const typename C2<R>::T *__restrict__ b, int n,
    long long state_stride, unsigned long long mask, double *__restrict__ partials) {
    a += (long long)blockIdx.y * state_stride;
    b += (long long)blockIdx.y * state_stride;
    const long long dim = 1ll << n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    double acc[2] = {0.0, 0.0};
    for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < dim; i0 += stride * RED_RUN) {
        R f0 = 0, f1 = 0;
#pragma unroll
        for (int u = 0; u < RED_RUN; ++u) {
            long long i = i0 + u * stride;
            if (i < dim) {
                auto x = a[i];
                auto y = b[i ^ (long long)mask];
                f0 += x.x * y.x + x.y * y.y;
                f1 += x.x * y.y - x.y * y.x;
            }
        }
        acc[0] += (double)f0;
        acc[1] += (double)f1;
    }
    block_store<2>(acc, partials + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * RED_NV);
}

// res[b * RED_NV + v] = sum over the nblk partials of batch b (fixed order)
__global__ void k_finish(const double *__restrict__ partials, int nblk, int nval,
                         double *__restrict__ res) {
    __shared__ double sh[RED_THREADS];
    const int b = blockIdx.x;
    for (int v = 0; v < nval; ++v) {
        double s = 0.0;
        for (int k = threadIdx.x; k < nblk; k += blockDim.x)
            s += partials[((long long)b * nblk + k) * RED_NV + v];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) res[b * RED_NV + v] = sh[0];
        __syncthreads();
    }
}

}  // namespace qsim

namespace qsim {

// ---------------------------------------------------------------------------
// Operator records built on the device from the schedule s[] and the couplings.
// A record describes one Trotter factor group: X angles per class, then the Z
// table (nA+1)(nB+1) and, for the unitary gauge, the Hadamard-basis X table.
// Every exp(i t) is stored as (u, s) = (2 sin^2(t/2), sin t) computed in FP64; for
// complex64 the float pair within +-3 ulps minimising |(1-u)^2 + s^2 - 1| is kept.
// ---------------------------------------------------------------------------
struct RecGeom {
    int n_steps, order, fsal;    // fsal: second order with merged X half-steps
    int path;                    // 1: couplings per step (cpl[k * batch + b]) with s = 1
    int batch, rec_stride;
    int nA, nB, nXA, nXB, xlut_off;
    int f32;
    int tan_off, nX0, nX1;       // tangent-form triple (0: none); X qubits per class
    double dt;
};

struct DevCouplings { double J, h, g, lambda; };

__device__ inline void dev_unit_pair(bool f32, double t, double *ou, double *os) {
    double sh = sin(0.5 * t);
    double u = 2.0 * sh * sh, s = sin(t);
    if (!f32) { *ou = u; *os = s; return; }
    float u0 = (float)u, s0 = (float)s, bu = u0, bs = s0;
    double c0 = 1.0 - (double)u0;
    double be = fabs(c0 * c0 + (double)s0 * (double)s0 - 1.0), bd = 0.0;
    float uu = u0;
    for (int i = 0; i < 3; ++i) uu = nextafterf(uu, -4.0f);
    for (int i = -3; i <= 3; ++i, uu = nextafterf(uu, 4.0f)) {
        float ss = s0;
        for (int j = 0; j < 3; ++j) ss = nextafterf(ss, -4.0f);
        for (int j = -3; j <= 3; ++j, ss = nextafterf(ss, 4.0f)) {
            double c = 1.0 - (double)uu;
            double e = fabs(c * c + (double)ss * (double)ss - 1.0);
            double dd = fabs((double)uu - u) + fabs((double)ss - s);
            if (e < be || (e == be && dd < bd)) { be = e; bd = dd; bu = uu; bs = ss; }
        }
    }
    *ou = bu; *os = bs;
}

// Careful pair of exp(i t) = (1 - u) + i s for per-step tables built inside a kernel:
// one FP64 sincos, then a 3 x 3 search over the float neighbours of s and of the u that
// makes (1 - u)^2 + s^2 = 1 for each of them, keeping the pair with the smallest
// |(1 - u)^2 + s^2 - 1| (evaluated in FP64).  complex128 tables take (u, s) as they are.
// About a tenth of dev_unit_pair's FP64 work, which matters where a table is rebuilt
// for every Trotter step inside a persistent kernel (GB300 retires about two FP64 FMAs
// per clock per SM).
template <typename R>
__device__ inline void dev_unit_pair_fast(double t, R *ou, R *os) {
    double sh, ch;
    sincos(0.5 * t, &sh, &ch);
    const double u = 2.0 * sh * sh, s = 2.0 * sh * ch;
    if (sizeof(R) == 8) { *ou = (R)u; *os = (R)s; return; }
    const bool neg = u > 1.0;           // cos t < 0: 1 - u = -sqrt(1 - s^2)
    float bu = (float)u, bs = (float)s;
    double be = 1e300;
    float sc = nextafterf((float)s, -4.0f);
    for (int i = 0; i < 3; ++i, sc = nextafterf(sc, 4.0f)) {
        const double s2 = (double)sc * (double)sc;
        const double r = sqrt(fmax(0.0, 1.0 - s2));
        const double us = neg ? 1.0 + r : s2 / (1.0 + r);
        float uc = nextafterf((float)us, -4.0f);
        for (int j = 0; j < 3; ++j, uc = nextafterf(uc, 4.0f)) {
            const double c = 1.0 - (double)uc;
            const double e = fabs(c * c + s2 - 1.0);
            if (e < be) { be = e; bu = uc; bs = sc; }
        }
    }
    *ou = (R)bu; *os = (R)bs;
}

// X angles and Z angles of factor group `op` for couplings c:
//   order 1:      op k (< N): X theta(s_k) dt, Z at s_k
//   second order: op k (<= N): X theta(s_k) dt/2 [k < N] + theta(s_{k-1}) dt/2 [k > 0],
//                 Z at s_k for k < N (the last group is the trailing X half-step)
//   path mode: step k uses H1 with couplings cpl[k * batch + b] (s = 1)
__device__ inline void dev_op_angles(const RecGeom &G, const DevCouplings *__restrict__ cpl, int b,
                                     const double *__restrict__ sv, int op, double *thx, double *zA, double *zB,
                                     bool *has_z) {
    thx[0] = thx[1] = 0.0;
    *zA = *zB = 0.0;
    *has_z = false;
    const int N = G.n_steps;
    auto cp = [&](int k) -> const DevCouplings & { return G.path ? cpl[(long long)k * G.batch + b] : cpl[b]; };
    auto sk = [&](int k) -> double { return G.path ? 1.0 : sv[k]; };
    auto add = [&](int k, double tau) {
        const double s = sk(k);
        const DevCouplings &c = cp(k);
        thx[0] += ((1.0 - s) + s * c.g) * tau;
        thx[1] += ((1.0 - s) + s * c.J) * tau;
    };
    auto zs = [&](int k) {
        const double s = sk(k);
        const DevCouplings &c = cp(k);
        *zA = s * c.h * G.dt; *zB = s * c.lambda * G.dt; *has_z = true;
    };
    if (!G.fsal) {
        add(op, G.dt);
        zs(op);
    } else {
        if (op < N) add(op, 0.5 * G.dt);
        if (op > 0) add(op - 1, 0.5 * G.dt);
        if (op < N) zs(op);
    }
}

// Tangent form of one X layer for the complex64 kernels.  In the real-rotation frame
// exp(i th X) is cos th [[1, t], [-t, 1]] with t = tan th: a butterfly a' = a + t b,
// b' = b - t a (one rounded FMA per output), and the cos th of all n0 + n1 X qubits
// multiply to one scalar C, applied once per factor group.  t is rounded to the kernel
// precision and C is computed in FP64 from the rounded t, C = (1 + t0^2)^(-n0/2)
// (1 + t1^2)^(-n1/2), so the butterflies and C together keep the norm exactly; C is
// applied through the scaled Z table (dev_scaled_pair) or, for a factor group without
// a Z layer, rounded once.  Used when |th| <= pi/4 and C >= 1/2 (the host checks;
// otherwise the (u, s) form runs).  o = [t0, t1, C, 0].
__device__ inline void dev_tan_triple(bool f32, double th0, double th1, int n0, int n1, double *o) {
    double t0 = tan(th0), t1 = tan(th1);
    if (f32) { t0 = (double)(float)t0; t1 = (double)(float)t1; }
    o[0] = t0; o[1] = t1;
    o[2] = pow(1.0 + t0 * t0, -0.5 * n0) * pow(1.0 + t1 * t1, -0.5 * n1);
    o[3] = 0.0;
}

// C exp(i phi) as (u, s) with (1 - u) + i s, u = 1 - C cos phi, s = C sin phi; for
// complex64 the float pair within +-3 ulps of each component minimising
// |(1 - u)^2 + s^2 - C^2| (in double), so the modulus of every table entry is C to
// ~1e-10 relative, as the unit pairs of dev_unit_pair are 1.
__device__ inline void dev_scaled_pair(bool f32, double phi, double C, double *ou, double *os) {
    const double sh = sin(0.5 * phi);
    const double u = (1.0 - C) + C * 2.0 * sh * sh, s = C * sin(phi);
    if (!f32) { *ou = u; *os = s; return; }
    const double C2 = C * C;
    float u0 = (float)u, s0 = (float)s, bu = u0, bs = s0;
    double c0 = 1.0 - (double)u0;
    double be = fabs(c0 * c0 + (double)s0 * (double)s0 - C2), bd = 0.0;
    float uu = u0;
    for (int i = 0; i < 3; ++i) uu = nextafterf(uu, -4.0f);
    for (int i = -3; i <= 3; ++i, uu = nextafterf(uu, 4.0f)) {
        float ss = s0;
        for (int j = 0; j < 3; ++j) ss = nextafterf(ss, -4.0f);
        for (int j = -3; j <= 3; ++j, ss = nextafterf(ss, 4.0f)) {
            const double c = 1.0 - (double)uu;
            const double e = fabs(c * c + (double)ss * (double)ss - C2);
            const double dd = fabs((double)uu - u) + fabs((double)ss - s);
            if (e < be || (e == be && dd < bd)) { be = e; bd = dd; bu = uu; bs = ss; }
        }
    }
    *ou = bu; *os = bs;
}

// one thread per (op, batch, entry); entry 0 = X header, then Z table, then X table;
// records of ops op0 .. op0 + n_ops - 1 are written from recs[0]
__global__ void k_build_records(RecGeom G, const DevCouplings *__restrict__ cpl, const double *__restrict__ sv,
                                int op0, int n_ops, double *__restrict__ recs) {
    const int nz = (G.nA + 1) * (G.nB + 1);
    const int nx = G.xlut_off > 0 ? (G.nXA + 1) * (G.nXB + 1) : 0;
    const int nt = G.tan_off > 0 ? nz : 0;
    const long long per = 1 + nz + nx + nt;
    const long long total = (long long)n_ops * G.batch * per;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
        const long long ob = id / per;
        const int e = (int)(id - ob * per);
        const int op = op0 + (int)(ob / G.batch), b = (int)(ob % G.batch);
        double thx[2], zA, zB;
        bool has_z;
        dev_op_angles(G, cpl, b, sv, op, thx, &zA, &zB, &has_z);
        double *r = recs + ob * G.rec_stride;
        if (e == 0) {
            dev_unit_pair(G.f32, thx[0], &r[0], &r[1]);
            dev_unit_pair(G.f32, thx[1], &r[2], &r[3]);
            if (G.tan_off > 0) dev_tan_triple(G.f32, thx[0], thx[1], G.nX0, G.nX1, &r[G.tan_off]);
        } else if (e <= nz) {
            const int k = e - 1, a = k / (G.nB + 1), bb = k % (G.nB + 1);
            double phi = has_z ? zA * (double)(G.nA - 2 * a) + zB * (double)(G.nB - 2 * bb) : 0.0;
            dev_unit_pair(G.f32, phi, &r[4 + 2 * k], &r[5 + 2 * k]);
        } else if (e <= nz + nx) {
            const int k = e - 1 - nz, a = k / (G.nXB + 1), bb = k % (G.nXB + 1);
            double phi = thx[1] * (double)(G.nXA - 2 * a) + thx[0] * (double)(G.nXB - 2 * bb);
            dev_unit_pair(G.f32, phi, &r[G.xlut_off + 2 * k], &r[G.xlut_off + 2 * k + 1]);
        } else {
            // Z table scaled by the tangent form's C
            const int k = e - 1 - nz - nx, a = k / (G.nB + 1), bb = k % (G.nB + 1);
            double tc[4];
            dev_tan_triple(G.f32, thx[0], thx[1], G.nX0, G.nX1, tc);
            double phi = has_z ? zA * (double)(G.nA - 2 * a) + zB * (double)(G.nB - 2 * bb) : 0.0;
            double *tl = r + G.tan_off + 4;
            dev_scaled_pair(G.f32, phi, tc[2], &tl[2 * k], &tl[2 * k + 1]);
        }
    }
}

}  // namespace qsim

namespace qsim {

// Density of states of Z~ = -sum_l sigma^z_l (Sec. V): P(k) = sum over amplitudes with k
// links in sigma^z = -1 of |psi_i|^2 (Z~ = 2k - n_links).  Per-block bins in shared
// memory (FP64 atomics), then per-block partials; partials[(b * gridDim.x + blk) * nbins + k].
template <typename R>
__global__ void __launch_bounds__(RED_THREADS) k_dos(const typename C2<R>::T *__restrict__ psi, int n,
                                                     long long state_stride, unsigned long long linkmask, int nbins,
                                                     double *__restrict__ partials) {
    __shared__ double bins[64];
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) bins[k] = 0.0;
    __syncthreads();
    psi += (long long)blockIdx.y * state_stride;
    const long long dim = 1ll << n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < dim;
         i += (long long)gridDim.x * blockDim.x) {
        auto a = psi[i];
        double p = (double)a.x * (double)a.x + (double)a.y * (double)a.y;
        atomicAdd(&bins[__popcll((unsigned long long)i & linkmask)], p);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nbins; k += blockDim.x)
        partials[((long long)blockIdx.y * gridDim.x + blockIdx.x) * nbins + k] = bins[k];
}

// out[b * nval + v] = sum over nblk partials (layout [b][blk][v]), fixed order
__global__ void k_finish_wide(const double *__restrict__ partials, int nblk, int nval, double *__restrict__ out) {
    const int b = blockIdx.x;
    for (int v = threadIdx.x; v < nval; v += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nblk; ++k) s += partials[((long long)b * nblk + k) * nval + v];
        out[(long long)b * nval + v] = s;
    }
}

}  // namespace qsim

namespace qsim {

// Toric-code initial states of Sec. IV (before normalisation): amplitude 1 where every
// plaquette parity is even (psi_1: the B_p = +1 projection of |+>), and additionally both
// Wilson-loop masks w0, w1 even (psi_1': the A_v = +1 projection of |0...0>, whose support
// is the star-flip orbit of |0...0>, i.e. the configurations orthogonal to every closed
// loop); 0 elsewhere.
template <typename R>
__global__ void k_init_even(typename C2<R>::T *__restrict__ psi, int n, long long state_stride,
                            const uint32_t *__restrict__ colA, unsigned long long w0, unsigned long long w1) {
    __shared__ uint2 tab[MAXBYTES * 256];
    // parity table of the plaquette columns only
    for (int e = threadIdx.x; e < ((n + 7) / 8) * 256; e += blockDim.x) {
        int k = e >> 8, val = e & 255;
        uint32_t a = 0;
        for (int j = 0; j < 8; ++j) {
            int q = 8 * k + j;
            if (q < n && ((val >> j) & 1)) a ^= colA[q];
        }
        tab[e] = make_uint2(a, 0u);
    }
    __syncthreads();
    psi += (long long)blockIdx.y * state_stride;
    const int nbytes = (n + 7) / 8;
    const long long dim = 1ll << n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < dim;
         i += (long long)gridDim.x * blockDim.x) {
        const uint2 p = parity_of(tab, i, nbytes);
        const bool keep = p.x == 0 && !(__popcll((unsigned long long)i & w0) & 1) &&
                          !(__popcll((unsigned long long)i & w1) & 1);
        psi[i] = mk<R>(keep ? (R)1 : (R)0, (R)0);
    }
}

}  // namespace qsim
