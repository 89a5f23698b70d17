// adjoint.cuh -- reverse-mode (adjoint) kernels for d<value>/ds_k.
//
// Forward: psi_N = F_L ... F_1 psi_0, every factor F = exp(i theta(s) P) with P a
// Pauli string of one commuting group (Eq. (8)).  For a scalar value V(psi_N)
// seeded by lambda = dV/d<psi_N| (lambda = H1 psi_N for the energy), the derivative
// with respect to the angle of a factor is
//     dV/dtheta = 2 Re <lambda_j| i P |psi_j> = -2 Im <lambda_j|P|psi_j>,
// with psi_j, lambda_j both taken just after that factor.  Walking the factors in
// reverse, psi and lambda are uncomputed together (F^dagger = angle -theta), so no
// intermediate state is stored.  Inside one commuting group every P commutes with
// the group's other factors, so all of the group's contributions can be read at the
// same point.  Per Trotter factor group the kernels return, per batch element,
//     [ sum_{q in class sigma} Im<lambda|X_q|psi>, sum_{q in class tau} Im<lambda|X_q|psi>,
//       sum_i Im(conj(lambda_i) psi_i) (nA - 2 oddA(i)), sum_i Im(conj(lambda_i) psi_i) (nB - 2 oddB(i)) ]
// and the host combines them with d theta / d s_k.
#pragma once
#include "kernels.cuh"

namespace qsim {

// Im( conj(la) pb + conj(lb) pa ): the pair's share of Im<lambda|X_q|psi>
template <typename V, typename R>
__device__ __forceinline__ R pair_im(const V &pa, const V &pb, const V &la, const V &lb) {
    return la.x * pb.y - la.y * pb.x + lb.x * pa.y - lb.y * pa.x;
}

template <typename R, typename V>
__device__ __forceinline__ void adj_stage(V (&p)[NR], V (&l)[NR], unsigned mask, const int (&cls)[RB], R u0, R s0,
                                          R u1, R s1, R &g0, R &g1) {
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        if (!((mask >> k) & 1u)) continue;
        const bool c = cls[k] != 0;
        const R u = c ? u1 : u0;
        const R s = c ? s1 : s0;     // already negated: the inverse rotation
        R g = 0;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if ((r >> k) & 1) continue;
            const int q = r | (1 << k);
            g += pair_im<V, R>(p[r], p[q], l[r], l[q]);
            xrot(p[r], p[q], u, s);
            xrot(l[r], l[q], u, s);
        }
        if (c) g1 += g; else g0 += g;
    }
}

// One reverse X pass over psi and lambda (register-staged tiles, grid-stride over
// tiles).  zinv: first undo the Z layer (phase table conjugated) and accumulate the
// Z-group values.  partials[(b * nblk + slot0 + blockIdx.x) * RED_NV + v].
template <typename R>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 2 : 1) k_adj_xpass(typename C2<R>::T *__restrict__ psi,
                                                  typename C2<R>::T *__restrict__ lam, long long state_stride,
                                                  long long ntiles, const double *__restrict__ recs,
                                                  int rec_stride, const PassDesc *__restrict__ d, int zinv,
                                                  double *__restrict__ partials, int nblk, int slot0) {
    using V = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *tp = reinterpret_cast<V *>(smem_raw);
    V *tl = tp + (1 << LT);
    V *lut = tl + (1 << LT);
    const int t = threadIdx.x;
    psi += (long long)blockIdx.y * state_stride;
    lam += (long long)blockIdx.y * state_stride;
    const double *rec = recs + (long long)blockIdx.y * rec_stride;
    const R u0 = (R)rec[0], s0 = -(R)rec[1], u1 = (R)rec[2], s1 = -(R)rec[3];
    const int nB1 = d->nB + 1, nA = d->nA, nB = d->nB;
    if (zinv) {
        const int nl = (nA + 1) * nB1;
        for (int i = t; i < nl; i += NT) lut[i] = mk<R>((R)rec[4 + 2 * i], -(R)rec[5 + 2 * i]);
    }
    int lm[LT];
#pragma unroll
    for (int j = 0; j < LT; ++j) lm[j] = d->lmap[j];
    int cls0[RB], cls1[RB], cls2[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) { cls0[k] = d->reg_cls[0][k]; cls1[k] = d->reg_cls[1][k]; cls2[k] = d->reg_cls[2][k]; }
    const unsigned rm0 = d->rot_mask[0], rm1 = d->rot_mask[1], rm2 = d->rot_mask[2];
    const int nfixed = d->nfixed;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    __syncthreads();

    for (long long tau = blockIdx.x; tau < ntiles; tau += gridDim.x) {
        long long base = 0;
        for (int k = 0; k < nfixed; ++k)
            if ((tau >> k) & 1) base |= 1ll << d->fixed_pos[k];
        R g0 = 0, g1 = 0, ga = 0, gb = 0;
        V p[NR], l[NR];
        // ---- stage 0: global -> registers (local bits 8..11 in registers) ----
        {
            long long toff = base;
#pragma unroll
            for (int j = 0; j < TB; ++j)
                if ((t >> j) & 1) toff |= 1ll << lm[j];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                long long off = toff;
#pragma unroll
                for (int k = 0; k < RB; ++k)
                    if ((r >> k) & 1) off |= 1ll << lm[TB + k];
                p[r] = psi[off];
                l[r] = lam[off];
            }
            if (zinv) {
                uint32_t pa = 0, pb = 0;
                for (int k = 0; k < nfixed; ++k)
                    if ((tau >> k) & 1) { int g = d->fixed_pos[k]; pa ^= d->colA[g]; pb ^= d->colB[g]; }
#pragma unroll
                for (int j = 0; j < TB; ++j)
                    if ((t >> j) & 1) { pa ^= d->colA[lm[j]]; pb ^= d->colB[lm[j]]; }
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    uint32_t a = pa, b = pb;
#pragma unroll
                    for (int k = 0; k < RB; ++k)
                        if ((r >> k) & 1) { a ^= d->colA[lm[TB + k]]; b ^= d->colB[lm[TB + k]]; }
                    const int oa = __popc(a), ob = __popc(b);
                    const R im = l[r].x * p[r].y - l[r].y * p[r].x;     // Im(conj(lambda_i) psi_i)
                    ga += im * (R)(nA - 2 * oa);
                    gb += im * (R)(nB - 2 * ob);
                    const V ph = lut[oa * nB1 + ob];
                    p[r] = cphase(p[r], ph);
                    l[r] = cphase(l[r], ph);
                }
            }
            adj_stage<R>(p, l, rm0, cls0, u0, s0, u1, s1, g0, g1);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                tp[swz(t | (r << TB))] = p[r];
                tl[swz(t | (r << TB))] = l[r];
            }
        }
        __syncthreads();
        if (rm1) {
#pragma unroll
            for (int r = 0; r < NR; ++r) { p[r] = tp[swz(r | (t << RB))]; l[r] = tl[swz(r | (t << RB))]; }
            adj_stage<R>(p, l, rm1, cls1, u0, s0, u1, s1, g0, g1);
#pragma unroll
            for (int r = 0; r < NR; ++r) { tp[swz(r | (t << RB))] = p[r]; tl[swz(r | (t << RB))] = l[r]; }
            __syncthreads();
        }
        const int tlo = t & 15, thi = t >> 4;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int li = swz(tlo | (r << 4) | (thi << 8));
            p[r] = tp[li];
            l[r] = tl[li];
        }
        adj_stage<R>(p, l, rm2, cls2, u0, s0, u1, s1, g0, g1);
        long long toff = base;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if ((tlo >> j) & 1) toff |= 1ll << lm[j];
            if ((thi >> j) & 1) toff |= 1ll << lm[8 + j];
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            long long off = toff;
#pragma unroll
            for (int k = 0; k < RB; ++k)
                if ((r >> k) & 1) off |= 1ll << lm[4 + k];
            psi[off] = p[r];
            lam[off] = l[r];
        }
        acc[0] += (double)g0; acc[1] += (double)g1; acc[2] += (double)ga; acc[3] += (double)gb;
        __syncthreads();   // tiles are rewritten by the next iteration
    }
    block_store<4>(acc, partials + ((long long)blockIdx.y * nblk + slot0 + blockIdx.x) * RED_NV);
}

// lambda <- H psi for a Hamiltonian -H = sum_q c_class(q) X_q + D(i), built pass by
// pass: the first pass sets lambda_i = dtab(oddA(i), oddB(i)) psi_i; every pass adds
// c X_q psi for its rotated qubits.  Record layout as the operator records: rec[0] =
// coefficient of class 0, rec[2] = coefficient of class 1, table entries (re) = D.
template <typename R>
__global__ void __launch_bounds__(NT) k_apply_h_pass(const typename C2<R>::T *__restrict__ psi,
                                                     typename C2<R>::T *__restrict__ lam, long long state_stride,
                                                     long long ntiles, const double *__restrict__ recs,
                                                     int rec_stride, const PassDesc *__restrict__ d, int first) {
    using V = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *tp = reinterpret_cast<V *>(smem_raw);
    V *tl = tp + (1 << LT);
    R *dtab = reinterpret_cast<R *>(tl + (1 << LT));
    const int t = threadIdx.x;
    psi += (long long)blockIdx.y * state_stride;
    lam += (long long)blockIdx.y * state_stride;
    const double *rec = recs + (long long)blockIdx.y * rec_stride;
    const R c0 = (R)rec[0], c1 = (R)rec[2];
    const int nB1 = d->nB + 1;
    if (first) {
        const int nl = (d->nA + 1) * nB1;
        for (int i = t; i < nl; i += NT) dtab[i] = (R)rec[4 + 2 * i];
    }
    int lm[LT];
#pragma unroll
    for (int j = 0; j < LT; ++j) lm[j] = d->lmap[j];
    const int nfixed = d->nfixed;
    __syncthreads();
    auto add_x = [&](V (&p)[NR], V (&l)[NR], unsigned mask, int st) {
#pragma unroll
        for (int k = 0; k < RB; ++k) {
            if (!((mask >> k) & 1u)) continue;
            const R c = d->reg_cls[st][k] ? c1 : c0;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int q = r ^ (1 << k);
                l[r].x += c * p[q].x;
                l[r].y += c * p[q].y;
            }
        }
    };
    for (long long tau = blockIdx.x; tau < ntiles; tau += gridDim.x) {
        long long base = 0;
        for (int k = 0; k < nfixed; ++k)
            if ((tau >> k) & 1) base |= 1ll << d->fixed_pos[k];
        V p[NR], l[NR];
        long long toff = base;
#pragma unroll
        for (int j = 0; j < TB; ++j)
            if ((t >> j) & 1) toff |= 1ll << lm[j];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            long long off = toff;
#pragma unroll
            for (int k = 0; k < RB; ++k)
                if ((r >> k) & 1) off |= 1ll << lm[TB + k];
            p[r] = psi[off];
            l[r] = first ? mk<R>((R)0, (R)0) : lam[off];
        }
        if (first) {
            uint32_t pa = 0, pb = 0;
            for (int k = 0; k < nfixed; ++k)
                if ((tau >> k) & 1) { int g = d->fixed_pos[k]; pa ^= d->colA[g]; pb ^= d->colB[g]; }
#pragma unroll
            for (int j = 0; j < TB; ++j)
                if ((t >> j) & 1) { pa ^= d->colA[lm[j]]; pb ^= d->colB[lm[j]]; }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                uint32_t a = pa, b = pb;
#pragma unroll
                for (int k = 0; k < RB; ++k)
                    if ((r >> k) & 1) { a ^= d->colA[lm[TB + k]]; b ^= d->colB[lm[TB + k]]; }
                const R dv = dtab[__popc(a) * nB1 + __popc(b)];
                l[r].x = dv * p[r].x;
                l[r].y = dv * p[r].y;
            }
        }
        add_x(p, l, d->rot_mask[0], 0);
#pragma unroll
        for (int r = 0; r < NR; ++r) { tp[swz(t | (r << TB))] = p[r]; tl[swz(t | (r << TB))] = l[r]; }
        __syncthreads();
        if (d->rot_mask[1]) {
#pragma unroll
            for (int r = 0; r < NR; ++r) { p[r] = tp[swz(r | (t << RB))]; l[r] = tl[swz(r | (t << RB))]; }
            add_x(p, l, d->rot_mask[1], 1);
#pragma unroll
            for (int r = 0; r < NR; ++r) { tp[swz(r | (t << RB))] = p[r]; tl[swz(r | (t << RB))] = l[r]; }
            __syncthreads();
        }
        const int tlo = t & 15, thi = t >> 4;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int li = swz(tlo | (r << 4) | (thi << 8));
            p[r] = tp[li];
            l[r] = tl[li];
        }
        add_x(p, l, d->rot_mask[2], 2);
        long long toff2 = base;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if ((tlo >> j) & 1) toff2 |= 1ll << lm[j];
            if ((thi >> j) & 1) toff2 |= 1ll << lm[8 + j];
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            long long off = toff2;
#pragma unroll
            for (int k = 0; k < RB; ++k)
                if ((r >> k) & 1) off |= 1ll << lm[4 + k];
            lam[off] = l[r];
        }
        __syncthreads();
    }
}

// Read-only X measurement on the tiled passes: for every qubit of the pass, in the
// stage where it is a register bit, sum Re(conj(a) b) over its amplitude pairs, i.e.
// <X_q> / 2, accumulated per X class.  partials[(b * nblk + slot0 + blockIdx.x) * RED_NV + {0, 1}].
template <typename R>
__global__ void __launch_bounds__(NT) k_xmeasure(const typename C2<R>::T *__restrict__ psi, long long state_stride,
                                                 long long ntiles, const PassDesc *__restrict__ d,
                                                 double *__restrict__ partials, int nblk, int slot0) {
    using V = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *tp = reinterpret_cast<V *>(smem_raw);
    const int t = threadIdx.x;
    psi += (long long)blockIdx.y * state_stride;
    int lm[LT];
#pragma unroll
    for (int j = 0; j < LT; ++j) lm[j] = d->lmap[j];
    const unsigned rm0 = d->rot_mask[0], rm1 = d->rot_mask[1], rm2 = d->rot_mask[2];
    int cls[3][RB];
#pragma unroll
    for (int st = 0; st < 3; ++st)
#pragma unroll
        for (int k = 0; k < RB; ++k) cls[st][k] = d->reg_cls[st][k];
    const int nfixed = d->nfixed;
    double acc[2] = {0.0, 0.0};
    auto pairs = [&](const V (&v)[NR], unsigned mask, const int (&c)[RB], R &g0, R &g1) {
#pragma unroll
        for (int k = 0; k < RB; ++k) {
            if (!((mask >> k) & 1u)) continue;
            R g = 0;
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if (!((r >> k) & 1)) g += v[r].x * v[r | (1 << k)].x + v[r].y * v[r | (1 << k)].y;
            if (c[k]) g1 += g; else g0 += g;
        }
    };
    for (long long tau = blockIdx.x; tau < ntiles; tau += gridDim.x) {
        long long base = 0;
        for (int k = 0; k < nfixed; ++k)
            if ((tau >> k) & 1) base |= 1ll << d->fixed_pos[k];
        R g0 = 0, g1 = 0;
        V v[NR];
        long long toff = base;
#pragma unroll
        for (int j = 0; j < TB; ++j)
            if ((t >> j) & 1) toff |= 1ll << lm[j];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            long long off = toff;
#pragma unroll
            for (int k = 0; k < RB; ++k)
                if ((r >> k) & 1) off |= 1ll << lm[TB + k];
            v[r] = psi[off];
        }
        pairs(v, rm0, cls[0], g0, g1);
#pragma unroll
        for (int r = 0; r < NR; ++r) tp[swz(t | (r << TB))] = v[r];
        __syncthreads();
        if (rm1) {
#pragma unroll
            for (int r = 0; r < NR; ++r) v[r] = tp[swz(r | (t << RB))];
            pairs(v, rm1, cls[1], g0, g1);
        }
        const int tlo = t & 15, thi = t >> 4;
#pragma unroll
        for (int r = 0; r < NR; ++r) v[r] = tp[swz(tlo | (r << 4) | (thi << 8))];
        pairs(v, rm2, cls[2], g0, g1);
        acc[0] += (double)g0;
        acc[1] += (double)g1;
        __syncthreads();
    }
    block_store<2>(acc, partials + ((long long)blockIdx.y * nblk + slot0 + blockIdx.x) * RED_NV);
}

// lambda_b <- w_b * phi_b with w_b = (res[b * RED_NV], res[b * RED_NV + 1]) = <phi_b|psi_b>
template <typename R>
__global__ void k_scaled_copy(typename C2<R>::T *__restrict__ lam, const typename C2<R>::T *__restrict__ phi,
                              long long state_stride, const double *__restrict__ w) {
    lam += (long long)blockIdx.y * state_stride;
    phi += (long long)blockIdx.y * state_stride;
    const R wr = (R)w[RED_NV * blockIdx.y], wi = (R)w[RED_NV * blockIdx.y + 1];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < state_stride;
         i += (long long)gridDim.x * blockDim.x) {
        auto a = phi[i];
        typename C2<R>::T r;
        r.x = wr * a.x - wi * a.y;
        r.y = wr * a.y + wi * a.x;
        lam[i] = r;
    }
}

}  // namespace qsim
