/*
 * qs_oracle.c -- plain FP64 CPU reference primitives for the Trotterised
 * adiabatic evolution of the Z2 gauge-Higgs model.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the bench load this library.  It shares no code with the
 * CUDA path.
 *
 * Every routine is one plain loop over amplitudes, one Pauli term at a time, in
 * double precision.  State vectors are interleaved (re, im) doubles of length
 * 2 * 2^n; amplitude index i has bit q equal to 0 when qubit q is in the Z=+1
 * eigenstate.
 *
 * Factors follow Eq. (7)-(8) of Sec. III: every factor of the Trotter product
 * is exp(i*theta*P) for a Pauli string P whose summands commute, so
 *     exp(i theta P) = cos(theta) I + i sin(theta) P        (P^2 = I).
 * OpenMP splits the amplitude loops only; every amplitude is computed by the
 * same arithmetic whatever the thread count, and the reductions run serially.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef long long i64;

static inline int parity64(uint64_t x) { return __builtin_parityll(x); }

/* |+>^n : the ground state of H0 = -sum_q X_q. */
void or_init_plus(double *psi, int n) {
    i64 dim = 1LL << n;
    double a = 1.0 / sqrt((double)dim);
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < dim; ++i) { psi[2 * i] = a; psi[2 * i + 1] = 0.0; }
}

/* exp(i theta X_q), Eq. (8) first line (R_x(-2 theta) in the gate form, Eq. (9)). */
void or_apply_xrot(double *psi, int n, int q, double theta) {
    i64 dim = 1LL << n, bit = 1LL << q;
    double c = cos(theta), s = sin(theta);
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < dim; ++i) {
        if (i & bit) continue;
        i64 j = i | bit;
        double ar = psi[2 * i], ai = psi[2 * i + 1];
        double br = psi[2 * j], bi = psi[2 * j + 1];
        /* a' = c a + i s b ; b' = i s a + c b */
        psi[2 * i] = c * ar - s * bi;
        psi[2 * i + 1] = c * ai + s * br;
        psi[2 * j] = c * br - s * ai;
        psi[2 * j + 1] = c * bi + s * ar;
    }
}

/* exp(i theta X_m) for an X string on the qubits of mask m (the star A_v,
 * Eq. (8) second line, realised in the paper by Hadamards plus an ancilla). */
void or_apply_xstring(double *psi, int n, uint64_t mask, double theta) {
    i64 dim = 1LL << n;
    double c = cos(theta), s = sin(theta);
    if (mask == 0) return;
    int top = 63 - __builtin_clzll(mask);
    i64 tb = 1LL << top;
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < dim; ++i) {
        if (i & tb) continue;            /* visit each pair {i, i^m} once */
        i64 j = i ^ (i64)mask;
        double ar = psi[2 * i], ai = psi[2 * i + 1];
        double br = psi[2 * j], bi = psi[2 * j + 1];
        psi[2 * i] = c * ar - s * bi;
        psi[2 * i + 1] = c * ai + s * br;
        psi[2 * j] = c * br - s * ai;
        psi[2 * j + 1] = c * bi + s * ar;
    }
}

/* exp(i theta Z_m): amplitude i gets phase exp(i theta (-1)^{popcount(i & m)}).
 * Plaquette B_p, bond tau^z sigma^z tau^z, or sigma^z_l (Eq. (8), Eq. (9)). */
void or_apply_zphase(double *psi, int n, uint64_t mask, double theta) {
    i64 dim = 1LL << n;
    double c = cos(theta), s = sin(theta);
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < dim; ++i) {
        double sg = parity64((uint64_t)i & mask) ? -1.0 : 1.0;
        double ps = sg * s;
        double ar = psi[2 * i], ai = psi[2 * i + 1];
        psi[2 * i] = c * ar - ps * ai;
        psi[2 * i + 1] = c * ai + ps * ar;
    }
}

/* out += coef * X_m in   (X string: amplitude i takes in[i ^ m]). */
void or_axpy_xstring(double *out, const double *in, int n, uint64_t mask, double coef) {
    i64 dim = 1LL << n;
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < dim; ++i) {
        i64 j = i ^ (i64)mask;
        out[2 * i] += coef * in[2 * j];
        out[2 * i + 1] += coef * in[2 * j + 1];
    }
}

/* out += coef * Z_m in   (Z string: sign (-1)^{popcount(i & m)}). */
void or_axpy_zstring(double *out, const double *in, int n, uint64_t mask, double coef) {
    i64 dim = 1LL << n;
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < dim; ++i) {
        double sg = parity64((uint64_t)i & mask) ? -coef : coef;
        out[2 * i] += sg * in[2 * i];
        out[2 * i + 1] += sg * in[2 * i + 1];
    }
}

/* <a|b> = sum_i conj(a_i) b_i (serial, fixed order). */
void or_inner(const double *a, const double *b, int n, double *re, double *im) {
    i64 dim = 1LL << n;
    double sr = 0.0, si = 0.0;
    for (i64 i = 0; i < dim; ++i) {
        double ar = a[2 * i], ai = a[2 * i + 1], br = b[2 * i], bi = b[2 * i + 1];
        sr += ar * br + ai * bi;
        si += ar * bi - ai * br;
    }
    *re = sr; *im = si;
}

/* <psi|Z_m|psi> = sum_i |psi_i|^2 (-1)^{popcount(i & m)}. */
double or_expect_zstring(const double *psi, int n, uint64_t mask) {
    i64 dim = 1LL << n;
    double acc = 0.0;
    for (i64 i = 0; i < dim; ++i) {
        double p = psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
        acc += parity64((uint64_t)i & mask) ? -p : p;
    }
    return acc;
}

/* <psi|X_m|psi> = sum_i conj(psi_i) psi_{i^m} (real for Hermitian X_m). */
double or_expect_xstring(const double *psi, int n, uint64_t mask) {
    i64 dim = 1LL << n;
    double acc = 0.0;
    for (i64 i = 0; i < dim; ++i) {
        i64 j = i ^ (i64)mask;
        acc += psi[2 * i] * psi[2 * j] + psi[2 * i + 1] * psi[2 * j + 1];
    }
    return acc;
}

/*
 * Forward-mode tangents for the schedule gradient.  A factor F = exp(i theta P)
 * whose angle depends on a parameter a maps the pair (psi, dpsi = d psi/da) to
 *     psi'  = F psi,
 *     dpsi' = F dpsi + (d theta/d a) * i P psi'.
 * ntan tangents are stored back to back (ntan x 2^n complex); dtheta[k] is the
 * angle derivative for tangent k.  psi is updated once, after the tangents.
 */
void or_xrot_tangent(double *psi, double *dpsi, int ntan, const double *dtheta,
                     int n, int q, double theta) {
    i64 dim = 1LL << n, bit = 1LL << q;
    double c = cos(theta), s = sin(theta);
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < dim; ++i) {
        if (i & bit) continue;
        i64 j = i | bit;
        double ar = psi[2 * i], ai = psi[2 * i + 1];
        double br = psi[2 * j], bi = psi[2 * j + 1];
        double nar = c * ar - s * bi, nai = c * ai + s * br;
        double nbr = c * br - s * ai, nbi = c * bi + s * ar;
        for (int k = 0; k < ntan; ++k) {
            double *d = dpsi + (i64)k * 2 * dim;
            double dar = d[2 * i], dai = d[2 * i + 1], dbr = d[2 * j], dbi = d[2 * j + 1];
            double t = dtheta[k];
            /* F dpsi */
            double ur = c * dar - s * dbi, ui = c * dai + s * dbr;
            double vr = c * dbr - s * dai, vi = c * dbi + s * dar;
            /* + t * i * X psi' : component i gets i * psi'_j, component j gets i * psi'_i */
            d[2 * i] = ur - t * nbi;
            d[2 * i + 1] = ui + t * nbr;
            d[2 * j] = vr - t * nai;
            d[2 * j + 1] = vi + t * nar;
        }
        psi[2 * i] = nar; psi[2 * i + 1] = nai;
        psi[2 * j] = nbr; psi[2 * j + 1] = nbi;
    }
}

void or_xstring_tangent(double *psi, double *dpsi, int ntan, const double *dtheta,
                        int n, uint64_t mask, double theta) {
    i64 dim = 1LL << n;
    double c = cos(theta), s = sin(theta);
    if (mask == 0) return;
    int top = 63 - __builtin_clzll(mask);
    i64 tb = 1LL << top;
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < dim; ++i) {
        if (i & tb) continue;
        i64 j = i ^ (i64)mask;
        double ar = psi[2 * i], ai = psi[2 * i + 1];
        double br = psi[2 * j], bi = psi[2 * j + 1];
        double nar = c * ar - s * bi, nai = c * ai + s * br;
        double nbr = c * br - s * ai, nbi = c * bi + s * ar;
        for (int k = 0; k < ntan; ++k) {
            double *d = dpsi + (i64)k * 2 * dim;
            double dar = d[2 * i], dai = d[2 * i + 1], dbr = d[2 * j], dbi = d[2 * j + 1];
            double t = dtheta[k];
            double ur = c * dar - s * dbi, ui = c * dai + s * dbr;
            double vr = c * dbr - s * dai, vi = c * dbi + s * dar;
            d[2 * i] = ur - t * nbi;
            d[2 * i + 1] = ui + t * nbr;
            d[2 * j] = vr - t * nai;
            d[2 * j + 1] = vi + t * nar;
        }
        psi[2 * i] = nar; psi[2 * i + 1] = nai;
        psi[2 * j] = nbr; psi[2 * j + 1] = nbi;
    }
}

void or_zphase_tangent(double *psi, double *dpsi, int ntan, const double *dtheta,
                       int n, uint64_t mask, double theta) {
    i64 dim = 1LL << n;
    double c = cos(theta), s = sin(theta);
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < dim; ++i) {
        double z = parity64((uint64_t)i & mask) ? -1.0 : 1.0;
        double ps = z * s;
        double ar = psi[2 * i], ai = psi[2 * i + 1];
        double nar = c * ar - ps * ai, nai = c * ai + ps * ar;
        for (int k = 0; k < ntan; ++k) {
            double *d = dpsi + (i64)k * 2 * dim;
            double dr = d[2 * i], di = d[2 * i + 1];
            double t = dtheta[k] * z;
            /* e^{i theta z} dpsi + t * i * psi' */
            d[2 * i] = c * dr - ps * di - t * nai;
            d[2 * i + 1] = c * di + ps * dr + t * nar;
        }
        psi[2 * i] = nar; psi[2 * i + 1] = nai;
    }
}

int or_max_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int t) {
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
