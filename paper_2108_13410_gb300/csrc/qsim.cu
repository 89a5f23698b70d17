// qsim.cu -- C ABI (include/qsim.h) over the sm_103a kernels of kernels.cuh.
//
// Host side: lattice term tables, the X-pass plan, FP64 operator records
// (cos/sin of the X angles and the Z-layer phase table per Trotter factor), launch
// sequencing on the bound stream, and FP64 reductions read back to the host.
#include <cuda_runtime.h>

#include <cmath>
#include <functional>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "qsim.h"
#include "lattice.h"
#include "kernels.cuh"
#include "xpass_tma.cuh"
#include "xpass_wl.cuh"
#include "xpass_df.cuh"
#include "adjoint.cuh"
#include "adjoint_tma.cuh"
#include "adjoint_wl.cuh"
#include "scan.cuh"
#include "scan_mixed.cuh"

using namespace qsim;

namespace {

thread_local std::string g_create_error;
constexpr int RED_BLOCKS = 152 * 4;  // reduction grid per batch element (fixed: deterministic)
constexpr int RES_SLOTS = 160;       // reduction result slots per readback

// One Trotter factor group: exp(-i tau H_X) (angles per X class), then optionally
// exp(-i dt H_Z) (plaquette and second-class Z angles).
struct Op {
    double thx[2];   // X angle per class (sigma^x / tau^x or A_v)
    double zA, zB;   // Z angles: s*h*dt and s*lambda*dt
    bool has_z;
};

struct Coef { double xs, xt, za, zb; };

// Pass variants: butterfly kind x diagonal phase applied before the store.
enum { V_ROT = 0, V_ROT_Z = 1, V_HAD = 2, V_HAD_Z = 3, V_HAD_X = 4, NVAR = 5 };

inline Coef coefficients(const qs_couplings &c, double s) {
    // -H(s) = sum coef * term, H(s) = (1-s) H0 + s H1
    return Coef{(1.0 - s) + s * c.g, (1.0 - s) + s * c.J, s * c.h, s * c.lambda};
}

}  // namespace

namespace qsim {
// Message reported by qs_last_error(NULL): the last failed qs_create or handle-free call.
void set_handle_free_error(const std::string &msg) { g_create_error = msg; }
}

struct qs_sim {
    Lattice lat;
    int boundary = 0, form = 0, dtype = 0, batch = 1, n = 0;
    long long dim = 0;
    void *state[2] = {nullptr, nullptr};
    size_t state_cap[2] = {0, 0};
    cudaStream_t stream = nullptr;
    int method = 0, renorm_every = 0, profile = 0, use_graph = 0;
    std::string err;
    // tables
    int nA = 0, nB = 0, rec_stride = 0;
    int nXA = 0, nXB = 0, xlut_off = 0;    // Hadamard-basis X table (unitary gauge)
    int max_lut = 0;                       // largest phase table (entries)
    std::vector<int> plan_k;               // new qubits of each pass after the first (empty: 8 per pass)
    std::vector<int> pass_q;               // qubits fused by each pass of the current plan
    long long plan_code = 0;               // QS_OPT_PLAN value of plan_k (0: default)
    std::vector<PassDesc> passes;          // pass plan (Z columns, no phase)
    std::vector<PassDesc> pvar;            // [NVAR * pass + variant]
    PassDesc *d_passes = nullptr;          // device copy of pvar
    uint32_t *d_colA = nullptr, *d_colB = nullptr;
    // operator records
    double *d_rec = nullptr; size_t d_rec_cap = 0;
    double *h_rec = nullptr; size_t h_rec_cap = 0;
    cudaEvent_t rec_done = nullptr; bool rec_pending = false;
    // reductions
    double *d_partials = nullptr, *d_res = nullptr, *h_res = nullptr;
    // profiling of the fused pass
    std::vector<cudaEvent_t> ev_pool; size_t ev_used = 0;
    std::vector<int> ev_kind;              // per timed launch: 0 one factor group, 1 shared pass
    long long launches = 0;
    // persistent TMA X pass (complex64)
    int xpass_impl = 0;                    // 0 auto, 1 register kernel, 2 TMA kernel
    int nbuf = 3;                          // TMA shared-memory buffers per CTA (2 or 3)
    int adj_nbuf = 1;                      // tile-pair buffers of the TMA adjoint pass (1 or 2)
    int tma_store = 1;                     // X pass writes tiles back with TMA stores
    int xmerge = 1;                        // share the pass of one qubit group between factor groups
    int pdl = 1;                           // X passes launched with programmatic stream serialisation
    int nbuf_shared = 0;                   // TMA tile buffers of the shared passes (0 auto, 2 or 3)
    int shared_kernel = 1;                 // shared rotation passes: 1 warp-local slices where they
                                           // apply (k_xpass_wl), 0 the CTA-staged kernel
    int tan_off = 0;                       // tangent triple in the operator record
    int nX0 = 0, nX1 = 0;                  // X qubits per class
    bool tan_active = false;               // this call's X passes use the tangent form
    int adj_impl = 0;                      // adjoint reverse pass: 0 auto (TMA), 1 register kernel
    int adj_early = 1;                     // one buffer, tangent form: next load issued before the stores
    int sm_count = 0;
    std::vector<TmaPass> tpasses;          // [NVAR * pass + variant]
    std::vector<CUtensorMap> tmaps;        // one per pass, encoded for the bound state
    bool tmaps_ok = false;
    std::vector<CUtensorMap> tmaps_aux;    // the same over the adjoint work state (slot 1)
    // complex128 unitary-gauge passes in double-float arithmetic (xpass_df.cuh): tensor
    // maps of the high and low halves of the blocked layout, one pair per pass
    std::vector<CUtensorMap> tmaps_dfh, tmaps_dfl;
    bool tmaps_df_ok = false;
    int c128_df = 1;                       // QS_OPT_C128_DF
    bool df_active = false;                // the state is in the blocked layout (inside a call)
    bool tmaps_aux_ok = false;
    int *d_err = nullptr;                  // device flag: bounded wait gave up
    // adjoint workspaces
    double *d_adj_part = nullptr; size_t adj_part_cap = 0;
    double *d_grad = nullptr; size_t grad_cap = 0;
    double *h_grad = nullptr; size_t h_grad_cap = 0;
    double *d_hrec = nullptr; size_t hrec_cap = 0;
    // CUDA graph of the last qs_evolve launch sequence (QS_OPT_GRAPH)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    long long graph_key[10] = {0};
    long long graph_launches = 0;
    cudaGraphExec_t scan_graph = nullptr;
    long long scan_key[10] = {0};
    // operator-record inputs (couplings, schedule) on the device
    double *d_in = nullptr; size_t d_in_cap = 0;
    bool in_path = false; size_t in_ncpl = 0;
    // scan workspaces
    double *d_scan = nullptr; size_t scan_cap = 0;
    int *d_queue = nullptr;                // work-queue counter of the mixed scan
    int scan_buffers = 3;                  // tile buffers of the mixed scan's 17-qubit passes
    double *h_scan = nullptr; size_t h_scan_cap = 0;
};

#define FAIL(sim, code, ...)                                   \
    do {                                                       \
        char _b[512];                                          \
        snprintf(_b, sizeof(_b), __VA_ARGS__);                 \
        (sim)->err = _b;                                       \
        return (code);                                         \
    } while (0)

#define CK(sim, call)                                                                   \
    do {                                                                                \
        cudaError_t _e = (call);                                                        \
        if (_e != cudaSuccess)                                                          \
            FAIL(sim, QS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(_e));           \
    } while (0)

#define CKL(sim)                                                                         \
    do {                                                                                 \
        cudaError_t _e = cudaGetLastError();                                             \
        if (_e != cudaSuccess) FAIL(sim, QS_ERR_CUDA, "launch: %s", cudaGetErrorString(_e)); \
    } while (0)

namespace {

// ---------------------------------------------------------------------------
// pass plan: pass 0 covers global bits 0..11; each further pass keeps a chunk of
// c >= 4 low bits (>= 128 contiguous bytes) and takes up to 8 new high bits.
// ---------------------------------------------------------------------------
void build_passes(qs_sim *s) {
    const int n = s->n;
    s->passes.clear();
    s->pass_q.clear();
    if (n < LT) return;
    int next = 0;
    size_t pi = 0;   // index into plan_k
    while (next < n) {
        PassDesc d;
        memset(&d, 0, sizeof(d));
        d.n = n;
        int first = (next == 0);
        int k = first ? LT : (pi < s->plan_k.size() ? s->plan_k[pi] : std::min(8, n - next));
        if (!first) ++pi;
        s->pass_q.push_back(k);
        int c = LT - k;                 // chunk bits (already rotated)
        bool rot_local[LT];
        for (int j = 0; j < LT; ++j) {
            if (j < c) { d.lmap[j] = j; rot_local[j] = first; }
            else { d.lmap[j] = next + (j - c); rot_local[j] = true; }
        }
        if (first) for (int j = 0; j < LT; ++j) { d.lmap[j] = j; rot_local[j] = true; }
        // stage register bits: stage0 local 8+k, stage1 local k, stage2 local 4+k
        const int stage_base[3] = {8, 0, 4};
        for (int st = 0; st < 3; ++st) {
            unsigned m = 0;
            for (int kk = 0; kk < RB; ++kk) {
                int lj = stage_base[st] + kk;
                if (rot_local[lj]) m |= 1u << kk;
                d.reg_cls[st][kk] = s->lat.x_class[d.lmap[lj]];
            }
            d.rot_mask[st] = m;
        }
        d.stage1_on = d.rot_mask[1] != 0;
        // tile-index bits: every global bit not in lmap, increasing
        bool used[64] = {false};
        for (int j = 0; j < LT; ++j) used[d.lmap[j]] = true;
        int nf = 0;
        for (int q = 0; q < n; ++q) if (!used[q]) d.fixed_pos[nf++] = q;
        d.nfixed = nf;
        d.nA = s->nA; d.nB = s->nB;
        for (int q = 0; q < n; ++q) {
            uint32_t a = 0, b = 0;
            for (size_t p = 0; p < s->lat.plaquettes.size(); ++p)
                if ((s->lat.plaquettes[p] >> q) & 1) a |= 1u << p;
            for (size_t p = 0; p < s->lat.second.size(); ++p)
                if ((s->lat.second[p] >> q) & 1) b |= 1u << p;
            d.colA[q] = a; d.colB[q] = b;
        }
        s->passes.push_back(d);
        next = first ? LT : next + k;
    }
}

// Variants of every pass: rotation or Hadamard butterflies, and which diagonal
// table (none, Z layer, or the Hadamard-basis X layer of the unitary gauge) is
// applied before the store.
void build_variants(qs_sim *s) {
    s->pvar.clear();
    uint32_t xa[64] = {0}, xb[64] = {0};
    if (!s->lat.gauge_higgs)
        for (int q = 0; q < s->n; ++q) {
            for (size_t v = 0; v < s->lat.stars.size(); ++v)
                if ((s->lat.stars[v] >> q) & 1) xa[q] |= 1u << v;
            xb[q] = 1u << q;                 // every unitary-gauge qubit is a link
        }
    for (const PassDesc &d : s->passes)
        for (int v = 0; v < NVAR; ++v) {
            PassDesc e = d;
            e.hadamard = v >= V_HAD;
            e.apply_z = (v == V_ROT_Z || v == V_HAD_Z || v == V_HAD_X);
            e.lut_off = 4;
            e.scale = 1.0;
            if (v == V_HAD_X) {
                for (int q = 0; q < MAXQ; ++q) { e.colA[q] = q < 64 ? xa[q] : 0; e.colB[q] = q < 64 ? xb[q] : 0; }
                e.nA = s->nXA; e.nB = s->nXB;
                e.lut_off = s->xlut_off;
                e.scale = ldexp(1.0, -s->n);   // two unnormalised transforms give 2^n
            }
            s->pvar.push_back(e);
        }
}

// TMA pass descriptors derived from the pass variants (local bit j < c is global j;
// local bit j >= c is global next + j - c).
void build_tma_passes(qs_sim *s) {
    s->tpasses.clear();
    const int n = s->n;
    for (const PassDesc &d : s->pvar) {
        int c = 0;
        while (c < LT && d.lmap[c] == c) ++c;
        const bool first = (c == LT);
        const int next = first ? LT : d.lmap[c];
        const int k = LT - c;
        if (first) c = LT;
        auto g = [&](int local) -> int { return local < c ? local : next + (local - c); };
        TmaPass P;
        memset(&P, 0, sizeof(P));
        P.c = c; P.next = first ? LT : next; P.k = first ? 0 : k;
        P.mid_bits = P.next - P.c;
        P.total_tiles = (long long)s->batch << (n - LT);
        const int thr_local[8] = {0, 1, 2, 3, 8, 9, 10, 11};
        for (int j = 0; j < 8; ++j) {
            int q = g(thr_local[j]);
            P.toff_c[j] = 1ll << q;
            P.pa_thr[j] = d.colA[q]; P.pb_thr[j] = d.colB[q];
        }
        for (int r = 0; r < NR; ++r) {
            long long off = 0; uint32_t a = 0, b = 0;
            for (int kk = 0; kk < RB; ++kk)
                if ((r >> kk) & 1) { int q = g(4 + kk); off += 1ll << q; a ^= d.colA[q]; b ^= d.colB[q]; }
            P.roff_c[r] = off; P.pa_reg[r] = a; P.pb_reg[r] = b;
        }
        for (int j = 0; j < 8; ++j) {
            int q = g(j);
            P.paA_thr[j] = d.colA[q]; P.pbA_thr[j] = d.colB[q];
            P.toff_a[j] = 1ll << q;
        }
        for (int r = 0; r < NR; ++r) {
            long long off = 0;
            for (int kk = 0; kk < RB; ++kk)
                if ((r >> kk) & 1) off += 1ll << g(8 + kk);
            P.roff_a[r] = off;
        }
        for (int r = 0; r < NR; ++r) {
            uint32_t a = 0, b = 0;
            for (int kk = 0; kk < RB; ++kk)
                if ((r >> kk) & 1) { int q = g(8 + kk); a ^= d.colA[q]; b ^= d.colB[q]; }
            P.paA_reg[r] = a; P.pbA_reg[r] = b;
        }
        const int stage_base[3] = {8, 0, 4};
        for (int st = 0; st < 3; ++st) {
            unsigned cl = 0;
            for (int kk = 0; kk < RB; ++kk)
                if (s->lat.x_class[g(stage_base[st] + kk)]) cl |= 1u << kk;
            P.cls[st] = cl;
            P.rot[st] = d.rot_mask[st];
        }
        P.stage_b = P.rot[1] != 0;
        P.nA = d.nA; P.nB = d.nB;
        P.apply_z = d.apply_z;
        P.hadamard = d.hadamard;
        P.lut_off = d.lut_off;
        P.scale = (float)d.scale;
        P.tile_bits = n - LT;
        P.tan_off = s->tan_off;
        for (int i = 0; i < P.tile_bits && i < 32; ++i) {
            int q = i < P.mid_bits ? P.c + i : P.next + P.k + (i - P.mid_bits);
            P.pa_tile[i] = d.colA[q]; P.pb_tile[i] = d.colB[q];
        }
        s->tpasses.push_back(P);
    }
}

// Encode one 5-D tensor map per pass over the bound complex64 state:
//   dims (8-byte elements) {16, 2^(c-4), 2^(next-c), 2^k, 2^(n-next-k) * batch},
//   box {16, 2^(c-4), 1, 2^k, 1}, 128-byte swizzle.
qs_status encode_tmaps(qs_sim *s, int slot = 0) {
    std::vector<CUtensorMap> &maps = slot == 0 ? s->tmaps : s->tmaps_aux;
    bool &ok = slot == 0 ? s->tmaps_ok : s->tmaps_aux_ok;
    ok = false;
    maps.clear();
    if (slot == 0) { s->tmaps_df_ok = false; s->tmaps_dfh.clear(); s->tmaps_dfl.clear(); }
    if (s->passes.empty() || !s->state[slot]) return QS_OK;
    if (s->dtype != QS_C64 && !(s->dtype == QS_C128 && slot == 0)) return QS_OK;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            FAIL(s, QS_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const int n = s->n;
    if (s->dtype == QS_C128) {
        // blocked double-float layout: per 16 amplitudes, 16 high (re, im) float pairs then
        // 16 low ones; each half is a complex64-like tile with doubled strides
        for (size_t p = 0; p < s->passes.size(); ++p) {
            const TmaPass &P = s->tpasses[NVAR * p];
            cuuint64_t dims[5] = {16, 1ull << (P.c - 4), 1ull << (P.next - P.c), 1ull << P.k,
                                  (1ull << (n - P.next - P.k)) * (cuuint64_t)s->batch};
            cuuint64_t strides[4] = {16 * 16, (1ull << P.c) * 16, (1ull << P.next) * 16, (1ull << (P.next + P.k)) * 16};
            cuuint32_t box[5] = {16, (cuuint32_t)(1u << (P.c - 4)), 1, (cuuint32_t)(1u << P.k), 1};
            cuuint32_t es[5] = {1, 1, 1, 1, 1};
            for (int half = 0; half < 2; ++half) {
                CUtensorMap m;
                CUresult r = encode(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5,
                                    (char *)s->state[0] + 128 * half, dims, strides, box, es,
                                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS)
                    FAIL(s, QS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for double-float pass %zu", (int)r, p);
                (half ? s->tmaps_dfl : s->tmaps_dfh).push_back(m);
            }
        }
        s->tmaps_df_ok = true;
        return QS_OK;
    }
    for (size_t p = 0; p < s->passes.size(); ++p) {
        const TmaPass &P = s->tpasses[NVAR * p];
        cuuint64_t dims[5] = {16, 1ull << (P.c - 4), 1ull << (P.next - P.c), 1ull << P.k,
                              (1ull << (n - P.next - P.k)) * (cuuint64_t)s->batch};
        cuuint64_t strides[4] = {16 * 8, (1ull << P.c) * 8, (1ull << P.next) * 8, (1ull << (P.next + P.k)) * 8};
        cuuint32_t box[5] = {16, (cuuint32_t)(1u << (P.c - 4)), 1, (cuuint32_t)(1u << P.k), 1};
        cuuint32_t es[5] = {1, 1, 1, 1, 1};
        CUtensorMap m;
        CUresult r = encode(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, s->state[slot], dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) FAIL(s, QS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for pass %zu", (int)r, p);
        maps.push_back(m);
    }
    ok = true;
    return QS_OK;
}

// Rebuild the pass tables after a change of plan_k: host descriptors, their device copy,
// the tensor maps of the bound states; the cached evolve graph holds the old ones.
qs_status rebuild_plan(qs_sim *s) {
    if (s->stream) CK(s, cudaStreamSynchronize(s->stream));
    build_passes(s);
    build_variants(s);
    build_tma_passes(s);
    if (s->d_passes) { CK(s, cudaFree(s->d_passes)); s->d_passes = nullptr; }
    if (!s->pvar.empty()) {
        CK(s, cudaMalloc((void **)&s->d_passes, s->pvar.size() * sizeof(PassDesc)));
        CK(s, cudaMemcpy(s->d_passes, s->pvar.data(), s->pvar.size() * sizeof(PassDesc), cudaMemcpyHostToDevice));
    }
    if (s->graph_exec) { cudaGraphExecDestroy(s->graph_exec); s->graph_exec = nullptr; }
    qs_status st;
    if (s->state[0] && (st = encode_tmaps(s, 0)) != QS_OK) return st;
    if (s->state[1] && (st = encode_tmaps(s, 1)) != QS_OK) return st;
    return QS_OK;
}

size_t tma_smem_bytes(const qs_sim *s, int nbuf, bool z) {
    size_t b = (size_t)nbuf * TMA_TILE_BYTES + 1024;
    if (z) b += (size_t)s->max_lut * 8 + 3 * 256 * 8;
    return b;
}

// Rotation / phase coefficients for exp(i t P) = (1 - u) + i s P, u = 1 - cos t =
// 2 sin^2(t/2), s = sin t, computed in FP64.  Keeping u instead of cos t keeps its
// full relative precision for the small angles of a Trotter step, so the rounded
// pair satisfies (1-u)^2 + s^2 = 1 to ~1e-10 instead of ~1e-7 (plain rounding of
// cos t near 1).  For complex64 the float pair is then chosen, within +-3 ulps of
// each component, to minimise |(1-u)^2 + s^2 - 1| evaluated in double; this keeps
// rotations and phases from scaling the norm systematically step after step.
void unit_pair(bool f32, double t, double *ou, double *os) {
    double sh = sin(0.5 * t);
    double u = 2.0 * sh * sh, s = sin(t);
    if (!f32) { *ou = u; *os = s; return; }
    auto err = [](float a, float b) {
        double c = 1.0 - (double)a;
        return fabs(c * c + (double)b * (double)b - 1.0);
    };
    float u0 = (float)u, s0 = (float)s;
    float bu = u0, bs = s0;
    double be = err(u0, s0);
    double bd = 0.0;
    float uu = u0;
    for (int i = 0; i < 3; ++i) uu = nextafterf(uu, -4.0f);
    for (int i = -3; i <= 3; ++i, uu = nextafterf(uu, 4.0f)) {
        float ss = s0;
        for (int j = 0; j < 3; ++j) ss = nextafterf(ss, -4.0f);
        for (int j = -3; j <= 3; ++j, ss = nextafterf(ss, 4.0f)) {
            double e = err(uu, ss);
            double dd = fabs((double)uu - u) + fabs((double)ss - s);
            if (e < be || (e == be && dd < bd)) { be = e; bd = dd; bu = uu; bs = ss; }
        }
    }
    *ou = bu; *os = bs;
}

// ops[k * batch + b].  path: step k uses H1 with couplings c[k * batch + b] (s = 1);
// otherwise H(s_k) with couplings c[b].  Only has_z and the angles of the per-gate form
// are used on the host; the fused path builds its records on the device.
std::vector<Op> build_ops(const qs_couplings *c, int batch, const double *sv, double dt,
                          int n_steps, int order, bool fsal, bool path = false) {
    std::vector<Op> ops;
    auto cpl = [&](int k, int b) -> const qs_couplings & { return path ? c[(size_t)k * batch + b] : c[b]; };
    auto sk = [&](int k) -> double { return path ? 1.0 : sv[k]; };
    auto xang = [&](int k, int b, double tau, double *out) {
        Coef q = coefficients(cpl(k, b), sk(k));
        out[0] += q.xs * tau; out[1] += q.xt * tau;
    };
    auto zang = [&](int k, int b, Op &o) {
        Coef q = coefficients(cpl(k, b), sk(k));
        o.zA = q.za * dt; o.zB = q.zb * dt; o.has_z = true;
    };
    for (int k = 0; k < n_steps; ++k) {
        if (order == 1) {
            for (int b = 0; b < batch; ++b) {
                Op o{}; xang(k, b, dt, o.thx); zang(k, b, o);
                ops.push_back(o);
            }
        } else if (fsal) {
            for (int b = 0; b < batch; ++b) {
                Op o{};
                xang(k, b, 0.5 * dt, o.thx);
                if (k > 0) xang(k - 1, b, 0.5 * dt, o.thx);
                zang(k, b, o);
                ops.push_back(o);
            }
            if (k == n_steps - 1)
                for (int b = 0; b < batch; ++b) {
                    Op o{}; xang(k, b, 0.5 * dt, o.thx);
                    ops.push_back(o);
                }
        } else {
            for (int b = 0; b < batch; ++b) {
                Op o{}; xang(k, b, 0.5 * dt, o.thx); zang(k, b, o);
                ops.push_back(o);
            }
            for (int b = 0; b < batch; ++b) {
                Op o{}; xang(k, b, 0.5 * dt, o.thx);
                ops.push_back(o);
            }
        }
    }
    return ops;
}

template <typename R>
using V = typename C2<R>::T;

typedef void (*XpassTmaKernel)(float2 *, const double *, const double *, int, int, int *, const CUtensorMap,
                               const TmaPass);

template <int NBUF, bool TAN>
XpassTmaKernel xpass_tma_kernel_nb(bool store_tma, bool merged) {
    if (merged) return store_tma ? k_xpass_tma<NBUF, true, true, TAN> : k_xpass_tma<NBUF, false, true, TAN>;
    return store_tma ? k_xpass_tma<NBUF, true, false, TAN> : k_xpass_tma<NBUF, false, false, TAN>;
}

// k_xpass_tma instantiation for (buffers, store mode, shared pass, tangent form)
XpassTmaKernel xpass_tma_kernel(int nbuf, bool store_tma, bool merged, bool tan) {
    if (tan) return nbuf == 3 ? xpass_tma_kernel_nb<3, true>(store_tma, merged)
                              : xpass_tma_kernel_nb<2, true>(store_tma, merged);
    return nbuf == 3 ? xpass_tma_kernel_nb<3, false>(store_tma, merged) : xpass_tma_kernel_nb<2, false>(store_tma, merged);
}

typedef void (*AdjKernel)(float2 *, float2 *, const double *, int, int, int *, double *, int, int, int,
                          const double *, double *, int, const CUtensorMap, const CUtensorMap, const TmaPass);

// k_adj_tma instantiation for (tile buffers, tangent form, shared reverse pass); shared
// reverse passes exist in the tangent form only
AdjKernel adj_tma_kernel(int nbuf, bool tan, bool merged = false, bool early = false) {
    if (nbuf == 1) {
        if (early && tan) return merged ? k_adj_tma<1, true, true, true> : k_adj_tma<1, true, false, true>;
        return tan ? (merged ? k_adj_tma<1, true, true, false> : k_adj_tma<1, true, false, false>)
                   : k_adj_tma<1, false, false, false>;
    }
    return tan ? (merged ? k_adj_tma<2, true, true, false> : k_adj_tma<2, true, false, false>)
               : k_adj_tma<2, false, false, false>;
}


// One complex128 Walsh-Hadamard pass in double-float arithmetic over the blocked layout
// (variants V_HAD, V_HAD_X, V_HAD_Z; merged: a second round of butterflies).
size_t df_smem_bytes(const qs_sim *s) {
    return 2 * (size_t)TMA_TILE_BYTES + 1024 + (size_t)s->max_lut * 32 + 3 * 256 * 8;
}

qs_status launch_xpass_df(qs_sim *s, int p, int variant, const double *rec, const double *rec2, int frame,
                          int xscale) {
    TmaPass P = s->tpasses[NVAR * p + variant];
    const bool merged = rec2 != nullptr;
    const bool rot = !P.hadamard;
    P.frame = rot ? frame : 0;
    P.xscale = rot ? xscale : 0;
    if (rot && !(s->tan_active && (frame & 1)))
        FAIL(s, QS_ERR_STATE, "double-float rotation passes run the tangent form only");
    const size_t sm = df_smem_bytes(s);
    auto kern = rot ? (merged ? k_xpass_df<true, true> : k_xpass_df<false, true>)
                    : (merged ? k_xpass_df<true, false> : k_xpass_df<false, false>);
    cudaEvent_t e1 = nullptr;
    if (s->profile) {   // per-launch CUDA events, as for the complex64 passes
        while (s->ev_pool.size() < s->ev_used + 2) {
            cudaEvent_t e;
            CK(s, cudaEventCreate(&e));
            s->ev_pool.push_back(e);
        }
        cudaEvent_t e0 = s->ev_pool[s->ev_used];
        e1 = s->ev_pool[s->ev_used + 1];
        s->ev_used += 2;
        s->ev_kind.resize(s->ev_used / 2);
        s->ev_kind.back() = merged ? 1 : 0;
        CK(s, cudaEventRecord(e0, s->stream));
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, sm);
    if (per_sm < 1) per_sm = 1;
    const long long g = std::min<long long>(P.total_tiles, (long long)per_sm * s->sm_count);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = s->pdl ? 1 : 0;
    CK(s, cudaLaunchKernelEx(&cfg, kern, (float2 *)s->state[0], rec, merged ? rec2 : rec, s->rec_stride, s->n - LT,
                             s->d_err, s->tmaps_dfh[p], s->tmaps_dfl[p], P));
    CKL(s);
    s->launches++;
    if (s->profile) CK(s, cudaEventRecord(e1, s->stream));
    return QS_OK;
}

// In-place conversion of the bound complex128 state to (to_df) or from the blocked
// double-float layout.
qs_status df_convert(qs_sim *s, bool to_df) {
    const long long amps = (long long)s->batch << s->n;
    const unsigned grid = (unsigned)std::min<long long>((amps / 128 + 7) / 8, (long long)s->sm_count * 8);
    if (to_df) k_df_split<<<grid, 256, 0, s->stream>>>((double2 *)s->state[0], amps);
    else k_df_join<<<grid, 256, 0, s->stream>>>((double2 *)s->state[0], amps);
    CKL(s);
    s->launches++;
    s->df_active = to_df;
    return QS_OK;
}

// One X pass.  rec2 != nullptr selects the merged TMA pass: X of the pass's qubits from
// rec, the Z layer of rec, then X of the same qubits from rec2 (the next factor group).
template <typename R>
qs_status launch_xpass(qs_sim *s, int p, int variant, const double *rec, int frame = 0,
                       const double *rec2 = nullptr, int xscale = 0) {
    if (sizeof(R) == 8 && s->df_active) return launch_xpass_df(s, p, variant, rec, rec2, frame, xscale);
    const PassDesc &d = s->pvar[NVAR * p + variant];
    const bool apply_z = d.apply_z != 0;
    dim3 grid((unsigned)(1ll << d.nfixed), (unsigned)s->batch);
    size_t smem = (size_t)(1 << LT) * sizeof(V<R>) + (size_t)s->max_lut * sizeof(V<R>);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (s->profile) {
        while (s->ev_pool.size() < s->ev_used + 2) {
            cudaEvent_t e;
            CK(s, cudaEventCreate(&e));
            s->ev_pool.push_back(e);
        }
        e0 = s->ev_pool[s->ev_used]; e1 = s->ev_pool[s->ev_used + 1];
        s->ev_used += 2;
        s->ev_kind.resize(s->ev_used / 2);
        s->ev_kind.back() = rec2 ? 1 : 0;
        CK(s, cudaEventRecord(e0, s->stream));
    }
    const bool tma = sizeof(R) == 4 && s->tmaps_ok && s->xpass_impl != 1;
    if (tma) {
        TmaPass P = s->tpasses[NVAR * p + variant];
        P.frame = frame;
        const bool tan = s->tan_active && (frame & 1);
        if (rec2 && (frame & 1) && !tan) FAIL(s, QS_ERR_STATE, "shared rotation pass needs the tangent form");
        P.xscale = tan ? xscale : 0;
        // shared passes: 0 = by form (tangent rotations fit three CTAs per SM with two
        // buffers; the Walsh-Hadamard ones measured faster with three buffers)
        const int nb = rec2 ? (s->nbuf_shared ? s->nbuf_shared : (tan ? 2 : 3)) : s->nbuf;
        size_t sm = tma_smem_bytes(s, nb, apply_z);
        XpassTmaKernel kern = xpass_tma_kernel(nb, s->tma_store != 0, rec2 != nullptr, tan);
        // warp-local slices: a shared rotation pass with its Z layer whose rotated qubits
        // all sit on local bits 4..11 (no stage-B rotation), one state, bulk stores
        int nthreads = NT;
        const bool wl_form = (tan && !P.hadamard) || (P.hadamard && !(frame & 1));
        if (rec2 && wl_form && s->shared_kernel == 1 && apply_z && P.rot[1] == 0 && !P.stage_b &&
            s->batch == 1 && s->tma_store && P.total_tiles < (1ll << 30)) {
            // geometry by QS_OPT_SHARED_BUFFERS: 0 one CTA of 24 warps per SM with six
            // buffers, 2 three CTAs of 8 warps with two, 3 two CTAs of 8 warps with three
            const int g = s->nbuf_shared;
            if (P.hadamard)
                kern = g == 2 ? k_xpass_wl<2, 8, 3, true> : g == 3 ? k_xpass_wl<3, 8, 2, true>
                                                                 : k_xpass_wl<6, 24, 1, true>;
            else
                kern = g == 2 ? k_xpass_wl<2, 8, 3, false> : g == 3 ? k_xpass_wl<3, 8, 2, false>
                                                                  : k_xpass_wl<6, 24, 1, false>;
            nthreads = g == 2 || g == 3 ? 256 : 768;
            sm = tma_smem_bytes(s, g == 2 || g == 3 ? g : 6, true);
        }
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nthreads, sm);
        if (per_sm < 1) per_sm = 1;
        long long g = std::min<long long>(P.total_tiles, (long long)per_sm * s->sm_count);
        // programmatic dependent launch: the pass may be scheduled while the previous
        // kernel drains; it waits (griddepcontrol.wait) before reading global memory
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)g);
        cfg.blockDim = dim3(nthreads);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = s->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = s->pdl ? 1 : 0;
        CK(s, cudaLaunchKernelEx(&cfg, kern, (float2 *)s->state[0], rec, rec2 ? rec2 : rec, s->rec_stride,
                                 s->n - LT, s->d_err, s->tmaps[p], P));
    } else {
        if (rec2) FAIL(s, QS_ERR_STATE, "merged X pass needs the TMA kernel");
        k_xpass<R><<<grid, NT, smem, s->stream>>>((V<R> *)s->state[0], s->dim, rec, s->rec_stride,
                                                   s->d_passes + NVAR * p + variant);
    }
    CKL(s);
    s->launches++;
    if (s->profile) CK(s, cudaEventRecord(e1, s->stream));
    return QS_OK;
}

unsigned grid_for(long long work, int threads) {
    long long g = (work + threads - 1) / threads;
    return (unsigned)(g < 1 ? 1 : g);
}

template <typename R>
qs_status launch_zdiag(qs_sim *s, const double *rec) {
    dim3 grid(152 * 8, (unsigned)s->batch);
    size_t smem = (size_t)(s->nA + 1) * (s->nB + 1) * sizeof(V<R>);
    k_zdiag<R><<<grid, 256, smem, s->stream>>>((V<R> *)s->state[0], s->n, s->dim, rec, s->rec_stride,
                                                s->d_colA, s->d_colB, s->nA, s->nB);
    CKL(s);
    s->launches++;
    return QS_OK;
}

// Apply one factor group (records already on the device at drec); k / nops place
// it in the current qs_evolve call (the TMA kernel keeps the state in the real-
// rotation frame between the first and the last pass of the call).
template <typename R>
qs_status run_op_fused(qs_sim *s, const Op *ops_b, const double *drec, size_t k = 0, size_t nops = 1) {
    qs_status st;
    const bool ug = !s->lat.gauge_higgs;
    const int np = (int)s->passes.size();
    const bool has_z = ops_b[0].has_z;
    if (np == 0) {
        // state smaller than one tile: per-term X factors, then the Z table in one pass
        for (int b = 0; b < s->batch; ++b) {
            V<R> *psi = (V<R> *)s->state[0] + (long long)b * s->dim;
            for (int q = 0; q < s->n; ++q) {
                double c, sn;   // (u, s)
                unit_pair(sizeof(R) == 4, ops_b[b].thx[s->lat.x_class[q]], &c, &sn);
                k_rx<R><<<grid_for(s->dim / 2, 256), 256, 0, s->stream>>>(psi, s->n, s->dim, q,
                                                                            (R)c, (R)sn);
                CKL(s); s->launches++;
            }
        }
    } else if (!ug) {
        // (complex128 with double-float passes: the same frame and C handling)
        const bool tma = (sizeof(R) == 4 && s->tmaps_ok && s->xpass_impl != 1) || (sizeof(R) == 8 && s->df_active);
        for (int p = 0; p < np; ++p) {
            bool z_here = has_z && p == np - 1;
            int frame = 0;
            if (tma) frame = 1 | ((k == 0 && p == 0) ? 2 : 0) | ((k + 1 == nops && p == np - 1) ? 4 : 0);
            const int xs = (!has_z && p == np - 1) ? 1 : 0;   // tangent form: C of a group without Z
            if ((st = launch_xpass<R>(s, p, z_here ? V_ROT_Z : V_ROT, drec, frame, nullptr, xs)) != QS_OK)
                return st;
        }
        return QS_OK;
    } else {
        // unitary gauge: the X layer (sigma^x and A_v) is diagonal in the Hadamard
        // basis: WHT, Hadamard-basis phase, WHT back (with the Z layer before the store)
        for (int p = 0; p < np; ++p)
            if ((st = launch_xpass<R>(s, p, p == np - 1 ? V_HAD_X : V_HAD, drec)) != QS_OK) return st;
        for (int p = 0; p < np; ++p) {
            bool z_here = has_z && p == np - 1;
            if ((st = launch_xpass<R>(s, p, z_here ? V_HAD_Z : V_HAD, drec)) != QS_OK) return st;
        }
        return QS_OK;
    }
    if (ug) {
        for (int b = 0; b < s->batch; ++b) {
            V<R> *psi = (V<R> *)s->state[0] + (long long)b * s->dim;
            double c, sn;
            unit_pair(sizeof(R) == 4, ops_b[b].thx[1], &c, &sn);
            for (uint64_t m : s->lat.stars) {
                int top = 63 - __builtin_clzll(m);
                k_xstring<R><<<grid_for(s->dim / 2, 256), 256, 0, s->stream>>>(
                    psi, s->n, s->dim, (unsigned long long)m, top, (R)c, (R)sn);
                CKL(s); s->launches++;
            }
        }
    }
    if (has_z && (ug || np == 0))
        if ((st = launch_zdiag<R>(s, drec)) != QS_OK) return st;
    return QS_OK;
}

// Plain per-gate form: one launch per Pauli factor.
template <typename R>
qs_status run_op_pergate(qs_sim *s, const Op *ops_b) {
    for (int b = 0; b < s->batch; ++b) {
        const Op &o = ops_b[b];
        V<R> *psi = (V<R> *)s->state[0] + (long long)b * s->dim;
        const bool f32 = sizeof(R) == 4;
        double cx[2], sx[2], ca, sa, cb, sb;
        unit_pair(f32, o.thx[0], &cx[0], &sx[0]);
        unit_pair(f32, o.thx[1], &cx[1], &sx[1]);
        unit_pair(f32, o.zA, &ca, &sa);
        unit_pair(f32, o.zB, &cb, &sb);
        for (int q = 0; q < s->n; ++q) {
            int k = s->lat.x_class[q];
            k_rx<R><<<grid_for(s->dim / 2, 256), 256, 0, s->stream>>>(psi, s->n, s->dim, q,
                                                                        (R)cx[k], (R)sx[k]);
            CKL(s); s->launches++;
        }
        if (!s->lat.gauge_higgs) {
            for (uint64_t m : s->lat.stars) {
                int top = 63 - __builtin_clzll(m);
                k_xstring<R><<<grid_for(s->dim / 2, 256), 256, 0, s->stream>>>(
                    psi, s->n, s->dim, (unsigned long long)m, top, (R)cx[1], (R)sx[1]);
                CKL(s); s->launches++;
            }
        }
        if (o.has_z) {
            for (uint64_t m : s->lat.plaquettes) {
                k_zterm<R><<<grid_for(s->dim, 256), 256, 0, s->stream>>>(
                    psi, s->n, s->dim, (unsigned long long)m, (R)ca, (R)sa);
                CKL(s); s->launches++;
            }
            for (uint64_t m : s->lat.second) {
                k_zterm<R><<<grid_for(s->dim, 256), 256, 0, s->stream>>>(
                    psi, s->n, s->dim, (unsigned long long)m, (R)cb, (R)sb);
                CKL(s); s->launches++;
            }
        }
    }
    return QS_OK;
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
template <typename R>
qs_status reduce_diag(qs_sim *s, const void *state, uint64_t zmask, int slot) {
    dim3 grid(RED_BLOCKS, (unsigned)s->batch);
    k_reduce_diag<R><<<grid, RED_THREADS, 0, s->stream>>>((const V<R> *)state, s->n, s->dim, s->d_colA,
                                                          s->d_colB, s->nA, s->nB,
                                                          (unsigned long long)zmask, s->d_partials);
    CKL(s); s->launches++;
    k_finish<<<s->batch, RED_THREADS, 0, s->stream>>>(s->d_partials, RED_BLOCKS, 4,
                                                      s->d_res + (size_t)slot * s->batch * RED_NV);
    CKL(s); s->launches++;
    return QS_OK;
}

template <typename R>
qs_status reduce_xmask(qs_sim *s, const void *a, const void *b, uint64_t mask, int slot) {
    dim3 grid(RED_BLOCKS, (unsigned)s->batch);
    k_reduce_xmask<R><<<grid, RED_THREADS, 0, s->stream>>>((const V<R> *)a, (const V<R> *)b, s->n, s->dim,
                                                           (unsigned long long)mask, s->d_partials);
    CKL(s); s->launches++;
    k_finish<<<s->batch, RED_THREADS, 0, s->stream>>>(s->d_partials, RED_BLOCKS, 2,
                                                      s->d_res + (size_t)slot * s->batch * RED_NV);
    CKL(s); s->launches++;
    return QS_OK;
}

qs_status check_device_flag(qs_sim *s) {
    int flag = 0;
    CK(s, cudaMemcpy(&flag, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        cudaMemset(s->d_err, 0, sizeof(int));
        FAIL(s, QS_ERR_TIMEOUT, "a bounded device wait gave up (flag %d)", flag);
    }
    return QS_OK;
}

qs_status read_results(qs_sim *s, int slots) {
    size_t bytes = (size_t)slots * s->batch * RED_NV * sizeof(double);
    CK(s, cudaMemcpyAsync(s->h_res, s->d_res, bytes, cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    qs_status st = check_device_flag(s);
    if (st != QS_OK) return st;
    for (size_t i = 0; i < (size_t)slots * s->batch * RED_NV; ++i)
        if (!std::isfinite(s->h_res[i])) FAIL(s, QS_ERR_NONFINITE, "non-finite reduction result");
    return QS_OK;
}

inline double res(const qs_sim *s, int slot, int b, int v) {
    return s->h_res[((size_t)slot * s->batch + b) * RED_NV + v];
}

template <typename R>
qs_status renormalise(qs_sim *s) {
    qs_status st;
    if (sizeof(R) == 8 && s->df_active) {   // blocked double-float layout: join, rescale, split
        if ((st = df_convert(s, false)) != QS_OK) return st;
        if ((st = renormalise<R>(s)) != QS_OK) return st;
        return df_convert(s, true);
    }
    if ((st = reduce_diag<R>(s, s->state[0], 0, 0)) != QS_OK) return st;
    dim3 grid(152 * 8, (unsigned)s->batch);
    k_scale_by_norm<R><<<grid, 256, 0, s->stream>>>((V<R> *)s->state[0], s->dim, s->d_res);
    CKL(s); s->launches++;
    return QS_OK;
}

template <typename T>
qs_status grow(qs_sim *s, T **p, size_t *cap, size_t need, bool host) {
    if (need <= *cap) return QS_OK;
    if (*p) {
        if (host) cudaFreeHost(*p);
        else { CK(s, cudaStreamSynchronize(s->stream)); cudaFree(*p); }
    }
    *p = nullptr; *cap = 0;
    cudaError_t e = host ? cudaMallocHost((void **)p, need * sizeof(T)) : cudaMalloc((void **)p, need * sizeof(T));
    if (e != cudaSuccess) FAIL(s, QS_ERR_OOM, "workspace of %zu elements", need);
    *cap = need;
    return QS_OK;
}

// Operator records for the fused path are built on the device by k_build_records
// from the couplings and the schedule: upload_inputs copies those (the only
// host->device bytes of a call) and build_records fills the records of ops
// [op0, op0 + n) into d_rec.
constexpr size_t REC_CHUNK = 2048;   // ops whose records are resident at once

qs_status upload_inputs(qs_sim *s, const qs_couplings *c, const double *sv, int n_steps, bool path) {
    const int B = s->batch;
    const size_t ncpl = (size_t)B * (path ? n_steps : 1);
    const size_t in_doubles = ncpl * 4 + (path ? 0 : (size_t)n_steps);
    if (s->rec_pending) {
        CK(s, cudaEventSynchronize(s->rec_done));
        s->rec_pending = false;
    }
    if (in_doubles > s->h_rec_cap) {
        if (s->h_rec) cudaFreeHost(s->h_rec);
        s->h_rec = nullptr;
        s->h_rec_cap = 0;
        if (cudaMallocHost((void **)&s->h_rec, in_doubles * sizeof(double)) != cudaSuccess)
            FAIL(s, QS_ERR_OOM, "pinned schedule buffer (%zu doubles)", in_doubles);
        s->h_rec_cap = in_doubles;
    }
    qs_status st;
    if ((st = grow(s, &s->d_in, &s->d_in_cap, in_doubles, false)) != QS_OK) return st;
    for (size_t i = 0; i < ncpl; ++i) {
        s->h_rec[4 * i + 0] = c[i].J; s->h_rec[4 * i + 1] = c[i].h;
        s->h_rec[4 * i + 2] = c[i].g; s->h_rec[4 * i + 3] = c[i].lambda;
    }
    if (!path) memcpy(s->h_rec + 4 * ncpl, sv, (size_t)n_steps * sizeof(double));
    CK(s, cudaMemcpyAsync(s->d_in, s->h_rec, in_doubles * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    CK(s, cudaEventRecord(s->rec_done, s->stream));
    s->rec_pending = true;
    s->in_path = path;
    s->in_ncpl = ncpl;
    return QS_OK;
}

qs_status build_records(qs_sim *s, size_t op0, size_t n, double dt, int n_steps, int order) {
    const int B = s->batch;
    qs_status st;
    if ((st = grow(s, &s->d_rec, &s->d_rec_cap, n * B * (size_t)s->rec_stride, false)) != QS_OK) return st;
    RecGeom G;
    G.n_steps = n_steps; G.order = order; G.fsal = (order == 2); G.path = s->in_path ? 1 : 0;
    G.batch = B; G.rec_stride = s->rec_stride;
    G.nA = s->nA; G.nB = s->nB; G.nXA = s->nXA; G.nXB = s->nXB;
    G.xlut_off = s->lat.gauge_higgs ? 0 : s->xlut_off;
    G.f32 = s->dtype == QS_C64;
    // tangent records only where the tangent form can run (gauge-Higgs; complex128 with
    // double-float passes)
    G.tan_off = (s->lat.gauge_higgs && (s->dtype == QS_C64 || s->tan_active)) ? s->tan_off : 0;
    G.nX0 = s->nX0; G.nX1 = s->nX1;
    G.dt = dt;
    long long entries = (long long)n * B * (1 + (G.tan_off ? 2 : 1) * (s->nA + 1) * (s->nB + 1) +
                                            (G.xlut_off ? (s->nXA + 1) * (s->nXB + 1) : 0));
    unsigned blocks = (unsigned)std::min<long long>((entries + 255) / 256, 152 * 16);
    k_build_records<<<blocks, 256, 0, s->stream>>>(G, reinterpret_cast<const DevCouplings *>(s->d_in),
                                                   s->d_in + 4 * s->in_ncpl, (int)op0, (int)n, s->d_rec);
    CKL(s);
    s->launches++;
    return QS_OK;
}

// The merged schedule applies to the complex64 gauge-Higgs form on the TMA kernel with
// at least two qubit groups (passes).
template <typename R>
bool merged_schedule(const qs_sim *s) {
    if (sizeof(R) == 8)
        return s->df_active && s->xmerge && s->lat.gauge_higgs && s->passes.size() >= 2 && s->tan_active;
    return sizeof(R) == 4 && s->method == 0 && s->xmerge && s->lat.gauge_higgs && s->tmaps_ok &&
           s->xpass_impl != 1 && s->passes.size() >= 2 && s->tan_active;
}

// Factor groups [j0, j1) (records resident from op j0) with shared passes: the last
// pass of factor group k applies its Z layer and then the next group's X factors on
// the same qubits, and group k+1 skips that pass.  The shared passes alternate between
// the two cheapest qubit groups ga = np-2 and gb = np-1 (two register stages each;
// pass 0 rotates twelve qubits in three stages and always runs alone):
//   dir 0: ga, 0 .. np-3, gb        dir 1: gb, 0 .. np-3, ga
// With np passes per X layer a Trotter step costs np - 1 passes instead of np.  Only
// groups with a Z layer end in a shared pass; at the end of the resident records the
// chain restarts.
template <typename R>
qs_status launch_ops_merged(qs_sim *s, const std::vector<Op> &ops, int steps_per_renorm_unit, size_t j0,
                            size_t j1) {
    qs_status st;
    const int B = s->batch;
    const size_t nops = ops.size() / B;
    const int np = (int)s->passes.size();
    const size_t rs = (size_t)B * s->rec_stride;
    bool carried = false;   // the first qubit group of op k was applied by op k-1's last pass
    int dir = 0;            // which of the two orders below
    int ord[2][64];
    for (int i = 0; i < np; ++i) {
        const int mid = i - 1;   // middle groups 0 .. np-3
        ord[0][i] = i == 0 ? np - 2 : (i == np - 1 ? np - 1 : mid);
        ord[1][i] = i == 0 ? np - 1 : (i == np - 1 ? np - 2 : mid);
    }
    for (size_t k = j0; k < j1; ++k) {
        const double *rec = s->d_rec + (k - j0) * rs;
        const bool has_z = ops[k * B].has_z;
        const int i0 = carried ? 1 : 0;
        carried = false;
        for (int i = i0; i < np; ++i) {
            const int p = ord[dir][i];
            const bool last = i == np - 1;
            const int frame = 1 | ((k == 0 && i == 0) ? 2 : 0) | ((k + 1 == nops && last) ? 4 : 0);
            if (last && has_z && k + 1 < j1) {
                // (the next group may be the trailing X half of a second-order run)
                if ((st = launch_xpass<R>(s, p, V_ROT_Z, rec, frame, rec + rs)) != QS_OK) return st;
                carried = true;
                dir ^= 1;
            } else {
                if ((st = launch_xpass<R>(s, p, (last && has_z) ? V_ROT_Z : V_ROT, rec, frame, nullptr,
                                          (last && !has_z) ? 1 : 0)) != QS_OK)
                    return st;
            }
        }
        if (s->renorm_every > 0 && steps_per_renorm_unit > 0 &&
            ((k + 1) % ((size_t)s->renorm_every * steps_per_renorm_unit) == 0 || k + 1 == nops))
            if ((st = renormalise<R>(s)) != QS_OK) return st;
    }
    return QS_OK;
}

// Unitary gauge with shared passes: the X layer of factor group k is H^n D_X H^n
// (unnormalised Walsh-Hadamard passes around the Hadamard-basis phase table D_X) and
// the Z layer is diagonal.  The D_X pass applies H(gx) D_X H(gx) on one qubit group, and
// the Z pass applies H(gz), the Z layer of group k and the first H(gz) of group k+1, which
// skips it (all Walsh-Hadamard butterflies on different qubits commute):
//   [H(gz)]  H(0 .. np-3)  [H(gx) D_X H(gx)]  H(np-3 .. 0)  [H(gz) Z_k H(gz)]
// with gx = np-1, gz = np-2: 2 np - 2 passes per factor group instead of 2 np.
template <typename R>
qs_status launch_ops_merged_ug(qs_sim *s, const std::vector<Op> &ops, int steps_per_renorm_unit, size_t j0,
                               size_t j1) {
    qs_status st;
    const int B = s->batch;
    const size_t nops = ops.size() / B;
    const int np = (int)s->passes.size();
    const size_t rs = (size_t)B * s->rec_stride;
    const int gx = np - 1, gz = np - 2;
    bool carried = false;   // H(gz) of op k was applied by op k-1's Z pass
    for (size_t k = j0; k < j1; ++k) {
        const double *rec = s->d_rec + (k - j0) * rs;
        const bool has_z = ops[k * B].has_z;
        if (!carried && (st = launch_xpass<R>(s, gz, V_HAD, rec)) != QS_OK) return st;
        for (int p = 0; p < np - 2; ++p)
            if ((st = launch_xpass<R>(s, p, V_HAD, rec)) != QS_OK) return st;
        if ((st = launch_xpass<R>(s, gx, V_HAD_X, rec, 0, rec)) != QS_OK) return st;   // H D_X H
        for (int p = np - 3; p >= 0; --p)
            if ((st = launch_xpass<R>(s, p, V_HAD, rec)) != QS_OK) return st;
        carried = has_z && k + 1 < j1;
        if (carried) st = launch_xpass<R>(s, gz, V_HAD_Z, rec, 0, rec + rs);      // H Z_k H(next)
        else st = launch_xpass<R>(s, gz, has_z ? V_HAD_Z : V_HAD, rec);
        if (st != QS_OK) return st;
        if (s->renorm_every > 0 && steps_per_renorm_unit > 0 &&
            ((k + 1) % ((size_t)s->renorm_every * steps_per_renorm_unit) == 0 || k + 1 == nops))
            if ((st = renormalise<R>(s)) != QS_OK) return st;
    }
    return QS_OK;
}

template <typename R>
bool merged_schedule_ug(const qs_sim *s) {
    if (sizeof(R) == 8) return s->df_active && s->xmerge && s->passes.size() >= 2;
    return sizeof(R) == 4 && s->method == 0 && s->xmerge && !s->lat.gauge_higgs && s->tmaps_ok &&
           s->xpass_impl != 1 && s->passes.size() >= 2;
}

// complex128 unitary gauge, fused kernels: passes in double-float arithmetic
template <typename R>
bool df_schedule(const qs_sim *s) {
    return sizeof(R) == 8 && s->method == 0 && s->c128_df && s->tmaps_df_ok && s->xpass_impl != 1 &&
           s->passes.size() >= 2 && (!s->lat.gauge_higgs || s->tan_active);
}

template <typename R>
qs_status launch_ops(qs_sim *s, const std::vector<Op> &ops, int steps_per_renorm_unit, size_t j0 = 0,
                     size_t j1 = (size_t)-1) {
    qs_status st;
    const int B = s->batch;
    const size_t nops = ops.size() / B;
    if (j1 > nops) j1 = nops;
    if (merged_schedule<R>(s)) return launch_ops_merged<R>(s, ops, steps_per_renorm_unit, j0, j1);
    if (df_schedule<R>(s) && !s->df_active) {
        // split into the blocked double-float layout, run the passes, join back
        if ((st = df_convert(s, true)) != QS_OK) return st;
        st = launch_ops<R>(s, ops, steps_per_renorm_unit, j0, j1);
        qs_status st2 = df_convert(s, false);
        return st != QS_OK ? st : st2;
    }
    if (merged_schedule_ug<R>(s)) return launch_ops_merged_ug<R>(s, ops, steps_per_renorm_unit, j0, j1);
    for (size_t k = j0; k < j1; ++k) {
        if (s->method == 0)
            st = run_op_fused<R>(s, &ops[k * B], s->d_rec + (k - j0) * B * (size_t)s->rec_stride, k, nops);
        else
            st = run_op_pergate<R>(s, &ops[k * B]);
        if (st != QS_OK) return st;
        if (s->renorm_every > 0 && steps_per_renorm_unit > 0 &&
            ((k + 1) % ((size_t)s->renorm_every * steps_per_renorm_unit) == 0 || k + 1 == nops))
            if ((st = renormalise<R>(s)) != QS_OK) return st;
    }
    return QS_OK;
}

template <typename R>
qs_status run_ops(qs_sim *s, const std::vector<Op> &ops, int steps_per_renorm_unit, const qs_couplings *c,
                  const double *sv, double dt, int n_steps, int order, bool path = false) {
    qs_status st;
    const int B = s->batch;
    const size_t nops = ops.size() / B;
    // tangent form for complex64 gauge-Higgs TMA passes when every factor group of the
    // call has |theta| <= pi/4 and C >= 1/2, i.e. (1 + t0^2)^n0 (1 + t1^2)^n1 <= 4:
    // bounded growth before C is applied, and the scaled Z table u = 1 - C cos phi stays
    // away from 1, where rounding u would cost relative precision in C
    s->tan_active = false;
    const bool tma_path = sizeof(R) == 4 ? s->tmaps_ok : (s->c128_df && s->tmaps_df_ok);
    if (s->method == 0 && s->lat.gauge_higgs && tma_path && s->xpass_impl != 1) {
        bool ok = true;
        for (const Op &o : ops) {
            const double t0 = std::tan(o.thx[0]), t1 = std::tan(o.thx[1]);
            ok = ok && std::fabs(o.thx[0]) <= 0.25 * M_PI && std::fabs(o.thx[1]) <= 0.25 * M_PI &&
                 s->nX0 * std::log1p(t0 * t0) + s->nX1 * std::log1p(t1 * t1) <= 2.0 * std::log(2.0);
        }
        s->tan_active = ok;
    }
    if (s->method == 0) {
        if ((st = upload_inputs(s, c, sv, n_steps, path)) != QS_OK) return st;
        if (nops > REC_CHUNK) {
            // long schedules: records of REC_CHUNK ops at a time, direct launches
            for (size_t j0 = 0; j0 < nops; j0 += REC_CHUNK) {
                const size_t j1 = std::min(nops, j0 + REC_CHUNK);
                if ((st = build_records(s, j0, j1 - j0, dt, n_steps, order)) != QS_OK) return st;
                if ((st = launch_ops<R>(s, ops, steps_per_renorm_unit, j0, j1)) != QS_OK) return st;
            }
            return QS_OK;
        }
        if ((st = build_records(s, 0, nops, dt, n_steps, order)) != QS_OK) return st;
    }
    if (!s->use_graph || s->profile) return launch_ops<R>(s, ops, steps_per_renorm_unit);
    // Replay the launch sequence as a CUDA graph, captured once per configuration on a
    // private stream; the records it reads are rebuilt in place before every replay.
    const long long key[10] = {(long long)nops, order, n_steps, B, (long long)(uintptr_t)s->state[0],
                               (long long)(uintptr_t)s->d_rec, s->renorm_every,
                               s->xpass_impl * 16 + s->nbuf + 256 * s->tma_store + 1024 * s->xmerge +
                                   4096 * (int)s->tan_active + 8192 * s->pdl + 16384 * s->nbuf_shared +
                                   65536 * s->shared_kernel + 131072 * s->c128_df,
                               s->method, (long long)s->dtype};
    if (!s->graph_exec || memcmp(key, s->graph_key, sizeof(key)) != 0) {
        if (s->graph_exec) { cudaGraphExecDestroy(s->graph_exec); s->graph_exec = nullptr; }
        if (!s->cap_stream) CK(s, cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
        cudaStream_t user = s->stream;
        s->stream = s->cap_stream;
        long long before = s->launches;
        CK(s, cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
        st = launch_ops<R>(s, ops, steps_per_renorm_unit);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s->cap_stream, &g);
        s->stream = user;
        s->graph_launches = s->launches - before;
        s->launches = before;
        if (st != QS_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) FAIL(s, QS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&s->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { s->graph_exec = nullptr; FAIL(s, QS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
        memcpy(s->graph_key, key, sizeof(key));
    }
    CK(s, cudaGraphLaunch(s->graph_exec, s->stream));
    s->launches += s->graph_launches;
    return QS_OK;
}

// ---------------------------------------------------------------------------
// adjoint gradient
// ---------------------------------------------------------------------------

template <typename R>
qs_status adjoint_impl(qs_sim *s, const qs_couplings *c, const double *sv, double dt, int n_steps, int order,
                       int target, const void *ref, double *grad_out, double *value_out) {
    qs_status st;
    const int B = s->batch;
    const int np = (int)s->passes.size();
    const long long ntiles = 1ll << (s->n - LT);
    // ---- forward (fused kernels, no renormalisation) ----
    const int saved_method = s->method, saved_renorm = s->renorm_every;
    s->method = 0; s->renorm_every = 0;
    std::vector<Op> ops = build_ops(c, B, sv, dt, n_steps, order, true);
    st = run_ops<R>(s, ops, 1, c, sv, dt, n_steps, order);
    s->method = saved_method; s->renorm_every = saved_renorm;
    if (st != QS_OK) return st;
    const size_t nops = ops.size() / B;
    V<R> *psi = (V<R> *)s->state[0];
    V<R> *lam = (V<R> *)s->state[1];
    const size_t smem = 2 * (size_t)(1 << LT) * sizeof(V<R>) + (size_t)(s->nA + 1) * (s->nB + 1) * sizeof(V<R>);
    const unsigned G = (unsigned)std::min<long long>(ntiles, (long long)s->sm_count * 2);
    // ---- seed lambda ----
    if (target == 0) {
        if ((st = grow(s, &s->d_hrec, &s->hrec_cap, (size_t)B * s->rec_stride, false)) != QS_OK) return st;
        std::vector<double> h((size_t)B * s->rec_stride, 0.0);
        for (int b = 0; b < B; ++b) {
            double *r = &h[(size_t)b * s->rec_stride];
            Coef q = coefficients(c[b], 1.0);          // H1
            r[0] = -q.xs; r[2] = -q.xt;
            for (int a = 0; a <= s->nA; ++a)
                for (int bb = 0; bb <= s->nB; ++bb)
                    r[4 + 2 * (a * (s->nB + 1) + bb)] = -(q.za * (s->nA - 2 * a) + q.zb * (s->nB - 2 * bb));
        }
        CK(s, cudaMemcpyAsync(s->d_hrec, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        for (int p = 0; p < np; ++p) {
            k_apply_h_pass<R><<<dim3(G, B), NT, smem, s->stream>>>(psi, lam, s->dim, ntiles, s->d_hrec, s->rec_stride,
                                                                  s->d_passes + NVAR * p, p == 0);
            CKL(s); s->launches++;
        }
        CK(s, cudaStreamSynchronize(s->stream));   // h is a host temporary
        if ((st = reduce_xmask<R>(s, psi, lam, 0, 0)) != QS_OK) return st;   // <psi|H1|psi>
    } else {
        if (!ref) FAIL(s, QS_ERR_ARG, "fidelity target needs a reference state");
        if ((st = reduce_xmask<R>(s, ref, psi, 0, 0)) != QS_OK) return st;   // <phi|psi>
        k_scaled_copy<R><<<dim3(152 * 8, B), 256, 0, s->stream>>>(lam, (const V<R> *)ref, s->dim, s->d_res);
        CKL(s); s->launches++;
    }
    if ((st = read_results(s, 1)) != QS_OK) return st;
    for (int b = 0; b < B; ++b) {
        double re = res(s, 0, b, 0), im = res(s, 0, b, 1);
        value_out[b] = target == 0 ? re : re * re + im * im;
    }
    // ---- reverse sweep ----
    const size_t nblk = (size_t)np * G;
    const bool use_tma = sizeof(R) == 4 && s->tmaps_ok && s->tmaps_aux_ok && s->adj_impl != 1;
    unsigned Gt = 1;
    // tangent form in the reverse sweep whenever the forward of this call used it (same
    // factor groups, so the same angle checks hold)
    const bool adj_tan = use_tma && s->tan_active;
    const int adj_threads = NT;
    const size_t adj_smem = 2 * (size_t)TMA_TILE_BYTES * s->adj_nbuf + 1024 + (size_t)s->max_lut * 8 + 3 * 256 * 8;
    const AdjKernel adj_kern = adj_tma_kernel(s->adj_nbuf, adj_tan, false, s->adj_early != 0);
    if (use_tma) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj_kern, adj_threads, adj_smem);
        if (per_sm < 1) per_sm = 1;
        Gt = (unsigned)std::min<long long>((long long)B << (s->n - LT), (long long)per_sm * s->sm_count);
    }
    const size_t nblk_t = (size_t)np * Gt;
    // TMA path: one partial-sum region per factor group, two used in turn (a shared reverse
    // pass writes the terms of two consecutive groups)
    const size_t region = nblk_t * B * RED_NV;
    if ((st = grow(s, &s->d_adj_part, &s->adj_part_cap, std::max(nblk * B * RED_NV, 2 * region), false)) != QS_OK)
        return st;
    // shared reverse passes: consecutive factor groups meet on one qubit group, as in the
    // forward sweep (orders ga, 0 .. np-3, gb and gb, 0 .. np-3, ga; ga = np-2, gb = np-1)
    const bool share = adj_tan && s->xmerge && np >= 2;
    const AdjKernel adj_kern_m = adj_tma_kernel(s->adj_nbuf, true, true, s->adj_early != 0);
    int ord[2][64];
    for (int i = 0; i < np; ++i) {
        ord[0][i] = i == 0 ? np - 2 : (i == np - 1 ? np - 1 : i - 1);
        ord[1][i] = i == 0 ? np - 1 : (i == np - 1 ? np - 2 : i - 1);
    }
    bool carried = false;   // the first qubit group of op jj was un-rotated by op jj+1's last pass
    int dir = 0, carry_done[2] = {0, 0};
    if ((st = grow(s, &s->d_grad, &s->grad_cap, nops * B * RED_NV, false)) != QS_OK) return st;
    if ((st = grow(s, &s->h_grad, &s->h_grad_cap, nops * B * RED_NV, true)) != QS_OK) return st;
    size_t chunk0 = (size_t)-1;   // first op whose record is resident in d_rec
    for (size_t jj = nops; jj-- > 0;) {
        if (chunk0 == (size_t)-1 || jj < chunk0) {
            // (re)build the records of the chunk holding op jj (the forward left the last one)
            const size_t c0 = (jj / REC_CHUNK) * REC_CHUNK;
            const size_t c1 = std::min(nops, c0 + REC_CHUNK);
            if ((st = build_records(s, c0, c1 - c0, dt, n_steps, order)) != QS_OK) return st;
            chunk0 = c0;
        }
        const double *rec = s->d_rec + (jj - chunk0) * B * (size_t)s->rec_stride;
        if (use_tma) {
            double *part_j = s->d_adj_part + (jj & 1) * region;
            if (!carried) CK(s, cudaMemsetAsync(part_j, 0, region * sizeof(double), s->stream));
            // X qubits per class already un-rotated in this factor group
            int done[2] = {carried ? carry_done[0] : 0, carried ? carry_done[1] : 0};
            bool next_carried = false;
            for (int i = carried ? 1 : 0; i < np; ++i) {
                const int p = share ? ord[dir][i] : np - 1 - i;
                const bool last = i == np - 1;
                TmaPass P = s->tpasses[NVAR * p + V_ROT];
                P.frame = 1 | ((jj + 1 == nops && i == 0) ? 2 : 0) | ((jj == 0 && last) ? 4 : 0);
                const int zinv = (i == 0 && ops[jj * B].has_z) ? 1 : 0;
                P.xscale = (adj_tan && i == 0 && !ops[jj * B].has_z) ? 1 : 0;
                for (int stg = 0; stg < 3; ++stg) {          // stages run A, B, C
                    P.adj_u[stg][0] = s->nX0 - done[0];
                    P.adj_u[stg][1] = s->nX1 - done[1];
                    for (int kk = 0; kk < RB; ++kk)
                        if ((P.rot[stg] >> kk) & 1u) done[(P.cls[stg] >> kk) & 1u]++;
                }
                const bool merge = share && last && jj >= 1 && jj - 1 >= chunk0 && ops[(jj - 1) * B].has_z;
                if (merge) {
                    // last pass of op jj, Z layer and first pass of op jj-1 on the same qubits
                    double *part_prev = s->d_adj_part + ((jj - 1) & 1) * region;
                    const double *rec_prev = rec - B * (size_t)s->rec_stride;
                    CK(s, cudaMemsetAsync(part_prev, 0, region * sizeof(double), s->stream));
                    int d2[2] = {0, 0};
                    for (int stg = 2; stg >= 0; --stg) {     // second rotation round runs C, B, A
                        P.adj_u2[stg][0] = s->nX0 - d2[0];
                        P.adj_u2[stg][1] = s->nX1 - d2[1];
                        for (int kk = 0; kk < RB; ++kk)
                            if ((P.rot[stg] >> kk) & 1u) d2[(P.cls[stg] >> kk) & 1u]++;
                    }
                    carry_done[0] = d2[0];
                    carry_done[1] = d2[1];
                    if (s->shared_kernel == 1 && B == 1 && P.rot[1] == 0 && !P.stage_b && P.frame == 1 &&
                        P.total_tiles < (1ll << 30)) {
                        // warp-local slices: one CTA of 12 warps per SM (11 consumers, 155
                        // registers), three pair buffers, each reloaded once its store has read
                        // it (measured against 10, 11, 14 and 16 warps and the later reload)
                        const size_t wsm = 2 * (size_t)TMA_TILE_BYTES * 3 + 1024 + (size_t)s->max_lut * 8 + 3 * 256 * 8;
                        const unsigned gw = (unsigned)std::min<long long>(P.total_tiles, (long long)s->sm_count);
                        k_adj_wl<3, 12, 1, 0><<<gw, 384, wsm, s->stream>>>(
                            (float2 *)s->state[0], (float2 *)s->state[1], rec, s->rec_stride, s->n - LT, s->d_err,
                            part_j, (int)nblk_t, i * (int)Gt, 0, rec_prev, part_prev, 0, s->tmaps[p], s->tmaps_aux[p],
                            P);
                    } else {
                        adj_kern_m<<<Gt, adj_threads, adj_smem, s->stream>>>(
                            (float2 *)s->state[0], (float2 *)s->state[1], rec, s->rec_stride, s->n - LT, s->d_err,
                            part_j, (int)nblk_t, i * (int)Gt, 0, rec_prev, part_prev, 0, s->tmaps[p], s->tmaps_aux[p],
                            P);
                    }
                    next_carried = true;
                    dir ^= 1;
                } else {
                    adj_kern<<<Gt, adj_threads, adj_smem, s->stream>>>(
                        (float2 *)s->state[0], (float2 *)s->state[1], rec, s->rec_stride, s->n - LT, s->d_err, part_j,
                        (int)nblk_t, i * (int)Gt, zinv, rec, part_j, 0, s->tmaps[p], s->tmaps_aux[p], P);
                }
                CKL(s); s->launches++;
            }
            if (done[0] != s->nX0 || done[1] != s->nX1)
                FAIL(s, QS_ERR_STATE, "reverse passes do not cover every X qubit once");
            k_finish<<<B, RED_THREADS, 0, s->stream>>>(part_j, (int)nblk_t, 4, s->d_grad + jj * B * RED_NV);
            CKL(s); s->launches++;
            carried = next_carried;
            continue;
        }
        for (int pi = 0; pi < np; ++pi) {
            const int p = np - 1 - pi;
            k_adj_xpass<R><<<dim3(G, B), NT, smem, s->stream>>>(psi, lam, s->dim, ntiles, rec, s->rec_stride,
                                                               s->d_passes + NVAR * p, (pi == 0 && ops[jj * B].has_z) ? 1 : 0,
                                                               s->d_adj_part, (int)nblk, pi * (int)G);
            CKL(s); s->launches++;
        }
        k_finish<<<B, RED_THREADS, 0, s->stream>>>(s->d_adj_part, (int)nblk, 4, s->d_grad + jj * B * RED_NV);
        CKL(s); s->launches++;
    }
    CK(s, cudaMemcpyAsync(s->h_grad, s->d_grad, nops * B * RED_NV * sizeof(double), cudaMemcpyDeviceToHost,
                          s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    if ((st = check_device_flag(s)) != QS_OK) return st;
    // ---- chain rule to s_k: dV/dtheta = -2 Im<lambda|P|psi> ----
    const int N = n_steps;
    for (int b = 0; b < B; ++b) {
        double *g = grad_out + (size_t)b * N;
        for (int k = 0; k < N; ++k) g[k] = 0.0;
        const double dxs = c[b].g - 1.0, dxt = c[b].J - 1.0;   // d/ds of the X coefficients
        for (size_t j = 0; j < nops; ++j) {
            const double *v = s->h_grad + (j * B + b) * RED_NV;
            for (int q = 0; q < 4; ++q)
                if (!std::isfinite(v[q])) FAIL(s, QS_ERR_NONFINITE, "non-finite adjoint reduction");
            const double gx = -2.0 * (dxs * v[0] + dxt * v[1]);
            if (order == 1) {
                g[j] += gx * dt;
            } else {
                if (j < (size_t)N) g[j] += gx * 0.5 * dt;
                if (j >= 1) g[j - 1] += gx * 0.5 * dt;
            }
            if (ops[j * B].has_z) g[j] += -2.0 * (c[b].h * dt * v[2] + c[b].lambda * dt * v[3]);
        }
    }
    return QS_OK;
}

// Parameters of the on-chip 12-qubit scan (the 2x2 torus in the gauge-Higgs form).
ScanParams scan12_params(const qs_sim *s, int n_points, int n_steps, int order, double dt) {
    ScanParams P;
    memset(&P, 0, sizeof(P));
    P.n_points = n_points; P.n_ops = order == 2 ? n_steps + 1 : n_steps;
    P.G.n_steps = n_steps; P.G.order = order; P.G.fsal = order == 2; P.G.batch = 1; P.G.dt = dt;
    P.G.f32 = s->dtype == QS_C64;
    P.nA = s->nA; P.nB = s->nB;
    for (int q = 0; q < LT; ++q) {
        for (int k = 0; k < s->nA; ++k) if ((s->lat.plaquettes[k] >> q) & 1) P.colA[q] |= 1u << k;
        for (int k = 0; k < s->nB; ++k) if ((s->lat.second[k] >> q) & 1) P.colB[q] |= 1u << k;
        if (s->lat.x_class[q]) P.cls_mask |= 1u << q;
    }
    if (s->lat.wilson.size() == 2) { P.wx = (uint32_t)s->lat.wilson[0]; P.wy = (uint32_t)s->lat.wilson[1]; }
    P.n_link = s->lat.n_links; P.n_vertex = s->n - s->lat.n_links;
    return P;
}

qs_status check_ready(qs_sim *s) {
    if (!s) return QS_ERR_ARG;
    if (!s->state[0]) FAIL(s, QS_ERR_STATE, "no state bound (qs_bind_state slot 0)");
    return QS_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

qs_status qs_create(int Lx, int Ly, int boundary, int form, int dtype, int batch, qs_sim **out) {
    g_create_error.clear();
    if (!out) { g_create_error = "out is NULL"; return QS_ERR_ARG; }
    *out = nullptr;
    if (boundary != QS_PERIODIC && boundary != QS_OPEN) { g_create_error = "bad boundary"; return QS_ERR_ARG; }
    if (form != QS_GAUGE_HIGGS && form != QS_UNITARY_GAUGE) { g_create_error = "bad form"; return QS_ERR_ARG; }
    if (dtype != QS_C64 && dtype != QS_C128) { g_create_error = "bad dtype"; return QS_ERR_ARG; }
    if (batch < 1 || batch > 65535) { g_create_error = "batch must be in [1, 65535]"; return QS_ERR_ARG; }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        g_create_error = "no CUDA device";
        return QS_ERR_CUDA;
    }
    qs_sim *s = new (std::nothrow) qs_sim();
    if (!s) { g_create_error = "host allocation failed"; return QS_ERR_OOM; }
    try {
        s->lat = make_lattice(Lx, Ly, boundary == QS_PERIODIC, form == QS_GAUGE_HIGGS);
    } catch (const std::exception &e) {
        g_create_error = e.what();
        delete s;
        return QS_ERR_ARG;
    }
    s->boundary = boundary; s->form = form; s->dtype = dtype; s->batch = batch;
    s->n = s->lat.n_qubits;
    if (s->n > 34 || s->n < 2) {
        g_create_error = "qubit count must be in [2, 34]";
        delete s;
        return QS_ERR_ARG;
    }
    s->dim = 1ll << s->n;
    s->nA = (int)s->lat.plaquettes.size();
    s->nB = (int)s->lat.second.size();
    if (s->nA > 32 || s->nB > 32) { g_create_error = "more than 32 terms in a Z class"; delete s; return QS_ERR_ARG; }
    s->rec_stride = record_doubles(s->nA, s->nB);
    s->max_lut = (s->nA + 1) * (s->nB + 1);
    if (!s->lat.gauge_higgs) {
        s->nXA = (int)s->lat.stars.size();
        s->nXB = s->lat.n_links;
        if (s->nXA > 32 || s->nXB > 32) { g_create_error = "more than 32 terms in an X class"; delete s; return QS_ERR_ARG; }
        s->xlut_off = s->rec_stride;
        s->rec_stride += 2 * (s->nXA + 1) * (s->nXB + 1);
        s->max_lut = std::max(s->max_lut, (s->nXA + 1) * (s->nXB + 1));
    }
    s->tan_off = s->rec_stride;
    s->rec_stride += 4 + 2 * (s->nA + 1) * (s->nB + 1);   // triple + scaled Z table
    for (int qb = 0; qb < s->n; ++qb) (s->lat.x_class[qb] ? s->nX1 : s->nX0)++;
    build_passes(s);
    build_variants(s);
    build_tma_passes(s);
    auto fail = [&](const char *what) {
        g_create_error = what;
        qs_destroy(s);
        return QS_ERR_OOM;
    };
    const std::vector<PassDesc> &dev = s->pvar;
    if (!dev.empty()) {
        if (cudaMalloc((void **)&s->d_passes, dev.size() * sizeof(PassDesc)) != cudaSuccess) return fail("pass table");
        if (cudaMemcpy(s->d_passes, dev.data(), dev.size() * sizeof(PassDesc), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail("pass table copy");
    }
    std::vector<uint32_t> ca(MAXQ, 0), cb(MAXQ, 0);
    for (int q = 0; q < s->n; ++q) {
        for (int p = 0; p < s->nA; ++p) if ((s->lat.plaquettes[p] >> q) & 1) ca[q] |= 1u << p;
        for (int p = 0; p < s->nB; ++p) if ((s->lat.second[p] >> q) & 1) cb[q] |= 1u << p;
    }
    if (cudaMalloc((void **)&s->d_colA, MAXQ * sizeof(uint32_t)) != cudaSuccess) return fail("columns");
    if (cudaMalloc((void **)&s->d_colB, MAXQ * sizeof(uint32_t)) != cudaSuccess) return fail("columns");
    if (cudaMemcpy(s->d_colA, ca.data(), MAXQ * 4, cudaMemcpyHostToDevice) != cudaSuccess) return fail("columns copy");
    if (cudaMemcpy(s->d_colB, cb.data(), MAXQ * 4, cudaMemcpyHostToDevice) != cudaSuccess) return fail("columns copy");
    size_t pbytes = (size_t)RED_BLOCKS * batch * RED_NV * sizeof(double);
    size_t rbytes = (size_t)RES_SLOTS * batch * RED_NV * sizeof(double);
    if (cudaMalloc((void **)&s->d_partials, pbytes) != cudaSuccess) return fail("partials");
    if (cudaMalloc((void **)&s->d_res, rbytes) != cudaSuccess) return fail("results");
    if (cudaMallocHost((void **)&s->h_res, rbytes) != cudaSuccess) return fail("pinned results");
    if (cudaEventCreateWithFlags(&s->rec_done, cudaEventDisableTiming) != cudaSuccess) return fail("event");
    if (cudaMalloc((void **)&s->d_err, sizeof(int)) != cudaSuccess) return fail("error flag");
    if (cudaMemset(s->d_err, 0, sizeof(int)) != cudaSuccess) return fail("error flag");
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (s->sm_count < 1) s->sm_count = 1;
        for (int nb = 2; nb <= 3; ++nb)
            for (int v = 0; v < 8; ++v)
                cudaFuncSetAttribute(xpass_tma_kernel(nb, v & 1, (v >> 1) & 1, (v >> 2) & 1),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem_bytes(s, nb, true));
        cudaFuncSetAttribute(k_xpass_df<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)df_smem_bytes(s));
        cudaFuncSetAttribute(k_xpass_df<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)df_smem_bytes(s));
        cudaFuncSetAttribute(k_xpass_df<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)df_smem_bytes(s));
        cudaFuncSetAttribute(k_xpass_df<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)df_smem_bytes(s));
        cudaFuncSetAttribute(k_adj_wl<3, 12, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * (size_t)TMA_TILE_BYTES * 3 + 1024 + (size_t)s->max_lut * 8 + 3 * 256 * 8));
        for (int h = 0; h < 2; ++h) {
            cudaFuncSetAttribute(h ? k_xpass_wl<2, 8, 3, true> : k_xpass_wl<2, 8, 3, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem_bytes(s, 2, true));
            cudaFuncSetAttribute(h ? k_xpass_wl<3, 8, 2, true> : k_xpass_wl<3, 8, 2, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem_bytes(s, 3, true));
            cudaFuncSetAttribute(h ? k_xpass_wl<6, 24, 1, true> : k_xpass_wl<6, 24, 1, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem_bytes(s, 6, true));
        }
        int adj64 = (int)(2 * (1 << LT) * 16 + (size_t)(s->nA + 1) * (s->nB + 1) * 16);
        cudaFuncSetAttribute(k_adj_xpass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, adj64);
        cudaFuncSetAttribute(k_adj_xpass<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, adj64);
        cudaFuncSetAttribute(k_apply_h_pass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, adj64);
        cudaFuncSetAttribute(k_apply_h_pass<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, adj64);
        cudaFuncSetAttribute(k_xmeasure<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)((1 << LT) * 16));
        for (int v = 0; v < 3; ++v) {
            const bool tn = v >= 1, mg = v == 2;
            cudaFuncSetAttribute(adj_tma_kernel(2, tn, mg), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(4 * TMA_TILE_BYTES + 1024 + (size_t)s->max_lut * 8 + 3 * 256 * 8));
            for (int ea = 0; ea < 2; ++ea)
                cudaFuncSetAttribute(adj_tma_kernel(1, tn, mg, ea != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(2 * TMA_TILE_BYTES + 1024 + (size_t)s->max_lut * 8 + 3 * 256 * 8));
        }

    }
    size_t smem64 = (size_t)(1 << LT) * 16 + (size_t)s->max_lut * 16;
    cudaFuncSetAttribute(k_xpass<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64);
    cudaFuncSetAttribute(k_xpass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64);
    *out = s;
    return QS_OK;
}

void qs_destroy(qs_sim *s) {
    if (!s) return;
    if (s->stream || true) cudaStreamSynchronize(s->stream);
    cudaFree(s->d_passes);
    cudaFree(s->d_colA);
    cudaFree(s->d_colB);
    cudaFree(s->d_rec);
    cudaFree(s->d_partials);
    cudaFree(s->d_res);
    cudaFree(s->d_err);
    cudaFree(s->d_adj_part);
    cudaFree(s->d_grad);
    cudaFree(s->d_hrec);
    cudaFree(s->d_scan);
    cudaFree(s->d_queue);
    cudaFree(s->d_in);
    if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
    if (s->scan_graph) cudaGraphExecDestroy(s->scan_graph);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->h_scan) cudaFreeHost(s->h_scan);
    if (s->h_grad) cudaFreeHost(s->h_grad);
    if (s->h_rec) cudaFreeHost(s->h_rec);
    if (s->h_res) cudaFreeHost(s->h_res);
    if (s->rec_done) cudaEventDestroy(s->rec_done);
    for (auto e : s->ev_pool) cudaEventDestroy(e);
    delete s;
}

const char *qs_last_error(const qs_sim *s) {
    return s ? s->err.c_str() : g_create_error.c_str();
}

int qs_num_qubits(const qs_sim *s) { return s ? s->n : -1; }

size_t qs_state_bytes(const qs_sim *s) {
    if (!s) return 0;
    return (size_t)s->batch * (size_t)s->dim * (s->dtype == QS_C64 ? 8u : 16u);
}

qs_status qs_bind_state(qs_sim *s, int slot, void *ptr, size_t bytes) {
    if (!s) return QS_ERR_ARG;
    if (slot < 0 || slot > 1) FAIL(s, QS_ERR_ARG, "slot must be 0 or 1");
    if (!ptr) FAIL(s, QS_ERR_ARG, "null device pointer");
    if (((uintptr_t)ptr & 255u) != 0) FAIL(s, QS_ERR_ARG, "state pointer must be 256-byte aligned");
    if (bytes < qs_state_bytes(s)) FAIL(s, QS_ERR_ARG, "buffer of %zu bytes < %zu", bytes, qs_state_bytes(s));
    s->state[slot] = ptr;
    s->state_cap[slot] = bytes;
    return encode_tmaps(s, slot);
}

qs_status qs_set_stream(qs_sim *s, void *stream) {
    if (!s) return QS_ERR_ARG;
    s->stream = (cudaStream_t)stream;
    return QS_OK;
}

qs_status qs_set_option(qs_sim *s, int key, long long value) {
    if (!s) return QS_ERR_ARG;
    switch (key) {
        case QS_OPT_METHOD:
            if (value != 0 && value != 1) FAIL(s, QS_ERR_ARG, "method must be 0 or 1");
            s->method = (int)value; return QS_OK;
        case QS_OPT_RENORM_EVERY:
            if (value < 0) FAIL(s, QS_ERR_ARG, "renorm interval must be >= 0");
            s->renorm_every = (int)value; return QS_OK;
        case QS_OPT_PROFILE: s->profile = value != 0; return QS_OK;
        case QS_OPT_GRAPH: s->use_graph = value != 0; return QS_OK;
        case QS_OPT_XPASS:
            if (value < 0 || value > 2) FAIL(s, QS_ERR_ARG, "xpass kernel must be 0 (auto), 1 or 2");
            s->xpass_impl = (int)value; return QS_OK;
        case QS_OPT_TMA_STORE:
            s->tma_store = value != 0; return QS_OK;
        case QS_OPT_XMERGE:
            s->xmerge = value != 0; return QS_OK;
        case QS_OPT_PDL:
            s->pdl = value != 0; return QS_OK;
        case QS_OPT_SHARED_BUFFERS:
            if (value != 0 && value != 2 && value != 3)
                FAIL(s, QS_ERR_ARG, "shared-pass TMA buffers must be 0 (by form), 2 or 3");
            s->nbuf_shared = (int)value; return QS_OK;
        case QS_OPT_C128_DF:
            if (value != 0 && value != 1) FAIL(s, QS_ERR_ARG, "double-float option must be 0 or 1");
            s->c128_df = (int)value; return QS_OK;
        case QS_OPT_SHARED_KERNEL:
            if (value != 0 && value != 1) FAIL(s, QS_ERR_ARG, "shared-pass kernel must be 0 or 1");
            s->shared_kernel = (int)value; return QS_OK;
        case QS_OPT_ADJOINT:
            if (value < 0 || value > 7) FAIL(s, QS_ERR_ARG, "adjoint option must be 0..7");
            s->adj_impl = (value & 1) ? 1 : 0;
            s->adj_nbuf = (value & 2) ? 2 : 1;
            s->adj_early = (value & 6) ? 0 : 1;
            return QS_OK;
        case QS_OPT_TMA_BUFFERS:
            if (value != 2 && value != 3) FAIL(s, QS_ERR_ARG, "TMA buffers must be 2 or 3");
            s->nbuf = (int)value; return QS_OK;
        case QS_OPT_SCAN_BUFFERS:
            if (value != 0 && value != 2 && value != 3 && value != 4 && value != 6)
                FAIL(s, QS_ERR_ARG, "scan tile buffers must be 0 (default 3), 2, 3, 4 or 6");
            s->scan_buffers = value ? (int)value : 3;
            return QS_OK;
        case QS_OPT_PLAN: {
            if (s->n <= LT) FAIL(s, QS_ERR_ARG, "a pass plan needs more than %d qubits", LT);
            if (value < 0) FAIL(s, QS_ERR_ARG, "bad plan");
            std::vector<int> k;
            int sum = 0;
            for (long long v = value; v; v >>= 4) {
                const int x = (int)(v & 15);
                if (x < 1 || x > 8) FAIL(s, QS_ERR_ARG, "each pass of a plan fuses 1 to 8 new qubits");
                k.push_back(x);
                sum += x;
            }
            if (value != 0 && sum != s->n - LT)
                FAIL(s, QS_ERR_ARG, "the plan fuses %d new qubits, the state has %d beyond the first pass", sum,
                     s->n - LT);
            s->plan_k = k;
            s->plan_code = value;
            return rebuild_plan(s);
        }
        default: FAIL(s, QS_ERR_ARG, "unknown option %d", key);
    }
}

qs_status qs_init_plus(qs_sim *s) {
    qs_status st;
    if ((st = check_ready(s)) != QS_OK) return st;
    long long count = s->dim * s->batch;
    double a = 1.0 / sqrt((double)s->dim);
    if (s->dtype == QS_C64)
        k_fill<float><<<152 * 8, 256, 0, s->stream>>>((float2 *)s->state[0], count, (float)a);
    else
        k_fill<double><<<152 * 8, 256, 0, s->stream>>>((double2 *)s->state[0], count, a);
    CKL(s); s->launches++;
    return QS_OK;
}

qs_status qs_init_toric(qs_sim *s, int which) {
    qs_status st;
    if ((st = check_ready(s)) != QS_OK) return st;
    if (s->lat.gauge_higgs) FAIL(s, QS_ERR_ARG, "toric-code initial states are defined in the unitary gauge");
    if (which != 0 && which != 1) FAIL(s, QS_ERR_ARG, "which must be 0 (B_p = +1 from |+>) or 1 (A_v = +1 from |0>)");
    // support: every plaquette even; for which = 1 also both Wilson loops even
    uint64_t w0 = 0, w1 = 0;
    if (which == 1 && s->lat.wilson.size() == 2) { w0 = s->lat.wilson[0]; w1 = s->lat.wilson[1]; }
    dim3 grid(152 * 8, (unsigned)s->batch);
    if (s->dtype == QS_C64)
        k_init_even<float><<<grid, 256, 0, s->stream>>>((float2 *)s->state[0], s->n, s->dim, s->d_colA,
                                                         (unsigned long long)w0, (unsigned long long)w1);
    else
        k_init_even<double><<<grid, 256, 0, s->stream>>>((double2 *)s->state[0], s->n, s->dim, s->d_colA,
                                                          (unsigned long long)w0, (unsigned long long)w1);
    CKL(s); s->launches++;
    return s->dtype == QS_C64 ? renormalise<float>(s) : renormalise<double>(s);
}

qs_status qs_upload_state(qs_sim *s, const void *host, size_t bytes) {
    qs_status st;
    if ((st = check_ready(s)) != QS_OK) return st;
    if (!host || bytes != qs_state_bytes(s)) FAIL(s, QS_ERR_ARG, "host buffer must hold qs_state_bytes");
    CK(s, cudaMemcpyAsync(s->state[0], host, bytes, cudaMemcpyHostToDevice, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    return QS_OK;
}

qs_status qs_download_state(qs_sim *s, void *host, size_t bytes) {
    qs_status st;
    if ((st = check_ready(s)) != QS_OK) return st;
    if (!host || bytes != qs_state_bytes(s)) FAIL(s, QS_ERR_ARG, "host buffer must hold qs_state_bytes");
    CK(s, cudaMemcpyAsync(host, s->state[0], bytes, cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    return QS_OK;
}

static qs_status evolve_impl(qs_sim *s, const qs_couplings *c, const double *sv, double dt, int n_steps,
                             int order, bool path = false) {
    qs_status st;
    if ((st = check_ready(s)) != QS_OK) return st;
    if (!c || (!sv && !path)) FAIL(s, QS_ERR_ARG, "null couplings or schedule");
    if (order != 1 && order != 2) FAIL(s, QS_ERR_ARG, "order must be 1 or 2");
    if (n_steps < 0) FAIL(s, QS_ERR_ARG, "n_steps < 0");
    if (!std::isfinite(dt)) FAIL(s, QS_ERR_ARG, "dt not finite");
    if (n_steps == 0) return QS_OK;
    bool fsal = (s->method == 0);
    std::vector<Op> ops = build_ops(c, s->batch, sv, dt, n_steps, order, fsal, path);
    int per_step = (order == 2 && !fsal) ? 2 : 1;
    if (s->dtype == QS_C64) return run_ops<float>(s, ops, per_step, c, sv, dt, n_steps, order, path);
    return run_ops<double>(s, ops, per_step, c, sv, dt, n_steps, order, path);
}

qs_status qs_evolve_path(qs_sim *s, const qs_couplings *per_step, double dt, int n_steps, int order) {
    return evolve_impl(s, per_step, nullptr, dt, n_steps, order, true);
}

qs_status qs_trotter_step(qs_sim *s, const qs_couplings *c, double sv, double dt, int order) {
    return evolve_impl(s, c, &sv, dt, 1, order);
}

qs_status qs_evolve(qs_sim *s, const qs_couplings *c, const double *sv, double dt, int n_steps, int order) {
    return evolve_impl(s, c, sv, dt, n_steps, order);
}

}  // extern "C"

template <typename R>
static qs_status expect_impl(qs_sim *s, int kind, int index, const qs_couplings *c, double sval, double *out) {
    qs_status st;
    const Lattice &L = s->lat;
    const int B = s->batch;
    auto xm = [&](uint64_t m, int slot) { return reduce_xmask<R>(s, s->state[0], s->state[0], m, slot); };
    switch (kind) {
        case QS_NORM:
            if ((st = reduce_diag<R>(s, s->state[0], 0, 0)) != QS_OK) return st;
            if ((st = read_results(s, 1)) != QS_OK) return st;
            for (int b = 0; b < B; ++b) out[b] = res(s, 0, b, 0);
            return QS_OK;
        case QS_PLAQUETTE:
        case QS_WILSON: {
            uint64_t m = 0;
            if (kind == QS_PLAQUETTE) {
                if (index < -1 || index >= (int)L.plaquettes.size()) FAIL(s, QS_ERR_ARG, "plaquette index");
                if (index >= 0) m = L.plaquettes[index];
            } else {
                if (index < 0 || index >= (int)L.wilson.size()) FAIL(s, QS_ERR_ARG, "Wilson loop index");
                m = L.wilson[index];
            }
            if ((st = reduce_diag<R>(s, s->state[0], m, 0)) != QS_OK) return st;
            if ((st = read_results(s, 1)) != QS_OK) return st;
            for (int b = 0; b < B; ++b)
                out[b] = (kind == QS_PLAQUETTE && index == -1) ? res(s, 0, b, 1) / L.plaquettes.size()
                                                               : res(s, 0, b, 3);
            return QS_OK;
        }
        case QS_X:
        case QS_GAUSS:
        case QS_THOOFT: {
            uint64_t m;
            if (kind == QS_X) {
                if (index < 0 || index >= s->n) FAIL(s, QS_ERR_ARG, "qubit index");
                m = 1ull << index;
            } else if (kind == QS_GAUSS) {
                if (index < 0 || index >= (int)L.gauss.size()) FAIL(s, QS_ERR_ARG, "Gauss index (gauge-Higgs form only)");
                m = L.gauss[index];
            } else {
                if (index < 0 || index >= (int)L.thooft.size()) FAIL(s, QS_ERR_ARG, "'t Hooft index");
                m = L.thooft[index];
            }
            if ((st = xm(m, 0)) != QS_OK) return st;
            if ((st = read_results(s, 1)) != QS_OK) return st;
            for (int b = 0; b < B; ++b) out[b] = res(s, 0, b, 0);
            return QS_OK;
        }
        case QS_ENERGY:
        case QS_ENERGY_S: {
            if (!c) FAIL(s, QS_ERR_ARG, "energy needs couplings");
            double sv = (kind == QS_ENERGY) ? 1.0 : sval;
            int slot = 0;
            if ((st = reduce_diag<R>(s, s->state[0], 0, slot++)) != QS_OK) return st;
            const int np = (int)s->passes.size();
            int xslot = -1;
            if (np > 0) {
                // single-qubit X terms: one read-only sweep per pass, sums per class
                const long long ntiles = 1ll << (s->n - LT);
                const unsigned G = (unsigned)std::min<long long>(ntiles, (long long)s->sm_count * 4);
                const size_t nblk = (size_t)np * G;
                if ((st = grow(s, &s->d_adj_part, &s->adj_part_cap, nblk * B * RED_NV, false)) != QS_OK) return st;
                const size_t smem = (size_t)(1 << LT) * sizeof(V<R>);
                for (int p = 0; p < np; ++p) {
                    k_xmeasure<R><<<dim3(G, B), NT, smem, s->stream>>>((const V<R> *)s->state[0], s->dim, ntiles,
                                                                      s->d_passes + NVAR * p, s->d_adj_part,
                                                                      (int)nblk, p * (int)G);
                    CKL(s); s->launches++;
                }
                xslot = slot++;
                k_finish<<<B, RED_THREADS, 0, s->stream>>>(s->d_adj_part, (int)nblk, 2,
                                                           s->d_res + (size_t)xslot * B * RED_NV);
                CKL(s); s->launches++;
            }
            const int q0 = slot;
            if (np == 0)
                for (int q = 0; q < s->n; ++q)
                    if ((st = xm(1ull << q, slot++)) != QS_OK) return st;
            int star0 = slot;
            if (!L.gauge_higgs)
                for (uint64_t m : L.stars)
                    if ((st = xm(m, slot++)) != QS_OK) return st;
            if ((st = read_results(s, slot)) != QS_OK) return st;
            for (int b = 0; b < B; ++b) {
                Coef q = coefficients(c[b], sv);
                double e = -q.za * res(s, 0, b, 1) - q.zb * res(s, 0, b, 2);
                if (xslot >= 0) {
                    // each pair counted once: <X_q> = 2 sum_pairs Re(conj(a) b)
                    e -= q.xs * 2.0 * res(s, xslot, b, 0) + q.xt * 2.0 * res(s, xslot, b, 1);
                } else {
                    for (int k = 0; k < s->n; ++k)
                        e -= (L.x_class[k] ? q.xt : q.xs) * res(s, q0 + k, b, 0);
                }
                for (int k = star0; k < slot; ++k) e -= q.xt * res(s, k, b, 0);
                out[b] = e;
            }
            return QS_OK;
        }
        default:
            FAIL(s, QS_ERR_ARG, "unknown observable %d", kind);
    }
}

extern "C" {

qs_status qs_expect(qs_sim *s, int kind, int index, const qs_couplings *c, double sval, double *out) {
    qs_status st;
    if ((st = check_ready(s)) != QS_OK) return st;
    if (!out) FAIL(s, QS_ERR_ARG, "null output");
    if (s->dtype == QS_C64) return expect_impl<float>(s, kind, index, c, sval, out);
    return expect_impl<double>(s, kind, index, c, sval, out);
}

qs_status qs_expect_pauli(qs_sim *s, int type, uint64_t mask, double *out) {
    qs_status st;
    if ((st = check_ready(s)) != QS_OK) return st;
    if (!out) FAIL(s, QS_ERR_ARG, "null output");
    if (type != 0 && type != 1) FAIL(s, QS_ERR_ARG, "type must be 0 (Z) or 1 (X)");
    if (s->n < 64 && (mask >> s->n) != 0) FAIL(s, QS_ERR_ARG, "mask has bits beyond the qubit count");
    if (type == 0) {
        st = s->dtype == QS_C64 ? reduce_diag<float>(s, s->state[0], mask, 0)
                                : reduce_diag<double>(s, s->state[0], mask, 0);
    } else {
        st = s->dtype == QS_C64 ? reduce_xmask<float>(s, s->state[0], s->state[0], mask, 0)
                                : reduce_xmask<double>(s, s->state[0], s->state[0], mask, 0);
    }
    if (st != QS_OK) return st;
    if ((st = read_results(s, 1)) != QS_OK) return st;
    for (int b = 0; b < s->batch; ++b) out[b] = res(s, 0, b, type == 0 ? 3 : 0);
    return QS_OK;
}

qs_status qs_fidelity(qs_sim *s, const void *ref, double *out) {
    qs_status st;
    if ((st = check_ready(s)) != QS_OK) return st;
    if (!ref || !out) FAIL(s, QS_ERR_ARG, "null argument");
    st = s->dtype == QS_C64 ? reduce_xmask<float>(s, ref, s->state[0], 0, 0)
                            : reduce_xmask<double>(s, ref, s->state[0], 0, 0);
    if (st != QS_OK) return st;
    if ((st = read_results(s, 1)) != QS_OK) return st;
    for (int b = 0; b < s->batch; ++b) {
        double re = res(s, 0, b, 0), im = res(s, 0, b, 1);
        out[b] = re * re + im * im;
    }
    return QS_OK;
}

qs_status qs_adjoint_grad(qs_sim *s, const qs_couplings *c, const double *sv, double dt, int n_steps, int order,
                          int target, const void *ref, double *dV_ds, double *value_out) {
    qs_status st;
    if ((st = check_ready(s)) != QS_OK) return st;
    if (!c || !sv || !dV_ds || !value_out) FAIL(s, QS_ERR_ARG, "null argument");
    if (!s->state[1]) FAIL(s, QS_ERR_STATE, "the adjoint needs a work state bound to slot 1");
    if (!s->lat.gauge_higgs) FAIL(s, QS_ERR_ARG, "the adjoint gradient supports the gauge-Higgs form");
    if (s->n < LT) FAIL(s, QS_ERR_ARG, "the adjoint gradient needs at least %d qubits", LT);
    if (order != 1 && order != 2) FAIL(s, QS_ERR_ARG, "order must be 1 or 2");
    if (n_steps < 1) FAIL(s, QS_ERR_ARG, "n_steps must be >= 1");
    if (target != 0 && target != 1) FAIL(s, QS_ERR_ARG, "target must be 0 (energy) or 1 (fidelity)");
    if (s->dtype == QS_C64)
        return adjoint_impl<float>(s, c, sv, dt, n_steps, order, target, ref, dV_ds, value_out);
    return adjoint_impl<double>(s, c, sv, dt, n_steps, order, target, ref, dV_ds, value_out);
}

qs_status qs_scan(qs_sim *s, const qs_couplings *points, int n_points, const double *sv, double dt, int n_steps,
                  int order, double *out) {
    if (!s) return QS_ERR_ARG;
    if (!points || !sv || !out) FAIL(s, QS_ERR_ARG, "null argument");
    if (n_points < 1 || n_steps < 1) FAIL(s, QS_ERR_ARG, "n_points and n_steps must be >= 1");
    if (order != 1 && order != 2) FAIL(s, QS_ERR_ARG, "order must be 1 or 2");
    if (s->n == LT && s->lat.gauge_higgs && s->nA + s->nB + 2 <= 64) {
        // ---- every point in one persistent launch, state in shared memory ----
        size_t in_doubles = (size_t)n_points * 4 + (size_t)n_steps;
        size_t out_doubles = (size_t)n_points * SCAN_NOBS;
        qs_status st;
        if ((st = grow(s, &s->d_scan, &s->scan_cap, in_doubles + out_doubles, false)) != QS_OK) return st;
        if ((st = grow(s, &s->h_scan, &s->h_scan_cap, in_doubles + out_doubles, true)) != QS_OK) return st;
        for (int p = 0; p < n_points; ++p) {
            s->h_scan[4 * p] = points[p].J; s->h_scan[4 * p + 1] = points[p].h;
            s->h_scan[4 * p + 2] = points[p].g; s->h_scan[4 * p + 3] = points[p].lambda;
        }
        memcpy(s->h_scan + 4 * (size_t)n_points, sv, (size_t)n_steps * sizeof(double));
        const ScanParams P = scan12_params(s, n_points, n_steps, order, dt);
        int per_sm = 0;
        if (s->dtype == QS_C64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan12<float>, NT, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan12<double>, NT, 0);
        if (per_sm < 1) per_sm = 1;
        unsigned grid = (unsigned)std::min<long long>(n_points, (long long)per_sm * s->sm_count);
        const DevCouplings *dc = reinterpret_cast<const DevCouplings *>(s->d_scan);
        double *dout = s->d_scan + in_doubles;
        // copy-in, the persistent launch and copy-out; with QS_OPT_GRAPH they are captured
        // once per shape as a CUDA graph and replayed (the copies read and write the
        // pinned staging buffer at replay time)
        auto enqueue = [&](cudaStream_t st) -> cudaError_t {
            cudaError_t e = cudaMemcpyAsync(s->d_scan, s->h_scan, in_doubles * sizeof(double),
                                            cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return e;
            if (s->dtype == QS_C64)
                k_scan12<float><<<grid, NT, 0, st>>>(dc, s->d_scan + 4 * n_points, dout, P);
            else
                k_scan12<double><<<grid, NT, 0, st>>>(dc, s->d_scan + 4 * n_points, dout, P);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            return cudaMemcpyAsync(s->h_scan + in_doubles, dout, out_doubles * sizeof(double),
                                   cudaMemcpyDeviceToHost, st);
        };
        if (s->use_graph) {
            const long long key[10] = {-1, n_points, n_steps, order, (long long)(uintptr_t)s->d_scan,
                                       (long long)(uintptr_t)s->h_scan, s->dtype, (long long)grid,
                                       (long long)llround(dt * 1e15), 0};
            if (!s->scan_graph || memcmp(key, s->scan_key, sizeof(key)) != 0) {
                if (s->scan_graph) { cudaGraphExecDestroy(s->scan_graph); s->scan_graph = nullptr; }
                if (!s->cap_stream) CK(s, cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
                CK(s, cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
                cudaError_t e1 = enqueue(s->cap_stream);
                cudaGraph_t g = nullptr;
                cudaError_t e2 = cudaStreamEndCapture(s->cap_stream, &g);
                if (e1 != cudaSuccess || e2 != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    FAIL(s, QS_ERR_CUDA, "scan graph capture: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
                }
                cudaError_t e3 = cudaGraphInstantiate(&s->scan_graph, g, 0);
                cudaGraphDestroy(g);
                if (e3 != cudaSuccess) { s->scan_graph = nullptr; FAIL(s, QS_ERR_CUDA, "scan graph: %s", cudaGetErrorString(e3)); }
                memcpy(s->scan_key, key, sizeof(key));
            }
            CK(s, cudaGraphLaunch(s->scan_graph, s->stream));
        } else {
            CK(s, enqueue(s->stream));
        }
        s->launches++;
        CK(s, cudaStreamSynchronize(s->stream));
        memcpy(out, s->h_scan + in_doubles, out_doubles * sizeof(double));
        return QS_OK;
    }
    // ---- larger lattices: chunks of `batch` points through the tiled passes ----
    qs_status st;
    if ((st = check_ready(s)) != QS_OK) return st;
    const int B = s->batch;
    std::vector<qs_couplings> chunk(B);
    std::vector<double> tmp(B);
    for (int p0 = 0; p0 < n_points; p0 += B) {
        const int cnt = std::min(B, n_points - p0);
        for (int b = 0; b < B; ++b) chunk[b] = points[p0 + std::min(b, cnt - 1)];
        if ((st = qs_init_plus(s)) != QS_OK) return st;
        if ((st = qs_evolve(s, chunk.data(), sv, dt, n_steps, order)) != QS_OK) return st;
        auto put = [&](int k, const double *v) {
            for (int b = 0; b < cnt; ++b) out[(size_t)(p0 + b) * SCAN_NOBS + k] = v[b];
        };
        if ((st = qs_expect(s, QS_ENERGY, 0, chunk.data(), 1.0, tmp.data())) != QS_OK) return st;
        put(0, tmp.data());
        if ((st = qs_expect(s, QS_PLAQUETTE, -1, nullptr, 1.0, tmp.data())) != QS_OK) return st;
        put(1, tmp.data());
        for (int w = 0; w < 2; ++w) {
            if (w < (int)s->lat.wilson.size()) {
                if ((st = qs_expect(s, QS_WILSON, w, nullptr, 1.0, tmp.data())) != QS_OK) return st;
            } else {
                std::fill(tmp.begin(), tmp.end(), 0.0);
            }
            put(2 + w, tmp.data());
        }
        if ((st = qs_expect(s, QS_NORM, 0, nullptr, 1.0, tmp.data())) != QS_OK) return st;
        put(4, tmp.data());
        // link / vertex <X> averages
        std::vector<double> xs(B, 0.0), xt(B, 0.0);
        for (int q = 0; q < s->n; ++q) {
            if ((st = qs_expect(s, QS_X, q, nullptr, 1.0, tmp.data())) != QS_OK) return st;
            for (int b = 0; b < B; ++b) (s->lat.x_class[q] ? xt : xs)[b] += tmp[b];
        }
        const int nl = s->lat.n_links, nv = s->n - s->lat.n_links;
        for (int b = 0; b < B; ++b) { xs[b] = nl ? xs[b] / nl : 0.0; xt[b] = nv ? xt[b] / nv : 0.0; }
        put(5, xs.data());
        put(6, xt.data());
        std::fill(tmp.begin(), tmp.end(), 0.0);
        put(7, tmp.data());
    }
    return QS_OK;
}

int qs_num_links(const qs_sim *s) { return s ? s->lat.n_links : -1; }

qs_status qs_dos(qs_sim *s, double *out) {
    qs_status st;
    if ((st = check_ready(s)) != QS_OK) return st;
    if (!out) FAIL(s, QS_ERR_ARG, "null output");
    const int nbins = s->lat.n_links + 1, B = s->batch;
    if (nbins > 64) FAIL(s, QS_ERR_ARG, "too many links");
    uint64_t linkmask = 0;
    for (int q = 0; q < s->n; ++q) if (!s->lat.x_class[q]) linkmask |= 1ull << q;
    const int G = 152 * 4;
    if ((st = grow(s, &s->d_adj_part, &s->adj_part_cap, (size_t)G * B * nbins + (size_t)B * nbins, false)) != QS_OK)
        return st;
    double *dout = s->d_adj_part + (size_t)G * B * nbins;
    if (s->dtype == QS_C64)
        k_dos<float><<<dim3(G, B), RED_THREADS, 0, s->stream>>>((const float2 *)s->state[0], s->n, s->dim, linkmask,
                                                                nbins, s->d_adj_part);
    else
        k_dos<double><<<dim3(G, B), RED_THREADS, 0, s->stream>>>((const double2 *)s->state[0], s->n, s->dim,
                                                                 linkmask, nbins, s->d_adj_part);
    CKL(s); s->launches++;
    k_finish_wide<<<B, 64, 0, s->stream>>>(s->d_adj_part, G, nbins, dout);
    CKL(s); s->launches++;
    CK(s, cudaMemcpyAsync(out, dout, (size_t)B * nbins * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    for (int i = 0; i < B * nbins; ++i)
        if (!std::isfinite(out[i])) FAIL(s, QS_ERR_NONFINITE, "non-finite density of states");
    return check_device_flag(s);
}

qs_status qs_scan_mixed(qs_sim *s12, const qs_couplings *p12, int n12, qs_sim *s, const qs_couplings *p17,
                        int n17, const double *sv, double dt, int n_steps, int order, double *out12, double *out17) {
    qs_status st;
    if (!s) return QS_ERR_ARG;
    if ((st = check_ready(s)) != QS_OK) return st;
    if (n12 < 0 || n17 < 0 || n12 + n17 < 1) FAIL(s, QS_ERR_ARG, "need at least one point");
    if (n_steps < 1) FAIL(s, QS_ERR_ARG, "n_steps must be >= 1");
    if (order != 1 && order != 2) FAIL(s, QS_ERR_ARG, "order must be 1 or 2");
    if (!sv || (n17 > 0 && (!p17 || !out17)) || (n12 > 0 && (!p12 || !out12 || !s12)))
        FAIL(s, QS_ERR_ARG, "null argument");
    if (s->lat.gauge_higgs || s->boundary != QS_OPEN || s->n <= LT || s->n > LT + 8 || s->dtype != QS_C64)
        FAIL(s, QS_ERR_ARG, "the mixed scan's second simulator must be an open unitary-gauge lattice of 13..20 "
                            "qubits in complex64");
    if (!s->tmaps_ok || s->passes.size() != 2) FAIL(s, QS_ERR_STATE, "no TMA pass plan over the bound state");
    if (n12 > 0 && (s12->n != LT || !s12->lat.gauge_higgs || s12->dtype != QS_C64 || s12->nA + s12->nB + 2 > 64))
        FAIL(s, QS_ERR_ARG, "the mixed scan's first simulator must be a 12-qubit gauge-Higgs lattice in complex64");
    const int nops = order == 2 ? n_steps + 1 : n_steps;
    const size_t in_doubles = 4 * (size_t)(n12 + n17) + (size_t)n_steps;
    const size_t out_doubles = (size_t)(n12 + n17) * SCAN_NOBS;
    if ((st = grow(s, &s->d_scan, &s->scan_cap, in_doubles + out_doubles, false)) != QS_OK) return st;
    if ((st = grow(s, &s->h_scan, &s->h_scan_cap, in_doubles + out_doubles, true)) != QS_OK) return st;
    if (!s->d_queue) CK(s, cudaMalloc((void **)&s->d_queue, sizeof(int)));
    auto put = [&](const qs_couplings *p, int n, double *dst) {
        for (int i = 0; i < n; ++i) {
            dst[4 * i] = p[i].J; dst[4 * i + 1] = p[i].h; dst[4 * i + 2] = p[i].g; dst[4 * i + 3] = p[i].lambda;
        }
    };
    put(p12, n12, s->h_scan);
    put(p17, n17, s->h_scan + 4 * (size_t)n12);
    memcpy(s->h_scan + 4 * (size_t)(n12 + n17), sv, (size_t)n_steps * sizeof(double));
    ScanParams P12;
    memset(&P12, 0, sizeof(P12));
    if (n12 > 0) P12 = scan12_params(s12, n12, n_steps, order, dt);
    P12.n_points = n12;
    ScanUGParams U;
    memset(&U, 0, sizeof(U));
    U.n_points = n17; U.n_ops = nops;
    U.G.n_steps = n_steps; U.G.order = order; U.G.fsal = order == 2; U.G.batch = 1; U.G.dt = dt; U.G.f32 = 1;
    U.n = s->n; U.nP = s->nA; U.nL = s->nB; U.nS = s->nXA;
    U.tiles_shift = s->n - LT;
    U.scale = (float)ldexp(1.0, -s->n);
    U.p0 = s->tpasses[NVAR * 0 + V_HAD_Z];
    U.p1 = s->tpasses[NVAR * 1 + V_HAD_X];
    // tile buffers of the 17-qubit passes: 2 or 3 (two CTAs per SM; 3, the default, measured
    // fastest with 2 x SMs scratch slots) or 4 or 6 (one CTA per SM)
    const int nb = s->scan_buffers;
    typedef void (*MixKernel)(const DevCouplings *, const DevCouplings *, const double *, double *, double *, int *,
                              int *, const CUtensorMap, const CUtensorMap, const ScanParams, const ScanUGParams);
    const MixKernel kern = nb == 2 ? k_scan_mixed<2> : nb == 3 ? k_scan_mixed<3> : nb == 4 ? k_scan_mixed<4>
                                                                                              : k_scan_mixed<6>;
    const size_t smem = (size_t)nb * TMA_TILE_BYTES + 1024;
    CK(s, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (per_sm < 1) per_sm = 1;
    long long g = std::min<long long>((long long)per_sm * s->sm_count, n12 + n17);
    if (n17 > 0) g = std::min<long long>(g, s->batch);   // one scratch slot per CTA
    const unsigned grid = (unsigned)g;
    const DevCouplings *c12 = reinterpret_cast<const DevCouplings *>(s->d_scan);
    const DevCouplings *c17 = c12 + n12;
    const double *dsv = s->d_scan + 4 * (size_t)(n12 + n17);
    double *dout12 = s->d_scan + in_doubles, *dout17 = dout12 + (size_t)n12 * SCAN_NOBS;
    auto enqueue = [&](cudaStream_t q) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(s->d_scan, s->h_scan, in_doubles * sizeof(double), cudaMemcpyHostToDevice, q);
        if (e != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(s->d_queue, 0, sizeof(int), q)) != cudaSuccess) return e;
        kern<<<grid, NT, smem, q>>>(c12, c17, dsv, dout12, dout17, s->d_queue, s->d_err, s->tmaps[0], s->tmaps[1],
                                     P12, U);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        return cudaMemcpyAsync(s->h_scan + in_doubles, dout12, out_doubles * sizeof(double), cudaMemcpyDeviceToHost,
                               q);
    };
    if (s->use_graph) {
        const long long key[10] = {-2 - 16 * nb, n12, n17, n_steps, order, (long long)(uintptr_t)s->d_scan,
                                   (long long)(uintptr_t)s->h_scan, (long long)grid,
                                   (long long)llround(dt * 1e15), (long long)(uintptr_t)s->state[0]};
        if (!s->scan_graph || memcmp(key, s->scan_key, sizeof(key)) != 0) {
            if (s->scan_graph) { cudaGraphExecDestroy(s->scan_graph); s->scan_graph = nullptr; }
            if (!s->cap_stream) CK(s, cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
            CK(s, cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e1 = enqueue(s->cap_stream);
            cudaGraph_t gr = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(s->cap_stream, &gr);
            if (e1 != cudaSuccess || e2 != cudaSuccess) {
                if (gr) cudaGraphDestroy(gr);
                FAIL(s, QS_ERR_CUDA, "scan graph capture: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
            }
            cudaError_t e3 = cudaGraphInstantiate(&s->scan_graph, gr, 0);
            cudaGraphDestroy(gr);
            if (e3 != cudaSuccess) { s->scan_graph = nullptr; FAIL(s, QS_ERR_CUDA, "scan graph: %s", cudaGetErrorString(e3)); }
            memcpy(s->scan_key, key, sizeof(key));
        }
        CK(s, cudaGraphLaunch(s->scan_graph, s->stream));
    } else {
        CK(s, enqueue(s->stream));
    }
    s->launches++;
    CK(s, cudaStreamSynchronize(s->stream));
    if ((st = check_device_flag(s)) != QS_OK) return st;
    if (n12 > 0) memcpy(out12, s->h_scan + in_doubles, (size_t)n12 * SCAN_NOBS * sizeof(double));
    if (n17 > 0) memcpy(out17, s->h_scan + in_doubles + (size_t)n12 * SCAN_NOBS, (size_t)n17 * SCAN_NOBS * sizeof(double));
    return QS_OK;
}

qs_status qs_autotune(qs_sim *s, int n_steps, int *best_xpass, int *best_buffers, int *best_store,
                      int *best_shared_buffers, int *best_shared_kernel, double *best_ms_per_step) {
    qs_status st;
    if ((st = check_ready(s)) != QS_OK) return st;
    if (n_steps < 1 || n_steps > 1000) FAIL(s, QS_ERR_ARG, "n_steps must be in [1, 1000]");
    if (!best_xpass || !best_buffers || !best_store || !best_shared_buffers || !best_shared_kernel ||
        !best_ms_per_step)
        FAIL(s, QS_ERR_ARG, "null output");
    struct Cand { int xpass, nbuf, store, nsh, skern; };
    std::vector<Cand> cands;
    if (s->dtype == QS_C64 && s->tmaps_ok) {
        for (int nb = 2; nb <= 3; ++nb)
            for (int so = 0; so <= 1; ++so)
                for (int ns = 2; ns <= 3; ++ns) cands.push_back({2, nb, so, ns, 0});
        // warp-local shared passes (bulk stores only)
        for (int nb = 2; nb <= 3; ++nb)
            for (int ns : {0, 2, 3}) cands.push_back({2, nb, 1, ns, 1});
    }
    cands.push_back({1, 2, 0, 0, 0});
    const int saved_method = s->method, saved_profile = s->profile, saved_graph = s->use_graph;
    s->method = 0; s->profile = 0; s->use_graph = 0;
    std::vector<qs_couplings> c(s->batch, qs_couplings{1.0, 1.0, 0.6, 0.6});
    std::vector<double> sv(n_steps + 2);
    for (int k = 0; k < n_steps + 2; ++k) sv[k] = (k + 0.5) / (n_steps + 2);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(s, cudaEventCreate(&e0));
    CK(s, cudaEventCreate(&e1));
    double best = 1e300;
    Cand pick = cands.back();
    for (const Cand &cd : cands) {
        s->xpass_impl = cd.xpass; s->nbuf = cd.nbuf; s->tma_store = cd.store; s->nbuf_shared = cd.nsh;
        s->shared_kernel = cd.skern;
        if ((st = qs_init_plus(s)) != QS_OK) break;
        if ((st = qs_evolve(s, c.data(), sv.data(), 0.02, 2, 2)) != QS_OK) break;   // warm-up
        CK(s, cudaEventRecord(e0, s->stream));
        if ((st = qs_evolve(s, c.data(), sv.data() + 2, 0.02, n_steps, 2)) != QS_OK) break;
        CK(s, cudaEventRecord(e1, s->stream));
        CK(s, cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(s, cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) { best = ms; pick = cd; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->method = saved_method; s->profile = saved_profile; s->use_graph = saved_graph;
    if (st != QS_OK) return st;
    s->xpass_impl = pick.xpass; s->nbuf = pick.nbuf; s->tma_store = pick.store; s->nbuf_shared = pick.nsh;
    s->shared_kernel = pick.skern;
    *best_xpass = pick.xpass; *best_buffers = pick.nbuf; *best_store = pick.store;
    *best_shared_buffers = pick.nsh;
    *best_shared_kernel = pick.skern;
    *best_ms_per_step = best / n_steps;
    return QS_OK;
}

int qs_plan(const qs_sim *s, int *qubits_per_pass, int max) {
    if (!s || max < 0 || (max > 0 && !qubits_per_pass)) return -1;
    const int np = (int)s->pass_q.size();
    if (max < np) return -1;
    for (int p = 0; p < np; ++p) qubits_per_pass[p] = s->pass_q[p];
    return np;
}

qs_status qs_autotune_plan(qs_sim *s, int n_steps, int *qubits_per_pass, int max, int *n_passes,
                           double *best_ms_per_step) {
    qs_status st;
    if ((st = check_ready(s)) != QS_OK) return st;
    if (n_steps < 1 || n_steps > 1000) FAIL(s, QS_ERR_ARG, "n_steps must be in [1, 1000]");
    if (!qubits_per_pass || !n_passes || !best_ms_per_step) FAIL(s, QS_ERR_ARG, "null output");
    if (s->n <= LT) FAIL(s, QS_ERR_ARG, "a pass plan needs more than %d qubits", LT);
    const int r = s->n - LT, P = (r + 7) / 8;
    if (max < P + 1) FAIL(s, QS_ERR_ARG, "qubits_per_pass needs %d entries", P + 1);
    // every composition of r into P parts, each part in [lo, 8] (lo = 4 when possible)
    const int lo = std::max(1, std::min(4, r / P));
    std::vector<std::vector<int>> plans;
    std::vector<int> cur;
    std::function<void(int, int)> rec = [&](int left, int parts) {
        if (parts == 0) { if (left == 0) plans.push_back(cur); return; }
        for (int x = lo; x <= 8 && x <= left; ++x) {
            cur.push_back(x);
            rec(left - x, parts - 1);
            cur.pop_back();
        }
    };
    rec(r, P);
    if (plans.empty()) FAIL(s, QS_ERR_STATE, "no pass plan");
    const std::vector<int> saved_k = s->plan_k;
    const long long saved_code = s->plan_code;
    const int saved_method = s->method, saved_profile = s->profile, saved_graph = s->use_graph;
    s->method = 0; s->profile = 0; s->use_graph = 0;
    std::vector<qs_couplings> c(s->batch, qs_couplings{1.0, 1.0, 0.6, 0.6});
    std::vector<double> sv(n_steps + 2);
    for (int k = 0; k < n_steps + 2; ++k) sv[k] = (k + 0.5) / (n_steps + 2);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(s, cudaEventCreate(&e0));
    CK(s, cudaEventCreate(&e1));
    double best = 1e300;
    size_t pick = 0;
    for (size_t i = 0; i < plans.size() && st == QS_OK; ++i) {
        s->plan_k = plans[i];
        if ((st = rebuild_plan(s)) != QS_OK) break;
        if ((st = qs_init_plus(s)) != QS_OK) break;
        if ((st = qs_evolve(s, c.data(), sv.data(), 0.02, 2, 2)) != QS_OK) break;   // warm-up
        if (cudaEventRecord(e0, s->stream) != cudaSuccess) { st = QS_ERR_CUDA; break; }
        if ((st = qs_evolve(s, c.data(), sv.data() + 2, 0.02, n_steps, 2)) != QS_OK) break;
        if (cudaEventRecord(e1, s->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            st = QS_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; pick = i; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->method = saved_method; s->profile = saved_profile; s->use_graph = saved_graph;
    if (st != QS_OK) {
        s->plan_k = saved_k;
        s->plan_code = saved_code;
        rebuild_plan(s);
        return st;
    }
    s->plan_k = plans[pick];
    s->plan_code = 0;
    for (size_t j = 0; j < plans[pick].size(); ++j) s->plan_code |= (long long)plans[pick][j] << (4 * j);
    if ((st = rebuild_plan(s)) != QS_OK) return st;
    *n_passes = qs_plan(s, qubits_per_pass, max);
    *best_ms_per_step = best / n_steps;
    return QS_OK;
}

qs_status qs_selftest_wait(qs_sim *s, double limit_ms) {
    if (!s) return QS_ERR_ARG;
    if (!(limit_ms > 0.0 && limit_ms <= 2000.0)) FAIL(s, QS_ERR_ARG, "limit_ms must be in (0, 2000]");
    int dev = 0, khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    if (khz <= 0) khz = 2000000;
    long long cycles = (long long)(limit_ms * (double)khz);
    k_wait_probe<<<1, 32, 0, s->stream>>>(s->d_err, cycles);
    CKL(s); s->launches++;
    CK(s, cudaStreamSynchronize(s->stream));
    return check_device_flag(s);
}

// ---- checkpoint: header + raw state ----
namespace {
struct CkptHeader {
    char magic[8];        // "QSIMCKP1"
    int32_t Lx, Ly, boundary, form, dtype, batch, n;
    int32_t reserved;
    uint64_t state_bytes;
};
}

qs_status qs_save(qs_sim *s, const char *path) {
    qs_status st;
    if ((st = check_ready(s)) != QS_OK) return st;
    if (!path) FAIL(s, QS_ERR_ARG, "null path");
    const size_t bytes = qs_state_bytes(s);
    void *host = nullptr;
    if (cudaMallocHost(&host, bytes) != cudaSuccess) FAIL(s, QS_ERR_OOM, "pinned staging of %zu bytes", bytes);
    st = qs_download_state(s, host, bytes);
    if (st == QS_OK) {
        FILE *f = fopen(path, "wb");
        if (!f) { cudaFreeHost(host); FAIL(s, QS_ERR_ARG, "cannot open %s for writing", path); }
        CkptHeader h;
        memset(&h, 0, sizeof(h));
        memcpy(h.magic, "QSIMCKP1", 8);
        h.Lx = s->lat.Lx; h.Ly = s->lat.Ly; h.boundary = s->boundary; h.form = s->form;
        h.dtype = s->dtype; h.batch = s->batch; h.n = s->n; h.state_bytes = bytes;
        bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(host, 1, bytes, f) == bytes;
        ok = (fclose(f) == 0) && ok;
        if (!ok) { cudaFreeHost(host); FAIL(s, QS_ERR_ARG, "short write to %s", path); }
    }
    cudaFreeHost(host);
    return st;
}

qs_status qs_load(qs_sim *s, const char *path) {
    qs_status st;
    if ((st = check_ready(s)) != QS_OK) return st;
    if (!path) FAIL(s, QS_ERR_ARG, "null path");
    FILE *f = fopen(path, "rb");
    if (!f) FAIL(s, QS_ERR_ARG, "cannot open %s", path);
    CkptHeader h;
    if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, "QSIMCKP1", 8) != 0) {
        fclose(f);
        FAIL(s, QS_ERR_ARG, "%s is not a qsim checkpoint", path);
    }
    const size_t bytes = qs_state_bytes(s);
    if (h.Lx != s->lat.Lx || h.Ly != s->lat.Ly || h.boundary != s->boundary || h.form != s->form ||
        h.dtype != s->dtype || h.batch != s->batch || h.n != s->n || h.state_bytes != bytes) {
        fclose(f);
        FAIL(s, QS_ERR_ARG, "checkpoint %s was written for another lattice, dtype or batch", path);
    }
    void *host = nullptr;
    if (cudaMallocHost(&host, bytes) != cudaSuccess) { fclose(f); FAIL(s, QS_ERR_OOM, "pinned staging"); }
    bool ok = fread(host, 1, bytes, f) == bytes;
    fclose(f);
    if (!ok) { cudaFreeHost(host); FAIL(s, QS_ERR_ARG, "truncated checkpoint %s", path); }
    st = qs_upload_state(s, host, bytes);
    cudaFreeHost(host);
    return st;
}

qs_status qs_sync(qs_sim *s) {
    if (!s) return QS_ERR_ARG;
    CK(s, cudaStreamSynchronize(s->stream));
    CK(s, cudaGetLastError());
    return check_device_flag(s);
}

qs_status qs_profile_read_kinds(qs_sim *s, double *total_ms, long long *count) {
    if (!s || !total_ms || !count) return QS_ERR_ARG;
    CK(s, cudaStreamSynchronize(s->stream));
    double t[2] = {0.0, 0.0};
    long long c[2] = {0, 0};
    for (size_t i = 0; i + 1 < s->ev_used; i += 2) {
        float ms = 0.f;
        CK(s, cudaEventElapsedTime(&ms, s->ev_pool[i], s->ev_pool[i + 1]));
        const int kd = s->ev_kind[i / 2];
        t[kd] += ms;
        c[kd] += 1;
    }
    for (int kd = 0; kd < 2; ++kd) { total_ms[kd] = t[kd]; count[kd] = c[kd]; }
    s->ev_used = 0;
    s->ev_kind.clear();
    return QS_OK;
}

qs_status qs_profile_read(qs_sim *s, double *total_ms, long long *count) {
    if (!s || !total_ms || !count) return QS_ERR_ARG;
    double t[2];
    long long c[2];
    qs_status st = qs_profile_read_kinds(s, t, c);
    if (st != QS_OK) return st;
    *total_ms = t[0] + t[1];
    *count = c[0] + c[1];
    return QS_OK;
}

long long qs_launch_count(qs_sim *s) {
    if (!s) return -1;
    long long v = s->launches;
    s->launches = 0;
    return v;
}

}  // extern "C"
