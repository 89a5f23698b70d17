/*
 * qsim.h -- C ABI of the GB300 state-vector engine for the Trotterised adiabatic
 * evolution of the Z2 gauge-Higgs model (Ding, Cui, Shi, "Digital quantum
 * simulation and pseudoquantum simulation of the Z2 gauge-Higgs model").
 *
 * Model (Sec. II).  Gauge-Higgs form, Eq. (1):
 *     H1 = -J sum_v tau^x_v - h sum_p B_p - g sum_l sigma^x_l
 *          - lambda sum_<jk> tau^z_j sigma^z_<jk> tau^z_k,   B_p = prod_{l in p} sigma^z_l.
 * Unitary-gauge (toric code in two transverse fields) form, Eq. (4):
 *     H1 = -J sum_v A_v - h sum_p B_p - g sum_l sigma^x_l - lambda sum_l sigma^z_l,
 *     A_v = prod_{l at v} sigma^x_l.
 * Adiabatic path (Sec. III): H(s) = (1 - s) H0 + s H1 with H0 = -sum of the X-type
 * fields (-sum sigma^x - sum tau^x, or -sum sigma^x - sum A_v), ground state |+>^n.
 * Trotter product (Eq. (7), Eq. (8)), operators acting right to left:
 *     order 1:  U = exp(-i dt H_Z) exp(-i dt H_X)
 *     order 2:  U = exp(-i dt/2 H_X) exp(-i dt H_Z) exp(-i dt/2 H_X)
 * where H_X collects sigma^x, tau^x, A_v and H_Z collects B_p, the bonds and sigma^z.
 *
 * Qubit numbering (periodic Lx x Ly torus, N = Lx*Ly vertices, v = y*Lx + x):
 *     horizontal link (x,y)->(x+1,y): qubit v;  vertical link (x,y)->(x,y+1): N + v;
 *     vertex tau_v (gauge-Higgs only): 2N + v.
 * Open boundary: Lx x Ly plaquettes, (Lx+1) x (Ly+1) vertices; the existing
 * horizontal links in vertex order, then the vertical links, then the vertices.
 * Plaquette (x,y) = {h(x,y), h(x,y+1), u(x,y), u(x+1,y)}; star A_v = the existing
 * links among {h(x,y), h(x-1,y), u(x,y), u(x,y-1)}.  Bit value 0 is Z = +1.
 *
 * State layout.  `batch` state vectors of 2^n amplitudes, back to back; amplitude
 * i of state b at element b * 2^n + i, stored as interleaved (re, im) float
 * (QS_C64) or double (QS_C128).  State memory is allocated by the caller (e.g.
 * PyTorch) and borrowed through qs_bind_state; the library never frees it.
 *
 * Conventions.  Every call returns a qs_status; on error no output is written
 * and qs_last_error() describes the failure.  Host pointers belong to the
 * caller.  All device work is stream-ordered on the stream given to
 * qs_set_stream (default: the legacy default stream).  Calls that return host
 * scalars synchronise that stream.  A qs_sim is not thread-safe.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qs_sim qs_sim;

typedef enum {
    QS_OK = 0,
    QS_ERR_ARG = 1,        /* invalid argument (null pointer, size, index, range) */
    QS_ERR_OOM = 2,        /* library workspace allocation failed */
    QS_ERR_CUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    QS_ERR_NONFINITE = 4,  /* a reduction produced NaN/Inf (e.g. a poisoned state) */
    QS_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up */
    QS_ERR_STATE = 6       /* call out of order (e.g. no state bound) */
} qs_status;

typedef enum { QS_PERIODIC = 0, QS_OPEN = 1 } qs_boundary;
typedef enum { QS_GAUGE_HIGGS = 0, QS_UNITARY_GAUGE = 1 } qs_form;
typedef enum { QS_C64 = 0, QS_C128 = 1 } qs_dtype;

/* Observables for qs_expect (Sec. II, Sec. IV). */
typedef enum {
    QS_NORM = 0,       /* <psi|psi>                                                  */
    QS_PLAQUETTE = 1,  /* <B_p>, index = p; index = -1: average over all plaquettes  */
    QS_WILSON = 2,     /* non-contractible Wilson loop: index 0 = W_x (links h(x,0)),
                          index 1 = W_y (links u(0,y)); periodic lattices only       */
    QS_X = 3,          /* <X_q>, index = qubit q                                      */
    QS_ENERGY = 4,     /* <H1> with the given couplings (s ignored)                   */
    QS_ENERGY_S = 5,   /* <H(s)> = (1-s)<H0> + s<H1>                                  */
    QS_GAUSS = 6,      /* <Q_v> = <tau^x_v A_v>, index = v (gauge-Higgs form only)    */
    QS_THOOFT = 7      /* 't Hooft loop: index 0 = prod_y X_h(0,y), 1 = prod_x X_u(x,0) */
} qs_obs;

/* Couplings of H1 (Eq. (1) / Eq. (4)); one record per batch element. */
typedef struct { double J, h, g, lambda; } qs_couplings;

/* Options for qs_set_option. */
typedef enum {
    QS_OPT_METHOD = 0,        /* 0: fused kernels (default); 1: one launch per Pauli
                                 term (the plain per-gate form)                      */
    QS_OPT_RENORM_EVERY = 1,  /* qs_evolve rescales the state to unit FP64 norm every
                                 this many steps and at the end (0 = never; default 0) */
    QS_OPT_PROFILE = 2,       /* 1: time every fused X-pass launch with CUDA events on
                                 the bound stream (read with qs_profile_read)        */
    QS_OPT_GRAPH = 3,         /* 1: qs_evolve replays its launches as a CUDA graph    */
    QS_OPT_XPASS = 4,         /* X-pass kernel for complex64: 0 auto (TMA), 1 the
                                 register-staged kernel, 2 the persistent TMA kernel */
    QS_OPT_TMA_BUFFERS = 5,   /* shared-memory tile buffers per CTA of the TMA kernel:
                                 2 (three CTAs per SM) or 3 (default; two CTAs per SM) */
    QS_OPT_ADJOINT = 6,       /* complex64 adjoint reverse pass: bit 0 set = register-
                                 staged kernel, clear = TMA kernel (default).  TMA
                                 kernel, 0 (default): one psi/lambda tile-pair buffer
                                 (two CTAs per SM), the next pair's load issued as soon
                                 as the current pair's last stage is read, stores from
                                 registers (tangent form); bit 1 set: two buffers (one
                                 CTA per SM); bit 2 set: one buffer, load issued at the
                                 start of each pair, bulk tensor stores              */
    QS_OPT_TMA_STORE = 7,     /* 1 (default): the TMA X pass writes each tile back with
                                 one bulk tensor store; 0: per-thread stores         */
    QS_OPT_XMERGE = 8,        /* 1 (default): complex64 runs on the TMA kernel share
                                 passes.  Gauge-Higgs: consecutive Trotter factor groups
                                 share the pass of one qubit group (X of group k, the Z
                                 layer of k, X of group k+1 on the same qubits; exact
                                 because all X-type factors commute), one pass fewer
                                 per step.  Unitary gauge: one pass applies H D_X H on
                                 one qubit group and one applies H, the Z layer and the
                                 next group's H, two passes fewer per step.  0: every
                                 factor group takes all its passes                    */
    QS_OPT_PDL = 9,           /* 1 (default): the TMA X passes are launched with
                                 programmatic stream serialisation, so a pass is
                                 scheduled and sets up while the previous kernel
                                 drains and waits for its writes before reading
                                 global memory; 0: plain stream order             */
    QS_OPT_SHARED_BUFFERS = 10, /* tile buffers per CTA of the shared X passes
                                 (QS_OPT_XMERGE): 2 (three CTAs per SM), 3 (two CTAs
                                 per SM) or 0 (default).  CTA-staged kernel: 0 is 2
                                 for tangent-form rotations (gauge-Higgs), 3 for
                                 Walsh-Hadamard passes (unitary gauge), the faster of
                                 the two for each as measured.  Warp-local kernel
                                 (QS_OPT_SHARED_KERNEL): 0 is one CTA of 24 warps per
                                 SM with six buffers; 2 and 3 use CTAs of 8 warps */
    QS_OPT_PLAN = 11,         /* pass plan of the tiled X layer: how many new qubits
                                 each pass after the first fuses (the first pass always
                                 takes qubits 0..11).  Value: one 4-bit field per pass,
                                 lowest first, each in [1, 8], summing to n - 12 (a pass
                                 fusing k new qubits keeps a contiguous chunk of 12 - k
                                 low qubits, 2^(12-k) amplitudes per row); 0 (default):
                                 8 per pass, the remainder last.  Rejected (QS_ERR_ARG)
                                 for states of fewer than 13 qubits.                  */
    QS_OPT_SCAN_BUFFERS = 12, /* qs_scan_mixed: 32 KB tile buffers per CTA of the
                                 larger lattice's passes, 2 or 3 (two CTAs per SM) or 4
                                 or 6 (one CTA per SM; a pass keeps buffers - 1 loads in
                                 flight); 0: the default, 3 (with one scratch slot
                                 per CTA, 2 x SMs slots, measured fastest)            */
    QS_OPT_SHARED_KERNEL = 13,/* shared X passes (QS_OPT_XMERGE; both forms) and shared
                                 reverse passes of the complex64 adjoint: 1 (default):
                                 warp-local slices where the pass allows them (its
                                 rotated qubits on tile bits 4..11, one state, bulk
                                 stores): each consumer warp takes 512-amplitude
                                 slices of a tile through both rounds with warp-level
                                 synchronisation only, one thread issues the TMA
                                 copies over pooled tile buffers; 0: the CTA-staged
                                 kernels                                              */
    QS_OPT_C128_DF = 14       /* complex128, unitary gauge, fused kernels: 1 (default):
                                 the Walsh-Hadamard passes run in double-float
                                 arithmetic (each real number an unevaluated sum of two
                                 floats, 48 significand bits, on the FP32 pipes; the
                                 state is converted in place to a blocked layout at the
                                 start of a call and back at its end); 0: FP64
                                 register-staged passes                               */
} qs_option;

/* Create a simulator for an Lx x Ly lattice.  Periodic needs Lx, Ly >= 2; open
 * needs Lx, Ly >= 1.  batch >= 1 independent states share the lattice; each has
 * its own couplings.  Fails with QS_ERR_ARG if the qubit count exceeds 34.
 * Allocates only small device workspaces (term tables, partial sums). */
qs_status qs_create(int Lx, int Ly, int boundary, int form, int dtype, int batch,
                    qs_sim **out);
void qs_destroy(qs_sim *sim);
/* Last error message of sim (or of the last failed qs_create when sim is NULL). */
const char *qs_last_error(const qs_sim *sim);

int qs_num_qubits(const qs_sim *sim);
/* Bytes of all batch states (batch * 2^n * 8 or 16). */
size_t qs_state_bytes(const qs_sim *sim);

/* Borrow device memory: slot 0 = the evolved state psi, slot 1 = the adjoint
 * work state (qs_adjoint_grad).  bytes must be >= qs_state_bytes and dev_ptr
 * 256-byte aligned. */
qs_status qs_bind_state(qs_sim *sim, int slot, void *dev_ptr, size_t bytes);
/* cudaStream_t passed as void*; NULL = legacy default stream. */
qs_status qs_set_stream(qs_sim *sim, void *stream);
qs_status qs_set_option(qs_sim *sim, int key, long long value);

/* psi <- |+>^n for every batch element (ground state of H0). */
qs_status qs_init_plus(qs_sim *sim);
/* Toric-code ground states of Sec. IV (unitary-gauge form only), normalised in FP64:
 * which = 0: psi_1, the projection of |+>^n onto B_p = +1 for every plaquette (Eq. (14));
 * which = 1: psi_1', the projection of |0...0> onto A_v = +1 for every vertex (Eq. (15)),
 * i.e. the uniform superposition over the star-flip orbit of |0...0> (on a torus: B_p = +1
 * and both non-contractible Wilson loops +1). */
qs_status qs_init_toric(qs_sim *sim, int which);
/* Copy batch states between host memory (pinned for asynchronous transfer) and
 * the bound state; bytes must equal qs_state_bytes.  Synchronises the stream. */
qs_status qs_upload_state(qs_sim *sim, const void *host, size_t bytes);
qs_status qs_download_state(qs_sim *sim, void *host, size_t bytes);

/* One Trotter step of H(s) over time dt (order 1 or 2), couplings[batch]. */
qs_status qs_trotter_step(qs_sim *sim, const qs_couplings *couplings, double s,
                          double dt, int order);

/* n_steps Trotter steps with s[k] (host array, the schedule at the midpoint of
 * step k).  Second order merges the adjacent X half-steps of consecutive steps
 * (the X-type terms commute), which leaves the product unchanged. */
qs_status qs_evolve(qs_sim *sim, const qs_couplings *couplings, const double *s,
                    double dt, int n_steps, int order);

/* Parameter path (Sec. III): n_steps Trotter steps of H1 with couplings that change
 * from step to step, per_step[k * batch + b] for step k (no interpolation with H0,
 * i.e. s = 1).  Otherwise as qs_evolve. */
qs_status qs_evolve_path(qs_sim *sim, const qs_couplings *per_step, double dt, int n_steps,
                         int order);

/* Expectation value per batch element, accumulated in FP64 (out: host [batch]).
 * couplings and s are used by QS_ENERGY / QS_ENERGY_S only (may be NULL else). */
qs_status qs_expect(qs_sim *sim, int kind, int index, const qs_couplings *couplings,
                    double s, double *out);
/* <psi|P|psi> for a Pauli string of one type: type 0 = Z string, 1 = X string,
 * on the qubits set in mask (out: host [batch]). */
qs_status qs_expect_pauli(qs_sim *sim, int type, uint64_t mask, double *out);
/* |<phi|psi>|^2 per batch element; ref_dev_state has the layout of the bound
 * state (same dtype, batch and size). out: host [batch]. */
qs_status qs_fidelity(qs_sim *sim, const void *ref_dev_state, double *out);

/* Reverse-mode gradient of a scalar of the final state with respect to the
 * schedule.  Runs n_steps Trotter steps from the currently bound state psi_0 (as
 * qs_evolve with the fused kernels), evaluates the value V (target 0: the final
 * energy <psi_N|H1|psi_N>; target 1: the fidelity |<phi|psi_N>|^2 with phi =
 * ref_dev_state, same layout as the bound state), then walks the Trotter factors in
 * reverse, uncomputing psi and propagating lambda = dV/d<psi_N| with inverse
 * factors (no stored intermediate states), and accumulates in FP64
 *     dV/dtheta = 2 Re <lambda| i P |psi>
 * for every factor exp(i theta P) of Eq. (8), chained to dV/ds_k.
 * Outputs (host): dV_ds[b * n_steps + k], value_out[b].  On return slot 0 holds the
 * reconstructed psi_0 (up to rounding) and slot 1 (which must be bound) is
 * overwritten.  Gauge-Higgs form, at least 12 qubits.  Synchronises the stream. */
qs_status qs_adjoint_grad(qs_sim *sim, const qs_couplings *couplings, const double *s, double dt,
                          int n_steps, int order, int target, const void *ref_dev_state,
                          double *dV_ds, double *value_out);

/* Observables returned per point by qs_scan. */
#define QS_SCAN_NOBS 8

/* Phase-diagram scan (Sec. V: energies along many parameter points).  Each of
 * n_points coupling records is an independent run from |+>^n through the same
 * schedule s[n_steps] (order 1 or 2, dt), with FP64 observables written to
 * out[p * QS_SCAN_NOBS + k]: k = 0 <H1>, 1 average <B_p>, 2 <W_x>, 3 <W_y>
 * (0 on open lattices), 4 norm, 5 average <sigma^x_l>, 6 average <tau^x_v>
 * (0 in the unitary gauge), 7 reserved (0).
 * A 12-qubit gauge-Higgs lattice (2x2 torus) runs every point in one persistent
 * launch with the state in shared memory; sim needs no bound state.  Other
 * lattices run in chunks of `batch` points through the tiled passes on the bound
 * state (slot 0), which is overwritten.  Synchronises the stream. */
qs_status qs_scan(qs_sim *sim, const qs_couplings *points, int n_points, const double *s, double dt,
                  int n_steps, int order, double *out);

/* Synchronise the bound stream and report device-side failures: QS_ERR_CUDA for
 * a failed launch, QS_ERR_TIMEOUT if a bounded wait inside a kernel gave up. */
qs_status qs_sync(qs_sim *sim);

/* Number of link (sigma) qubits of the lattice. */
int qs_num_links(const qs_sim *sim);

/* Density of states of Z~ = -sum_l sigma^z_l (Sec. V, the DOS analysis): for each
 * batch element, out[b * (n_links + 1) + k] = sum of |psi_i|^2 over the amplitudes
 * with exactly k links in sigma^z = -1, i.e. the weight of the Z~ eigenvalue
 * 2k - n_links.  FP64, host output; synchronises the stream. */
qs_status qs_dos(qs_sim *sim, double *out);

/* Autotuner: times n_steps second-order steps of every X-pass configuration that
 * applies (complex64: the persistent TMA kernel with 2 or 3 tile buffers for plain and
 * for shared passes and either store mode, the warp-local shared passes with 2 or 3
 * buffers, and the register-staged kernel; complex128: the register-staged kernel) on
 * the bound state, which is overwritten, and keeps the fastest (QS_OPT_XPASS,
 * QS_OPT_TMA_BUFFERS, QS_OPT_TMA_STORE, QS_OPT_SHARED_BUFFERS, QS_OPT_SHARED_KERNEL).
 * Outputs the choice and its ms per step (host). */
qs_status qs_autotune(qs_sim *sim, int n_steps, int *best_xpass, int *best_buffers, int *best_store,
                      int *best_shared_buffers, int *best_shared_kernel, double *best_ms_per_step);

/* Phase-diagram scan of two lattices in one persistent launch (Sec. V: the phase diagram
 * is mapped by independent adiabatic runs, Sec. III, at many coupling points).  sim12: a
 * 12-qubit gauge-Higgs lattice (the 2x2 torus), complex64; sim: an open unitary-gauge
 * lattice of 13..20 qubits (the 3x2 open lattice has 17), complex64, whose bound state
 * (slot 0, `batch` states) is the scratch: one state slot per CTA, so at most `batch`
 * CTAs run.  For each of the n12 points p12[i] (sim12's lattice) and n17 points p17[i]
 * (sim's lattice): |+>^n evolved over the schedule s[0 .. n_steps-1] (step midpoints),
 * time step dt, Trotter order 1 or 2, then the observables of qs_scan into out12[i * 8 +
 * k] and out17[i * 8 + k] (host; energy <H1>, mean <B_p>, W_x, W_y, norm, mean <X> on
 * links, mean <X> on vertices, 0).  CTAs take points from a work queue; a 12-qubit point
 * runs in shared memory, a larger one on the CTA's scratch slot as two TMA-pipelined
 * Walsh-Hadamard passes per Trotter factor group.  The bound state is overwritten.  With
 * QS_OPT_GRAPH set on sim the copies and the launch are captured once per shape as a CUDA
 * graph and replayed.  Stream-ordered on sim's stream, synchronises it.  Errors:
 * QS_ERR_ARG (lattices, dtypes, counts, null pointers), QS_ERR_STATE (no bound state),
 * QS_ERR_TIMEOUT (a bounded wait gave up), QS_ERR_CUDA. */
qs_status qs_scan_mixed(qs_sim *sim12, const qs_couplings *p12, int n12, qs_sim *sim, const qs_couplings *p17,
                        int n17, const double *s, double dt, int n_steps, int order, double *out12,
                        double *out17);

/* Pass-plan autotuner (the fusion width of the tiled X layer): times n_steps
 * second-order steps with every plan of the fewest passes whose passes each fuse 4 to 8
 * new qubits (rows of 128 B to 2 KB), on the bound state, which is overwritten, and keeps
 * the fastest (QS_OPT_PLAN).  Writes the qubits fused by each pass (the first pass 12)
 * to qubits_per_pass[0 .. *n_passes - 1] (host, at most max entries) and the best ms per
 * step.  QS_ERR_ARG for fewer than 13 qubits or max too small. */
qs_status qs_autotune_plan(qs_sim *sim, int n_steps, int *qubits_per_pass, int max, int *n_passes,
                           double *best_ms_per_step);

/* The current pass plan: qubits fused by each tiled X pass (the first 12), host output of
 * at most max entries; returns the number of passes (0 for states smaller than one tile,
 * -1 on a bad argument). */
int qs_plan(const qs_sim *sim, int *qubits_per_pass, int max);

/* Failure-detection self-test: launches a kernel that waits on an mbarrier which
 * never completes, with the same bounded wait as the TMA X pass, limited to
 * limit_ms (0 < limit_ms <= 2000).  Expected result: QS_ERR_TIMEOUT, with the
 * context still usable afterwards. */
qs_status qs_selftest_wait(qs_sim *sim, double limit_ms);

/* Checkpoint: write (qs_save) or read (qs_load) the bound state with a header
 * recording lattice, boundary, form, dtype, batch and size; qs_load rejects a file
 * written for a different simulator.  Resuming with qs_evolve from a loaded state
 * continues bit-identically.  Synchronise the stream. */
qs_status qs_save(qs_sim *sim, const char *path);
qs_status qs_load(qs_sim *sim, const char *path);

/* Total milliseconds and launch count of the fused X-pass kernel since the last
 * read, when QS_OPT_PROFILE is on.  Synchronises the stream. */
qs_status qs_profile_read(qs_sim *sim, double *total_ms, long long *launches);
/* The same, split by pass kind: total_ms[2] and launches[2] (host arrays of the
 * caller), index 0 = passes of one factor group, index 1 = shared passes (X of one
 * factor group, its Z layer, X of the next group; QS_OPT_XMERGE).  Resets like
 * qs_profile_read; writes nothing on error. */
qs_status qs_profile_read_kinds(qs_sim *sim, double *total_ms, long long *launches);
/* Number of kernels this library launched since the last call (all kinds). */
long long qs_launch_count(qs_sim *sim);

/* Largest batch accepted by qs_expect_z_noalloc. */
#define QS_NOALLOC_MAX_BATCH 16

/* Norm and Z-string expectation without any memory allocation.  The paper has no
 * counterpart: this entry point exists for callers that must not allocate device
 * memory, e.g. hosts that give all device memory to their own pool before they
 * load plug-ins (a cudaMalloc there fails or takes memory the pool counts on), or
 * loops where the device-wide synchronisation of cudaMalloc is not acceptable.
 *
 * For each of `batch` states of 2^n_qubits amplitudes (layout of qs_bind_state,
 * dtype QS_C64 or QS_C128) at state_dev, writes out_dev[2b] = <psi_b|psi_b> and
 * out_dev[2b + 1] = <psi_b|Z_mask|psi_b> (FP64, device memory supplied by the
 * caller), stream-ordered on `stream` (cudaStream_t as void*, NULL = legacy default).
 * Nothing is synchronised; read out_dev after the stream has completed.
 *
 * No qs_sim handle is needed and nothing is allocated: the block partial sums live
 * in one fixed device array of QS_NOALLOC_MAX_BATCH * 304 * 2 doubles (77,824
 * bytes), held by every GPU that loads the library until the process exits.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call before
 * any stream capture.  All calls on a device share the array, which keeps the last
 * call's partial sums (each call overwrites every slot it later reads, so nothing
 * needs clearing); calls whose kernels overlap on the GPU, e.g. on two streams at
 * once, race on it.  Errors: QS_ERR_ARG for a null pointer, n_qubits outside
 * [1, 34], a bad dtype, batch outside [1, QS_NOALLOC_MAX_BATCH] or mask bits
 * beyond n_qubits; QS_ERR_CUDA if a launch fails.  qs_last_error(NULL) gives the
 * message. */
qs_status qs_expect_z_noalloc(const void *state_dev, int n_qubits, int dtype, int batch,
                              uint64_t zmask, double *out_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* QSIM_H */
