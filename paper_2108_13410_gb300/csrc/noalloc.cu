// noalloc.cu -- a reduction entry point that allocates no memory.
//
// qs_expect_z_noalloc computes, per batch element, <psi|psi> and <psi|Z_mask|psi>
// (the same numbers as qs_expect(QS_NORM) and qs_expect_pauli(type 0)) without a
// qs_sim handle and without any device allocation.  It is meant for callers that
// may not allocate: hosts that hand all device memory to their own pool before
// they load plug-ins (a cudaMalloc there fails or steals memory the pool counts
// on), and latency-critical loops where cudaMalloc's implicit device
// synchronisation is not allowed.
//
// Its block partial sums live in a fixed file-scope device array.  Every GPU that
// loads this library holds that array (QS_NOALLOC_MAX_BATCH * 304 * 2 doubles,
// 77,824 bytes) until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "qsim.h"

namespace qsim {
void set_handle_free_error(const std::string &msg);   // read back by qs_last_error(NULL)
}

namespace {

struct ErrSink {
    std::string msg;
    ErrSink &operator=(const std::string &m) { msg = m; qsim::set_handle_free_error(m); return *this; }
    ErrSink &operator=(const char *m) { return *this = std::string(m); }
    // Only this thread's message is reset on entry; the handle-free message that
    // qs_last_error(NULL) reports is replaced when this entry point fails, never
    // erased by a call that succeeds.
    void clear() { msg.clear(); }
};
thread_local ErrSink g_err;


constexpr int NA_BLOCKS = 304;            // 2 blocks per SM on 152 SMs; fixed -> deterministic sums
constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BATCH = QS_NOALLOC_MAX_BATCH;
constexpr int NA_MAX_DEVICES = 64;

// Shared by every call on a device; each call overwrites the slots it reads.
static __device__ __align__(256) double g_noalloc_partials[NA_MAX_BATCH * NA_BLOCKS * 2];

std::mutex g_mu;
double *g_dev_ptr[NA_MAX_DEVICES] = {nullptr};

template <typename V>
__global__ void __launch_bounds__(NA_THREADS) k_norm_z_partials(const V *__restrict__ psi, int n,
                                                                unsigned long long zmask,
                                                                double *__restrict__ partials) {
    __shared__ double sh[NA_THREADS / 32][2];
    const long long dim = 1ll << n;
    psi += (long long)blockIdx.y * dim;
    double a0 = 0.0, a1 = 0.0;
    for (long long i = blockIdx.x * (long long)NA_THREADS + threadIdx.x; i < dim;
         i += (long long)gridDim.x * NA_THREADS) {
        V v = psi[i];
        double p = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        a0 += p;
        a1 += (__popcll((unsigned long long)i & zmask) & 1) ? -p : p;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sh[w][0] = a0; sh[w][1] = a1; }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int k = 0; k < NA_THREADS / 32; ++k) s += sh[k][threadIdx.x];
        partials[((long long)blockIdx.y * gridDim.x + blockIdx.x) * 2 + threadIdx.x] = s;
    }
}

__global__ void k_norm_z_finish(const double *__restrict__ partials, int nblk, double *__restrict__ out) {
    __shared__ double sh[2][NA_THREADS];
    const int b = blockIdx.x;
    double a0 = 0.0, a1 = 0.0;
    for (int k = threadIdx.x; k < nblk; k += NA_THREADS) {
        a0 += partials[((long long)b * nblk + k) * 2];
        a1 += partials[((long long)b * nblk + k) * 2 + 1];
    }
    sh[0][threadIdx.x] = a0;
    sh[1][threadIdx.x] = a1;
    __syncthreads();
    for (int w = NA_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[2 * b] = sh[0][0]; out[2 * b + 1] = sh[1][0]; }
}

// Device address of the partials array for the current device, looked up once.
qs_status scratch_for_current_device(double **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { g_err = std::string("cudaGetDevice: ") + cudaGetErrorString(e); return QS_ERR_CUDA; }
    if (dev < 0 || dev >= NA_MAX_DEVICES) { g_err = "device ordinal out of range"; return QS_ERR_ARG; }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) {
            g_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return QS_ERR_CUDA;
        }
        g_dev_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_dev_ptr[dev];
    return QS_OK;
}

}  // namespace

extern "C" qs_status qs_expect_z_noalloc(const void *state_dev, int n_qubits, int dtype, int batch,
                                         uint64_t zmask, double *out_dev, void *stream) {
    g_err.clear();
    if (!state_dev || !out_dev) { g_err = "null state or output pointer"; return QS_ERR_ARG; }
    if (n_qubits < 1 || n_qubits > 34) { g_err = "n_qubits must be in [1, 34]"; return QS_ERR_ARG; }
    if (dtype != QS_C64 && dtype != QS_C128) { g_err = "dtype must be QS_C64 or QS_C128"; return QS_ERR_ARG; }
    if (batch < 1 || batch > NA_MAX_BATCH) {
        char b[128];
        snprintf(b, sizeof(b), "batch %d outside [1, %d] (the fixed scratch array holds %d batch elements)",
                 batch, NA_MAX_BATCH, NA_MAX_BATCH);
        g_err = b;
        return QS_ERR_ARG;
    }
    if (n_qubits < 64 && (zmask >> n_qubits) != 0) { g_err = "zmask has bits beyond n_qubits"; return QS_ERR_ARG; }
    double *partials = nullptr;
    qs_status st = scratch_for_current_device(&partials);
    if (st != QS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    long long dim = 1ll << n_qubits;
    long long want = (dim + NA_THREADS - 1) / NA_THREADS;
    int blocks = (int)(want < NA_BLOCKS ? want : NA_BLOCKS);
    dim3 grid(blocks, batch);
    if (dtype == QS_C64)
        k_norm_z_partials<float2><<<grid, NA_THREADS, 0, s>>>(static_cast<const float2 *>(state_dev), n_qubits,
                                                              (unsigned long long)zmask, partials);
    else
        k_norm_z_partials<double2><<<grid, NA_THREADS, 0, s>>>(static_cast<const double2 *>(state_dev), n_qubits,
                                                               (unsigned long long)zmask, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { g_err = std::string("launch: ") + cudaGetErrorString(e); return QS_ERR_CUDA; }
    k_norm_z_finish<<<batch, NA_THREADS, 0, s>>>(partials, blocks, out_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) { g_err = std::string("launch: ") + cudaGetErrorString(e); return QS_ERR_CUDA; }
    return QS_OK;
}
