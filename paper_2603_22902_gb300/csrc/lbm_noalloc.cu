// lbm_noalloc.cu -- lbm_field_sums_noalloc: the diagnostics reduction for callers that
// must not allocate device memory.
//
// lbm_get_diagnostics reduces the state of a handle in two passes through a scratch
// buffer of block partial sums that lbm_create allocates with cudaMalloc.  Some callers
// cannot allocate at the time they need these sums: a host embedding that owns the
// device memory through its own arena or pool and forbids other allocators, a service
// whose device memory is fixed when it starts, or a timed loop where allocation latency
// is not allowed.  This entry point computes the same sums from
// caller-owned device fields into a caller-owned device result, using a scratch array
// that lives in this library's device image instead of the heap.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lbm.h"

namespace lbm {
void set_handle_free_error(const char* msg);
}

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 4 * 152;               // partial rows, one per block
constexpr int NA_MAX_K = 2 * LBM_MAXN + 2;           // sums per row
constexpr int NA_MAX_DEVICES = 64;

// Scratch for the block partial sums: NA_MAX_BLOCKS x NA_MAX_K doubles (48.6 KiB), held
// by every GPU that loads the library until the process exits.  Every call shares it.
static __device__ __align__(256) double g_noalloc_partial[NA_MAX_BLOCKS * NA_MAX_K];

// Device addresses of g_noalloc_partial, looked up once per device with that device
// current (the host-side symbol is only a stand-in, not a device address).  They stay
// valid for the life of the device's primary context: after cudaDeviceReset the module
// is loaded again and the cached address may be stale, so this entry point must not be
// used across a reset.
double* g_scratch_addr[NA_MAX_DEVICES] = {};
std::mutex g_scratch_mutex;

// Pass 1: per-block sums of phi_p, (1 - f_l) phi_p, max |sum_p phi_p - 1| and the count of
// non-finite cells, in a fixed order inside the block (same layout as the handle's
// diagnostics: row b holds mass[N], solid[N], max deviation, non-finite count).
__global__ void __launch_bounds__(NA_THREADS) na_partial(const double* __restrict__ phi, const double* __restrict__ fl,
                                                         long long cells, int N, double* __restrict__ partial)
{
    __shared__ double red[NA_MAX_K][NA_THREADS];
    const int K = 2 * N + 2;
    double acc[NA_MAX_K];
    for (int k = 0; k < NA_MAX_K; ++k) acc[k] = 0.0;
    for (long long c = blockIdx.x * (long long)NA_THREADS + threadIdx.x; c < cells;
         c += (long long)gridDim.x * NA_THREADS) {
        const double fs = 1.0 - fl[c];
        double sum = 0.0;
        bool bad = !isfinite(fl[c]);
        for (int p = 0; p < N; ++p) {
            const double v = phi[p * cells + c];
            acc[p] += v;
            acc[N + p] += fs * v;
            sum += v;
        }
        bad = bad || !isfinite(sum);
        acc[2 * N] = fmax(acc[2 * N], fabs(sum - 1.0));
        acc[2 * N + 1] += bad ? 1.0 : 0.0;
    }
    for (int k = 0; k < K; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < K; ++k)
                red[k][threadIdx.x] = (k == 2 * N) ? fmax(red[k][threadIdx.x], red[k][threadIdx.x + s])
                                                   : red[k][threadIdx.x] + red[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < K; ++k) partial[blockIdx.x * K + k] = red[k][0];
}

// Pass 2: one warp adds the block rows in a fixed order and writes the caller's result.
__global__ void na_final(const double* __restrict__ partial, int nblocks, int N, double* __restrict__ out)
{
    const int K = 2 * N + 2;
    const int lane = threadIdx.x;
    for (int k = 0; k < K; ++k) {
        double v = 0.0;
        for (int b = lane; b < nblocks; b += 32) {
            const double w = partial[b * K + k];
            v = (k == 2 * N) ? fmax(v, w) : v + w;
        }
        for (int off = 16; off > 0; off >>= 1) {
            const double o = __shfl_down_sync(0xffffffffu, v, off);
            v = (k == 2 * N) ? fmax(v, o) : v + o;
        }
        if (lane == 0) out[k] = v;
    }
}

}  // namespace

extern "C" int lbm_field_sums_noalloc(const double* phi, const double* fl, int nx, int ny, int N, double* out,
                                      void* stream)
{
    using lbm::set_handle_free_error;
    if (!phi || !fl || !out) {
        set_handle_free_error("lbm_field_sums_noalloc: NULL pointer");
        return LBM_EINVAL;
    }
    if (N < 1 || N > LBM_MAXN || nx < 1 || ny < 1) {
        set_handle_free_error("lbm_field_sums_noalloc: need 1 <= N <= LBM_MAXN and nx, ny >= 1");
        return LBM_EINVAL;
    }
    const long long cells = (long long)nx * ny;
    if (cells > (1LL << 31)) {  // the largest lattice the library accepts
        set_handle_free_error("lbm_field_sums_noalloc: nx * ny exceeds 2^31 cells");
        return LBM_EINVAL;
    }
    // an error left pending by earlier, unrelated work is reported as such and left in
    // place, not taken over as a failure of this call's launches
    if (cudaPeekAtLastError() != cudaSuccess) {
        set_handle_free_error("lbm_field_sums_noalloc: a CUDA error from earlier work is pending; nothing launched");
        return LBM_ECUDA;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        set_handle_free_error("lbm_field_sums_noalloc: no CUDA device, or device index >= 64");
        return LBM_ECUDA;
    }
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_partial) != cudaSuccess || !p) {
                cudaGetLastError();
                set_handle_free_error("lbm_field_sums_noalloc: cudaGetSymbolAddress of the scratch array failed");
                return LBM_ECUDA;
            }
            g_scratch_addr[dev] = (double*)p;
        }
        scratch = g_scratch_addr[dev];
    }
    long long nb = (cells + NA_THREADS - 1) / NA_THREADS;
    if (nb > NA_MAX_BLOCKS) nb = NA_MAX_BLOCKS;  // grid-stride: the scratch never holds more rows
    cudaStream_t st = (cudaStream_t)stream;
    na_partial<<<(int)nb, NA_THREADS, 0, st>>>(phi, fl, cells, N, scratch);
    if (cudaGetLastError() != cudaSuccess) {  // no second pass over rows that were not written
        set_handle_free_error("lbm_field_sums_noalloc: launch of the partial-sum kernel failed");
        return LBM_ECUDA;
    }
    na_final<<<1, 32, 0, st>>>(scratch, (int)nb, N, out);
    if (cudaGetLastError() != cudaSuccess) {
        set_handle_free_error("lbm_field_sums_noalloc: launch of the final-sum kernel failed");
        return LBM_ECUDA;
    }
    return LBM_OK;
}
