// lbm_adjoint_capi.cu -- lbm_adjoint_fl_loss (include/lbm.h): the forward run with
// checkpoints, the loss of the final liquid fraction, and the reverse sweep of the
// adjoint step (lbm_adjoint.cuh) with recomputation of each segment.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_handle.hpp"
#include "lbm_trace.hpp"
#include "lbm_launch.cuh"

using namespace lbm;

namespace {

constexpr int PS_NT = 256;   // threads of a plane-sum block
constexpr int PS_NB = 256;   // blocks per plane (partials per plane)

// Pass 1: block b of plane k sums a grid-stride slice in a fixed order.
__global__ void plane_partial_kernel(const double* __restrict__ planes, long long S, double* __restrict__ partial)
{
    __shared__ double red[PS_NT];
    const int k = blockIdx.y;
    const double* v = planes + (long long)k * S;
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)PS_NT + threadIdx.x; c < S; c += (long long)gridDim.x * PS_NT) acc += v[c];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = PS_NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(long long)k * gridDim.x + blockIdx.x] = red[0];
}

// Pass 2: one warp per plane adds the partials in a fixed order.
__global__ void plane_final_kernel(const double* __restrict__ partial, int nb, double* __restrict__ out)
{
    const int k = blockIdx.x;
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) v += partial[(long long)k * nb + b];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) out[k] = v;
}

}  // namespace

namespace lbm {
cudaError_t launch_plane_sums(const double* planes, int nplanes, long long S, double* partial, double* out,
                              cudaStream_t st)
{
    plane_partial_kernel<<<dim3(PS_NB, nplanes), PS_NT, 0, st>>>(planes, S, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    plane_final_kernel<<<nplanes, 32, 0, st>>>(partial, PS_NB, out);
    return cudaGetLastError();
}
}  // namespace lbm

namespace {

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { cudaFree(p); }
    cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes); }
    template <class T>
    T* as() const
    {
        return static_cast<T*>(p);
    }
};

int afail(lbm_handle* h, int code, const std::string& msg)
{
    h->err = msg;
    return code;
}

int acuda(lbm_handle* h, cudaError_t e, const char* where)
{
    cudaGetLastError();
    return afail(h, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

#define ADJ_TRY(h, call)                                  \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return acuda(h, e_, #call); \
    } while (0)

template <class F>
cudaError_t by_n(int N, F&& f)
{
    if (N == 2) return f(std::integral_constant<int, 2>{});
    if (N == 3) return f(std::integral_constant<int, 3>{});
    return f(std::integral_constant<int, 4>{});
}

}  // namespace

extern "C" int lbm_adjoint_fl_loss(lbm_handle* h, const double* phi0, const double* T0, const double* ux0,
                                   const double* uy0, const double* fl_target, const double* weight, int where,
                                   long nsteps, int checkpoint_every, lbm_fl_grad* out)
{
    const lbm::TraceRange trace_range("lbm_adjoint_fl_loss");
    if (!h) return LBM_EINVAL;
    if (!phi0 || !T0 || !fl_target || !out) return afail(h, LBM_EINVAL, "phi0, T0, fl_target and out are required");
    if (where != LBM_HOST && where != LBM_DEVICE) return afail(h, LBM_EINVAL, "bad where");
    if (h->precision != LBM_FP64) return afail(h, LBM_EINVAL, "the adjoint runs on FP64 handles");
    if (nsteps < 0) return afail(h, LBM_EINVAL, "nsteps must be >= 0");
    if (checkpoint_every < 1) return afail(h, LBM_EINVAL, "checkpoint_every must be >= 1");
    ADJ_TRY(h, cudaSetDevice(h->device));
    const int N = h->N;
    const long long S = h->P.S;
    const size_t plane = (size_t)S * sizeof(double);
    const KParams& P = h->P;
    cudaStream_t st = h->stream;
    const size_t set_bytes = h->pop_bytes + h->aux_bytes;
    const int K = (int)std::min<long>(checkpoint_every, std::max<long>(nsteps, 1));
    const long nck = (nsteps + K - 1) / K;

    // inputs on the device (the initial fields are needed again at the end)
    DevBuf in0, tgt;
    ADJ_TRY(h, in0.alloc((size_t)(N + 3) * plane));
    ADJ_TRY(h, tgt.alloc(2 * plane));
    double* d_phi0 = in0.as<double>();
    double* d_T0 = d_phi0 + N * S;
    double* d_ux0 = d_T0 + S;
    double* d_uy0 = d_ux0 + S;
    const cudaMemcpyKind kind = where == LBM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    ADJ_TRY(h, cudaMemcpyAsync(d_phi0, phi0, N * plane, kind, st));
    ADJ_TRY(h, cudaMemcpyAsync(d_T0, T0, plane, kind, st));
    ADJ_TRY(h, ux0 ? cudaMemcpyAsync(d_ux0, ux0, plane, kind, st) : cudaMemsetAsync(d_ux0, 0, plane, st));
    ADJ_TRY(h, uy0 ? cudaMemcpyAsync(d_uy0, uy0, plane, kind, st) : cudaMemsetAsync(d_uy0, 0, plane, st));
    ADJ_TRY(h, cudaMemcpyAsync(tgt.as<double>(), fl_target, plane, kind, st));
    if (weight) ADJ_TRY(h, cudaMemcpyAsync(tgt.as<double>() + S, weight, plane, kind, st));

    // working memory: checkpoints, one recomputed segment, adjoint sets and planes
    DevBuf ck, seg, abar, mac, own, sb, grad, part, sums;
    ADJ_TRY(h, ck.alloc(std::max<long>(nck, 1) * set_bytes));
    ADJ_TRY(h, seg.alloc((size_t)K * set_bytes));
    ADJ_TRY(h, abar.alloc(2 * set_bytes));
    ADJ_TRY(h, mac.alloc((size_t)(N + 2) * plane));
    ADJ_TRY(h, own.alloc((size_t)(N + 1) * plane));
    ADJ_TRY(h, sb.alloc((size_t)9 * (N + 2) * plane));
    ADJ_TRY(h, grad.alloc((size_t)(GS_COUNT + 1) * plane));
    ADJ_TRY(h, part.alloc((size_t)(GS_COUNT + 1) * 256 * sizeof(double)));
    ADJ_TRY(h, sums.alloc((size_t)(GS_COUNT + 1) * sizeof(double)));
    ADJ_TRY(h, cudaMemsetAsync(grad.p, 0, (size_t)(GS_COUNT + 1) * plane, st));
    auto pop_of = [&](char* set) { return (void*)set; };
    auto aux_of = [&](char* set) { return (void*)(set + h->pop_bytes); };

    // ---- forward: initial state, steps with a checkpoint every K ----
    cudaError_t e = dispatch(N, LBM_FP64, [&](auto n, auto pr) {
        return launch_init<decltype(n)::value, decltype(pr)>(P, d_phi0, d_T0, d_ux0, d_uy0, h->pop[0], h->aux[0], st);
    });
    if (e != cudaSuccess) return acuda(h, e, "init kernel");
    h->cur = 0;
    h->ready = true;
    h->steps = 0;
    for (long n = 0; n < nsteps; ++n) {
        const int a = h->cur, b = a ^ 1;
        if (n % K == 0) {
            char* c0 = ck.as<char>() + (size_t)(n / K) * set_bytes;
            ADJ_TRY(h, cudaMemcpyAsync(pop_of(c0), h->pop[a], h->pop_bytes, cudaMemcpyDeviceToDevice, st));
            ADJ_TRY(h, cudaMemcpyAsync(aux_of(c0), h->aux[a], h->aux_bytes, cudaMemcpyDeviceToDevice, st));
        }
        e = dispatch(N, LBM_FP64, [&](auto nn, auto pr) {
            return launch_step<decltype(nn)::value, decltype(pr)>(P, h->pop[a], h->pop[b], h->aux[a], h->aux[b],
                                                                  h->tile, st);
        });
        if (e != cudaSuccess) return acuda(h, e, "step kernel");
        h->cur = b;
        h->steps++;
    }

    // ---- loss of the final state and its adjoint ----
    char* abuf[2] = {abar.as<char>(), abar.as<char>() + set_bytes};
    int ia = 0;
    AdjBufs B{};
    B.mac = mac.as<double>();
    B.own = own.as<double>();
    B.sb = sb.as<double>();
    B.grad = grad.as<double>();
    B.fl_target = tgt.as<double>();
    B.weight = weight ? tgt.as<double>() + S : nullptr;
    B.pin = (const double*)h->pop[h->cur];
    B.ain = (const double*)h->aux[h->cur];
    B.apop = (double*)pop_of(abuf[ia]);
    B.aaux = (double*)aux_of(abuf[ia]);
    e = by_n(N, [&](auto n) { return launch_adj_moments<decltype(n)::value>(P, B, true, st); });
    if (e != cudaSuccess) return acuda(h, e, "loss seed kernel");

    // ---- reverse sweep: per segment, recompute its states, then step back ----
    for (long sgi = nck - 1; sgi >= 0; --sgi) {
        const long n0 = sgi * K, n1 = std::min<long>(nsteps, n0 + K);
        char* s0 = seg.as<char>();
        const char* c0 = ck.as<char>() + (size_t)sgi * set_bytes;
        ADJ_TRY(h, cudaMemcpyAsync(s0, c0, set_bytes, cudaMemcpyDeviceToDevice, st));
        for (long j = 1; j < n1 - n0; ++j) {
            char* sa = seg.as<char>() + (size_t)(j - 1) * set_bytes;
            char* sbn = seg.as<char>() + (size_t)j * set_bytes;
            e = dispatch(N, LBM_FP64, [&](auto nn, auto pr) {
                return launch_step<decltype(nn)::value, decltype(pr)>(P, pop_of(sa), pop_of(sbn), aux_of(sa), aux_of(sbn),
                                                                      h->tile, st);
            });
            if (e != cudaSuccess) return acuda(h, e, "recompute step kernel");
        }
        for (long n = n1 - 1; n >= n0; --n) {
            char* sa = seg.as<char>() + (size_t)(n - n0) * set_bytes;
            B.pin = (const double*)pop_of(sa);
            B.ain = (const double*)aux_of(sa);
            B.bpop = (const double*)pop_of(abuf[ia]);
            B.baux = (const double*)aux_of(abuf[ia]);
            B.apop = (double*)pop_of(abuf[ia ^ 1]);
            B.aaux = (double*)aux_of(abuf[ia ^ 1]);
            e = by_n(N, [&](auto nn) {
                constexpr int NN = decltype(nn)::value;
                cudaError_t r = launch_adj_mac<NN>(P, B.pin, B.ain, mac.as<double>(), st);
                if (r == cudaSuccess) r = launch_adj_cell<NN>(P, B, st);
                if (r == cudaSuccess) r = launch_adj_moments<NN>(P, B, false, st);
                return r;
            });
            if (e != cudaSuccess) return acuda(h, e, "adjoint step kernels");
            ia ^= 1;
        }
    }

    // ---- the initial state's share, then the sums ----
    e = by_n(N, [&](auto n) {
        return launch_adj_init<decltype(n)::value>(P, d_phi0, d_T0, (const double*)pop_of(abuf[ia]), B.grad, st);
    });
    if (e != cudaSuccess) return acuda(h, e, "adjoint init kernel");
    ADJ_TRY(h, launch_plane_sums(B.grad, GS_COUNT + 1, S, part.as<double>(), sums.as<double>(), st));
    double host[GS_COUNT + 1];
    ADJ_TRY(h, cudaMemcpyAsync(host, sums.p, sizeof host, cudaMemcpyDeviceToHost, st));
    ADJ_TRY(h, cudaStreamSynchronize(st));
    std::memset(out, 0, sizeof *out);
    out->loss = host[GS_LOSS];
    for (int s = 0; s < 4; ++s) out->T_wall[s] = host[GS_TW + s];
    for (int p = 0; p < N; ++p) {
        out->rhoL[p] = host[GS_RHOL + p];
        out->lambda_s[p] = host[GS_LAMS + p];
        out->lambda_l[p] = host[GS_LAML + p];
    }
    return LBM_OK;
}
