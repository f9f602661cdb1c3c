// lbm_capi.cu -- the C ABI declared in include/lbm.h: handle, parameter checks and
// derivations (Sections 2-3 of arXiv 2603.22902), device memory, launches.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/lbm.h"
#include "lbm_handle.hpp"
#include "lbm_trace.hpp"
#include "lbm_launch.cuh"
#include "lbm_staged.cuh"

using namespace lbm;

static thread_local std::string g_create_error;

namespace lbm {
// Message of a failing call that has no handle (reported by lbm_last_error(NULL)).
void set_handle_free_error(const char* msg) { g_create_error = msg; }
}  // namespace lbm

static int fail(lbm_handle* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

static int cuda_fail(lbm_handle* h, cudaError_t e, const char* where)
{
    return fail(h, LBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA_TRY(h, call)                                  \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

static size_t plane_bytes(const lbm_handle* h) { return (size_t)h->P.S * sizeof(double); }

static void free_all(lbm_handle* h)
{
    for (int k = 0; k < 2; ++k) {
        cudaFree(h->pop[k]);
        cudaFree(h->aux[k]);
        h->pop[k] = h->aux[k] = nullptr;
    }
    cudaFree(h->io);
    cudaFree(h->diag_partial);
    cudaFree(h->diag_out);
    cudaFree(h->dbg);
    cudaFree(h->stage_status);
    h->stage_status = nullptr;
    h->io = h->diag_partial = h->diag_out = nullptr;
    h->dbg = nullptr;
}

// Double-word copy of the coefficients, for the double-word policy.
static Coef<df64> split_coef(const Coef<double>& d)
{
    static_assert(sizeof(Coef<double>) == sizeof(Coef<df64>), "Coef holds only T members");
    Coef<df64> x{};
    const double* src = reinterpret_cast<const double*>(&d);
    df64* dst = reinterpret_cast<df64*>(&x);
    for (size_t k = 0; k < sizeof(Coef<double>) / sizeof(double); ++k) dst[k] = df64(src[k]);
    return x;
}

// FP32 copy of the coefficients, for the policies that compute in FP32.
static Coef<float> round_coef(const Coef<double>& d)
{
    static_assert(sizeof(Coef<double>) == 2 * sizeof(Coef<float>), "Coef holds only T members");
    Coef<float> f{};
    const double* src = reinterpret_cast<const double*>(&d);
    float* dst = reinterpret_cast<float*>(&f);
    for (size_t k = 0; k < sizeof(Coef<double>) / sizeof(double); ++k) dst[k] = (float)src[k];
    return f;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to the driver
// library); NULL when the driver does not provide it.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    }
    return fn;
}

// One 3D tensor map over `planes` planes [ny][nx] of esz-byte elements at base, with box
// (bx, by, bz).
static bool encode_map(CUtensorMap* m, void* base, int esz, int nx, int ny, int planes, int bx, int by, int bz)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const CUtensorMapDataType dt = esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                   : esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32
                                              : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * esz, (cuuint64_t)nx * ny * esz};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The six maps of a population set and a lagged set (boxes A..F of lbm_staged.cuh).
template <int N, class Pr>
static bool encode_stage_maps(const lbm_handle* h, const void* pop, const void* aux, StageMaps& M)
{
    using Lay = StageLayout<N, Pr>;
    const int nx = h->nx, ny = h->ny;
    char* rest = (char*)pop;
    char* move = rest + h->P.rest_elems * Lay::ER;
    char* lag = (char*)aux;
    return encode_map(&M.m[0], move, Lay::EM, nx, ny, 8 * (N + 2), STAGE_TX, STAGE_TY, 8) &&
           encode_map(&M.m[1], move, Lay::EM, nx, ny, 8 * (N + 2), Lay::WM, Lay::H, 8 * (N + 1)) &&
           encode_map(&M.m[2], rest, Lay::ER, nx, ny, N + 2, STAGE_TX, STAGE_TY, 1) &&
           encode_map(&M.m[3], rest, Lay::ER, nx, ny, N + 2, Lay::WR, Lay::H, N + 1) &&
           encode_map(&M.m[4], lag, Lay::EA, nx, ny, 3 + 2 * N, Lay::WA, Lay::H, 2) &&
           encode_map(&M.m[5], lag, Lay::EA, nx, ny, 3 + 2 * N, STAGE_TX, STAGE_TY, 1 + 2 * N);
}

bool lbm_encode_stage_maps(const lbm_handle* h, const void* pop, const void* aux, StageMaps* M)
{
    if (!h || !M || (h->N != 2 && h->N != 3) || h->nx % 8 != 0) return false;
    if (h->precision == LBM_FP16S)
        return h->N == 2 ? encode_stage_maps<2, PrecFP16S>(h, pop, aux, *M) : encode_stage_maps<3, PrecFP16S>(h, pop, aux, *M);
    if (h->precision == LBM_BF16S)
        return h->N == 2 ? encode_stage_maps<2, PrecBF16S>(h, pop, aux, *M) : encode_stage_maps<3, PrecBF16S>(h, pop, aux, *M);
    return false;
}

// Turn the staged step on where the handle allows it (see lbm_set_staging); with report,
// the reason it does not apply goes to lbm_last_error.
static int enable_staging(lbm_handle* h, bool report)
{
    if ((h->precision != LBM_FP16S && h->precision != LBM_BF16S) || (h->N != 2 && h->N != 3))
        return report ? fail(h, LBM_EINVAL, "the staged step is compiled for LBM_FP16S and LBM_BF16S with N = 2 or 3")
                      : LBM_EINVAL;
    if (h->nx % 8 != 0)
        return report ? fail(h, LBM_EINVAL, "the staged step needs nx a multiple of 8 (16-byte rows)") : LBM_EINVAL;
    if (h->tile != TILE_32x8) return report ? fail(h, LBM_EINVAL, "the staged step uses the 32x8 tile") : LBM_EINVAL;
    LBM_CUDA_TRY(h, cudaSetDevice(h->device));
    if (!h->stage_status) {
        LBM_CUDA_TRY(h, cudaMalloc(&h->stage_status, sizeof(int)));
        LBM_CUDA_TRY(h, cudaMemset(h->stage_status, 0, sizeof(int)));
    }
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k) ok = lbm_encode_stage_maps(h, h->pop[k], h->aux[k], &h->stage_maps[k]);
    if (!ok) return report ? fail(h, LBM_ECUDA, "tensor maps of the staged step could not be encoded") : LBM_ECUDA;
    h->staged = true;
    return LBM_OK;
}

extern "C" {

int lbm_create(const lbm_grid* grid, int N, const lbm_phase* phases, const lbm_thermal* th, const lbm_bc* bc,
               const lbm_numerics* num, lbm_handle** out)
{
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid || !phases || !th || !bc || !num) return fail(nullptr, LBM_EINVAL, "NULL argument");
    if (grid->nx < 3 || grid->ny < 3) return fail(nullptr, LBM_EINVAL, "nx and ny must be >= 3");
    if ((long long)grid->nx * grid->ny > (1LL << 31)) return fail(nullptr, LBM_EINVAL, "grid too large");
    if (N < 2 || N > LBM_MAXN) return fail(nullptr, LBM_EINVAL, "N must be in [2, 4]");
    if (num->precision < LBM_FP64 || num->precision > LBM_DF64)
        return fail(nullptr, LBM_EINVAL, "precision must be LBM_FP64, LBM_FP32, LBM_FP16S, LBM_BF16S or LBM_DF64");
    if (!(num->eps > 0.0) || !(num->mobility > 0.0)) return fail(nullptr, LBM_EINVAL, "eps and mobility must be > 0");
    if (num->diag_every < 0) return fail(nullptr, LBM_EINVAL, "diag_every must be >= 0");
    if (!(th->T_sol <= th->T_liq)) return fail(nullptr, LBM_EINVAL, "T_sol must be <= T_liq");
    if (!(th->rho_ref > 0.0) || !(th->cp_ref >= 0.0)) return fail(nullptr, LBM_EINVAL, "rho_ref > 0, cp_ref >= 0");
    for (int p = 0; p < N; ++p) {
        const lbm_phase& ph = phases[p];
        if (!(ph.rho_l > 0.0 && ph.rho_s > 0.0 && ph.cp_l > 0.0 && ph.cp_s > 0.0))
            return fail(nullptr, LBM_EINVAL, "densities and heat capacities must be > 0");
        // tau_f = mu / (rho c_s^2) + 1/2 > 1/2 and tau_h = lambda / (rho_ref c_ref c_s^2) + 1/2 > 1/2
        if (!(ph.mu_l > 0.0 && ph.mu_s > 0.0)) return fail(nullptr, LBM_EINVAL, "viscosities must be > 0 (tau_f > 1/2)");
        if (!(ph.lambda_l > 0.0 && ph.lambda_s > 0.0))
            return fail(nullptr, LBM_EINVAL, "conductivities must be > 0 (tau_h > 1/2)");
        if (!(ph.latent >= 0.0)) return fail(nullptr, LBM_EINVAL, "latent heat must be >= 0");
        for (int q = 0; q < N; ++q) {
            const double s = num->sigma[p * LBM_MAXN + q];
            if (s != num->sigma[q * LBM_MAXN + p] || !(s >= 0.0) || (p == q && s != 0.0))
                return fail(nullptr, LBM_EINVAL, "sigma must be symmetric, >= 0, zero on the diagonal");
        }
    }
    for (int s = 0; s < 4; ++s) {
        if (bc->kind[s] < LBM_BC_PERIODIC || bc->kind[s] > LBM_BC_OUTFLOW) return fail(nullptr, LBM_EINVAL, "bad bc kind");
        if (bc->tkind[s] != LBM_T_ADIABATIC && bc->tkind[s] != LBM_T_DIRICHLET)
            return fail(nullptr, LBM_EINVAL, "bad thermal bc kind");
        if (s < 2 && bc->kind[s] == LBM_BC_OUTFLOW) return fail(nullptr, LBM_EINVAL, "outflow only on y sides");
        if (bc->tkind[s] == LBM_T_DIRICHLET && (s < 2 || bc->kind[s] != LBM_BC_WALL))
            return fail(nullptr, LBM_EINVAL, "Dirichlet temperature only on y-side walls");
    }
    if ((bc->kind[0] == LBM_BC_PERIODIC) != (bc->kind[1] == LBM_BC_PERIODIC) ||
        (bc->kind[2] == LBM_BC_PERIODIC) != (bc->kind[3] == LBM_BC_PERIODIC))
        return fail(nullptr, LBM_EINVAL, "periodic sides must come in pairs");

    lbm_handle* h = new (std::nothrow) lbm_handle();
    if (!h) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return fail(nullptr, LBM_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    h->N = N;
    h->nx = grid->nx;
    h->ny = grid->ny;
    h->precision = num->precision;
    h->diag_every = num->diag_every;

    KParams& P = h->P;
    P.nx = grid->nx;
    P.ny = grid->ny;
    P.N = N;
    P.S = (long long)grid->nx * grid->ny;
    for (int s = 0; s < 4; ++s) {
        P.bc[s] = bc->kind[s];
        P.tbc[s] = bc->tkind[s];
        P.d.Tw[s] = bc->T_wall[s];
    }
    for (int p = 0; p < N; ++p) {
        const lbm_phase& ph = phases[p];
        P.d.rho_l[p] = ph.rho_l;
        P.d.rho_s[p] = ph.rho_s;
        P.d.mu_l[p] = ph.mu_l;
        P.d.mu_s[p] = ph.mu_s;
        P.d.lam_l[p] = ph.lambda_l;
        P.d.lam_s[p] = ph.lambda_s;
        P.d.cp_l[p] = ph.cp_l;
        P.d.cp_s[p] = ph.cp_s;
        P.rhoL[p] = ph.rho_l * ph.latent;
        P.d.rhoL[p] = P.rhoL[p];
        P.d.drho[p] = ph.rho_s - ph.rho_l;
        P.d.pcm[p] = ph.latent > 0.0 ? 1.0 : 0.0;
        for (int q = 0; q < N; ++q) {
            const double sig = num->sigma[p * LBM_MAXN + q];
            P.d.b2[p][q] = 2.0 * 3.0 / num->eps * sig;      // 2 beta_pq
            P.d.kk[p][q] = 3.0 * num->eps / 4.0 * sig;      // -k_pq
            for (int s = 0; s < 4; ++s)
                P.d.wet[s][p][q] = bc->kind[s] == LBM_BC_WALL ? 4.0 / num->eps * bc->wet_cos[s][p * LBM_MAXN + q] : 0.0;
        }
    }
    P.d.four_eps = 4.0 / num->eps;
    P.T_sol = P.d.T_sol = th->T_sol;
    P.T_liq = P.d.T_liq = th->T_liq;
    const double cp_ref = th->cp_ref > 0.0 ? th->cp_ref
                                           : 2.0 * phases[0].cp_s * phases[0].cp_l / (phases[0].cp_s + phases[0].cp_l);
    P.d.E_ref = th->rho_ref * cp_ref;
    P.d.tau_h_scale = 3.0 / P.d.E_ref;
    P.d.us[0] = th->u_solid[0];
    P.d.us[1] = th->u_solid[1];
    P.d.accel[0] = th->accel[0];
    P.d.accel[1] = th->accel[1];
    const double tau_g = num->mobility * 3.0 + 0.5;
    P.d.omega_g = 1.0 / tau_g;
    P.d.kg = 1.0 - 0.5 * P.d.omega_g;

    const size_t pb = plane_bytes(h);
    P.rest_elems = (long long)(N + 2) * P.S;
    P.move_elems = 8LL * (N + 2) * P.S;
    P.aux_elems = (long long)naux_planes(N) * P.S;
    P.d.inv_E_ref = 1.0 / P.d.E_ref;
    P.f = round_coef(P.d);
    P.x = split_coef(P.d);
    P.dbg = nullptr;
    dispatch(N, h->precision, [&](auto n, auto pr) {
        using Pr = decltype(pr);
        h->pop_bytes = (size_t)pop_set_bytes<Pr>(decltype(n)::value, P.S);
        h->aux_bytes = (size_t)aux_set_bytes<Pr>(decltype(n)::value, P.S);
        return 0;
    });
    const int nb = diag_blocks(P.S);
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k) {
        ok = cudaMalloc(&h->pop[k], h->pop_bytes) == cudaSuccess && cudaMalloc(&h->aux[k], h->aux_bytes) == cudaSuccess;
    }
    ok = ok && cudaMalloc(&h->io, (size_t)(N + 6) * pb) == cudaSuccess;
    ok = ok && cudaMalloc(&h->diag_partial, (size_t)nb * (2 * N + 2) * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc(&h->diag_out, (size_t)(2 * N + 2) * sizeof(double)) == cudaSuccess;
#ifdef LBM_CHECK_BOUNDS
    ok = ok && cudaMalloc(&h->dbg, 3 * sizeof(unsigned long long)) == cudaSuccess &&
         cudaMemset(h->dbg, 0, 3 * sizeof(unsigned long long)) == cudaSuccess;
    P.dbg = h->dbg;
#endif
    if (!ok) {
        cudaGetLastError();
        free_all(h);
        delete h;
        return fail(nullptr, LBM_ENOMEM, "device allocation failed");
    }
    // the TMA-staged step is the default where it applies (it computes every cell as the
    // one-launch form does, bit for bit)
    if (enable_staging(h, false) != LBM_OK) cudaGetLastError();
    *out = h;
    return LBM_OK;
}

int lbm_set_stream(lbm_handle* h, void* stream)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    h->stream = (cudaStream_t)stream;
    return LBM_OK;
}

int lbm_set_tile(lbm_handle* h, int bx, int by)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (bx == 0 && by == 0) {
        h->tile = TILE_32x8;
        return LBM_OK;
    }
    for (int id = 0; id < TILE_COUNT; ++id) {
        int tx, ty;
        tile_dims(id, tx, ty);
        if (tx == bx && ty == by) {
            if (h->precision == LBM_DF64 && id != TILE_32x8)
                return fail(h, LBM_EINVAL, "the LBM_DF64 policy is compiled for the 32x8 tile only");
            if (id != TILE_32x8) h->staged = false;  // the staged step is compiled for 32x8
            h->tile = id;
            return LBM_OK;
        }
    }
    return fail(h, LBM_EINVAL, "tile shape not compiled (32x8, 32x4, 64x4, 16x16)");
}

int lbm_set_staging(lbm_handle* h, int on)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!on) {
        h->staged = false;
        return LBM_OK;
    }
    return enable_staging(h, true);
}

int lbm_set_fields(lbm_handle* h, const double* phi, const double* T, const double* ux, const double* uy, int where)
{
    const lbm::TraceRange trace_range("lbm_set_fields");
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!phi || !T) return fail(h, LBM_EINVAL, "phi and T are required");
    if (where != LBM_HOST && where != LBM_DEVICE) return fail(h, LBM_EINVAL, "bad where");
    LBM_CUDA_TRY(h, cudaSetDevice(h->device));
    const size_t pb = plane_bytes(h);
    const double *dphi = phi, *dT = T, *dux = ux, *duy = uy;
    if (where == LBM_HOST) {
        double* s = h->io;
        LBM_CUDA_TRY(h, cudaMemcpyAsync(s, phi, h->N * pb, cudaMemcpyHostToDevice, h->stream));
        LBM_CUDA_TRY(h, cudaMemcpyAsync(s + h->N * h->P.S, T, pb, cudaMemcpyHostToDevice, h->stream));
        dphi = s;
        dT = s + h->N * h->P.S;
        if (ux) {
            LBM_CUDA_TRY(h, cudaMemcpyAsync(s + (h->N + 1) * h->P.S, ux, pb, cudaMemcpyHostToDevice, h->stream));
            dux = s + (h->N + 1) * h->P.S;
        }
        if (uy) {
            LBM_CUDA_TRY(h, cudaMemcpyAsync(s + (h->N + 2) * h->P.S, uy, pb, cudaMemcpyHostToDevice, h->stream));
            duy = s + (h->N + 2) * h->P.S;
        }
    }
    h->cur = 0;
    cudaError_t e = dispatch(h->N, h->precision, [&](auto n, auto pr) {
        return launch_init<decltype(n)::value, decltype(pr)>(h->P, dphi, dT, dux, duy, h->pop[0], h->aux[0], h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "init kernel");
    if (where == LBM_HOST) LBM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->ready = true;
    h->steps = 0;
    return LBM_OK;
}

// LBM_ETIMEOUT (and the status word cleared) when a staged step gave up an mbarrier wait.
static int check_stage_status(lbm_handle* h)
{
    if (!h->stage_status) return LBM_OK;
    int st = 0;
    LBM_CUDA_TRY(h, cudaMemcpyAsync(&st, h->stage_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (st != 0) {
        LBM_CUDA_TRY(h, cudaMemsetAsync(h->stage_status, 0, sizeof(int), h->stream));
        return fail(h, LBM_ETIMEOUT, "a staged step gave up waiting for its tensor copies; the state is undefined");
    }
    return LBM_OK;
}

static int run_diag(lbm_handle* h, double* host_out)
{
    cudaError_t e = dispatch(h->N, h->precision, [&](auto n, auto pr) {
        return launch_diag<decltype(n)::value, decltype(pr)>(h->P, h->pop[h->cur], h->aux[h->cur], h->diag_partial,
                                                             h->diag_out, h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics kernel");
    LBM_CUDA_TRY(h, cudaMemcpyAsync(host_out, h->diag_out, (2 * h->N + 2) * sizeof(double), cudaMemcpyDeviceToHost,
                                    h->stream));
    LBM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return check_stage_status(h);
}

int lbm_step(lbm_handle* h, long nsteps)
{
    const lbm::TraceRange trace_range("lbm_step");
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!h->ready) return fail(h, LBM_ESTATE, "lbm_set_fields has not been called");
    if (nsteps < 0) return fail(h, LBM_EINVAL, "nsteps must be >= 0");
    if (h->slab_inner_pending)
        return fail(h, LBM_ESTATE, "a slab step is half done: lbm_slab_step_part(LBM_SLAB_EDGE) first");
    LBM_CUDA_TRY(h, cudaSetDevice(h->device));
    for (long n = 0; n < nsteps; ++n) {
        const int a = h->cur, b = a ^ 1;
        cudaError_t e = dispatch(h->N, h->precision, [&](auto n, auto pr) {
            if (h->staged)
                return launch_staged<decltype(n)::value, decltype(pr)>(h->P, h->stage_maps[a], h->pop[a], h->pop[b],
                                                                       h->aux[a], h->aux[b], h->stage_status,
                                                                       h->stream);
            return launch_step<decltype(n)::value, decltype(pr)>(h->P, h->pop[a], h->pop[b], h->aux[a], h->aux[b],
                                                                 h->tile, h->stream);
        });
        if (e != cudaSuccess) return cuda_fail(h, e, "step kernel");
        h->cur = b;
        h->steps++;
        if (h->diag_every > 0 && h->steps % h->diag_every == 0) {
            double d[2 * LBM_MAXN + 2];
            int rc = run_diag(h, d);
            if (rc != LBM_OK) return rc;
            if (d[2 * h->N + 1] > 0.0) return fail(h, LBM_EUNSTABLE, "non-finite value in the state");
        }
    }
    return LBM_OK;
}

int lbm_get_fields(lbm_handle* h, double* phi, double* T, double* H, double* fl, double* ux, double* uy, double* p,
                   int where)
{
    const lbm::TraceRange trace_range("lbm_get_fields");
    if (!h) return fail(nullptr, LBM_EINVAL, "NULL handle");
    if (!h->ready) return fail(h, LBM_ESTATE, "lbm_set_fields has not been called");
    if (where != LBM_HOST && where != LBM_DEVICE) return fail(h, LBM_EINVAL, "bad where");
    LBM_CUDA_TRY(h, cudaSetDevice(h->device));
    const long long S = h->P.S;
    double* user[7] = {phi, T, H, fl, ux, uy, p};
    double* dev[7];
    if (where == LBM_DEVICE) {
        for (int k = 0; k < 7; ++k) dev[k] = user[k];
    } else {
        long long off = 0;
        for (int k = 0; k < 7; ++k) {
            dev[k] = user[k] ? h->io + off : nullptr;
            off += (k == 0 ? h->N : 1) * S;
        }
    }
    cudaError_t e = dispatch(h->N, h->precision, [&](auto n, auto pr) {
        return launch_export<decltype(n)::value, decltype(pr)>(h->P, h->pop[h->cur], h->aux[h->cur], dev[0], dev[1],
                                                               dev[2], dev[3], dev[4], dev[5], dev[6], h->stream);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "export kernel");
    if (where == LBM_HOST) {
        for (int k = 0; k < 7; ++k)
            if (user[k])
                LBM_CUDA_TRY(h, cudaMemcpyAsync(user[k], dev[k], (k == 0 ? h->N : 1) * plane_bytes(h),
                                                cudaMemcpyDeviceToHost, h->stream));
        LBM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    }
    return LBM_OK;
}

int lbm_get_diagnostics(lbm_handle* h, lbm_diag* out)
{
    const lbm::TraceRange trace_range("lbm_get_diagnostics");
    if (!h || !out) return fail(h, LBM_EINVAL, "NULL argument");
    if (!h->ready) return fail(h, LBM_ESTATE, "lbm_set_fields has not been called");
    LBM_CUDA_TRY(h, cudaSetDevice(h->device));
    double d[2 * LBM_MAXN + 2];
    int rc = run_diag(h, d);
    if (rc != LBM_OK) return rc;
    std::memset(out, 0, sizeof *out);
    for (int p = 0; p < h->N; ++p) {
        out->mass[p] = d[p];
        out->solid[p] = d[h->N + p];
    }
    out->max_sum_dev = d[2 * h->N];
    out->nonfinite = (long long)d[2 * h->N + 1];
    out->steps = h->steps;
    return LBM_OK;
}

int lbm_save_state(lbm_handle* h, void* buf, size_t* bytes)
{
    const lbm::TraceRange trace_range("lbm_save_state");
    if (!h || !bytes) return fail(h, LBM_EINVAL, "NULL argument");
    const size_t need = sizeof(long long) + h->pop_bytes + h->aux_bytes;
    if (!buf) {
        *bytes = need;
        return LBM_OK;
    }
    if (!h->ready) return fail(h, LBM_ESTATE, "lbm_set_fields has not been called");
    if (*bytes < need) return fail(h, LBM_EINVAL, "buffer too small");
    LBM_CUDA_TRY(h, cudaSetDevice(h->device));
    char* b = (char*)buf;
    std::memcpy(b, &h->steps, sizeof(long long));
    LBM_CUDA_TRY(h, cudaMemcpyAsync(b + sizeof(long long), h->pop[h->cur], h->pop_bytes, cudaMemcpyDeviceToHost,
                                    h->stream));
    LBM_CUDA_TRY(h, cudaMemcpyAsync(b + sizeof(long long) + h->pop_bytes, h->aux[h->cur], h->aux_bytes,
                                    cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    *bytes = need;
    return LBM_OK;
}

int lbm_load_state(lbm_handle* h, const void* buf, size_t bytes)
{
    const lbm::TraceRange trace_range("lbm_load_state");
    if (!h || !buf) return fail(h, LBM_EINVAL, "NULL argument");
    const size_t need = sizeof(long long) + h->pop_bytes + h->aux_bytes;
    if (bytes != need) return fail(h, LBM_EINVAL, "state size does not match this handle");
    LBM_CUDA_TRY(h, cudaSetDevice(h->device));
    const char* b = (const char*)buf;
    long long steps;
    std::memcpy(&steps, b, sizeof(long long));
    h->cur = 0;
    LBM_CUDA_TRY(h, cudaMemcpyAsync(h->pop[0], b + sizeof(long long), h->pop_bytes, cudaMemcpyHostToDevice,
                                    h->stream));
    LBM_CUDA_TRY(h, cudaMemcpyAsync(h->aux[0], b + sizeof(long long) + h->pop_bytes, h->aux_bytes,
                                    cudaMemcpyHostToDevice, h->stream));
    LBM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->steps = steps;
    h->ready = true;
    return LBM_OK;
}

long long lbm_get_steps(const lbm_handle* h) { return h ? h->steps : -1; }

int lbm_debug_bounds(lbm_handle* h, long long* out3)
{
    if (!h || !out3) return fail(h, LBM_EINVAL, "NULL argument");
#ifdef LBM_CHECK_BOUNDS
    unsigned long long v[3];
    LBM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    LBM_CUDA_TRY(h, cudaMemcpy(v, h->dbg, sizeof v, cudaMemcpyDeviceToHost));
    for (int k = 0; k < 3; ++k) out3[k] = (long long)v[k];
    return LBM_OK;
#else
    return fail(h, LBM_EINVAL, "library built without LBM_CHECK_BOUNDS");
#endif
}

const char* lbm_last_error(const lbm_handle* h)
{
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

void lbm_destroy(lbm_handle* h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    free_all(h);
    delete h;
}

}  // extern "C"
