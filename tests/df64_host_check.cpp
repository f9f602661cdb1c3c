// Host check of the double-word arithmetic (paper_2603_22902_gb300/csrc/lbm_df64.cuh) and
// of the double-word D2Q9 weights (lbm_lattice.cuh).  The CUDA rounding intrinsics are
// replaced by their IEEE definitions (single precision, round to nearest, FMA with one
// rounding); compile with -ffp-contract=off so the compiler fuses nothing itself.  Exact
// references come from long double (x86: 64-bit significand, enough for every product
// and sum of two double words checked here; aarch64: 113 bits).  Prints one line
// "name value" per measured maximum.
#include <cmath>
#include <cstdio>
#include <random>

#define __host__
#define __device__
#define __forceinline__ inline
#define __align__(n) alignas(n)
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
static inline float __frcp_rn(float a) { return 1.0f / a; }
// the hardware reciprocal square root is an approximation: model one 2^-22 off
static inline float rsqrtf(float a) { return (float)(1.0 / std::sqrt((double)a)) * (1.0f + 0x1p-22f); }

#include "../paper_2603_22902_gb300/csrc/lbm_df64.cuh"
#include "../paper_2603_22902_gb300/csrc/lbm_lattice.cuh"

using namespace lbm;
typedef long double LD;
static LD v(df64 a) { return (LD)a.hi + (LD)a.lo; }

int main()
{
    std::mt19937_64 gen(20260322);
    std::uniform_real_distribution<double> U(-1.0, 1.0), E(-6.0, 4.0);
    auto draw = [&]() { return U(gen) * std::pow(10.0, E(gen)); };
    double conv = 0, add = 0, mul = 0, mulf = 0, div = 0, rsq = 0, chain = 0, tiny = 0;
    long bad_cmp = 0, nonfinite = 0;
    for (int k = 0; k < 400000; ++k) {
        const double a = draw(), c = draw();
        double b = draw();
        if (k % 4 == 0) b = -a * (1.0 + 1e-7 * U(gen));  // near cancellation
        const df64 x(a), y(b), z(c);
        conv = std::fmax(conv, (double)(std::fabs(v(x) - (LD)a) / std::fabs((LD)a)));
        const LD xs = v(x), ys = v(y), zs = v(z);
        add = std::fmax(add, (double)(std::fabs(v(x + y) - (xs + ys)) / (std::fabs(xs) + std::fabs(ys))));
        mul = std::fmax(mul, (double)(std::fabs(v(x * y) - xs * ys) / std::fabs(xs * ys)));
        const float f = (float)c;
        mulf = std::fmax(mulf, (double)(std::fabs(v(x * f) - xs * (LD)f) / std::fabs(xs * (LD)f)));
        div = std::fmax(div, (double)(std::fabs(v(x / z) - xs / zs) / std::fabs(xs / zs)));
        const LD p = xs * ys;
        chain = std::fmax(chain, (double)(std::fabs(v(x * y + z) - (p + zs)) / (std::fabs(p) + std::fabs(zs))));
        const df64 ax(std::fabs(a));
        const LD r = 1.0L / std::sqrt(v(ax));
        rsq = std::fmax(rsq, (double)(std::fabs(v(rrsqrt(ax)) - r) / r));
        // an argument below FP32's normal range (scaled internally)
        // (the step calls it only on a strictly positive |G|^2)
        const df64 t(std::fabs(a) * 1e-38);
        if (t.hi > 0.0f) {
            const df64 rt = rrsqrt(t);
            if (!std::isfinite(rt.hi) || !std::isfinite(rt.lo)) ++nonfinite;
            else tiny = std::fmax(tiny, (double)(std::fabs(v(rt) - 1.0L / std::sqrt(v(t))) * std::sqrt(v(t))));
        }
        if ((x < y) != (xs < ys) || (x > y) != (xs > ys)) ++bad_cmp;
    }
    // D2Q9 weights
    LD wsum = 0, wdev = 0;
    for (int i = 0; i < 9; ++i) {
        const df64 w = wgt_r<df64>(i);
        const LD exact = i == 0 ? 4.0L / 9.0L : (i < 5 ? 1.0L / 9.0L : 1.0L / 36.0L);
        wsum += v(w);
        wdev = std::fmax((double)wdev, (double)(std::fabs(v(w) - exact) / exact));
        if ((double)w.hi + (double)w.lo != (double)v(w)) ++bad_cmp;
    }
    std::printf("conv %.6e\nadd %.6e\nmul %.6e\nmulf %.6e\ndiv %.6e\nchain %.6e\nrsqrt %.6e\ntiny_rsqrt %.6e\n", conv,
                add, mul, mulf, div, chain, rsq, tiny);
    std::printf("nonfinite %ld\nbad_cmp %ld\nweight_sum_minus_1 %.6Le\nweight_dev %.6Le\n", nonfinite, bad_cmp,
                wsum - 1.0L, wdev);
    return 0;
}
