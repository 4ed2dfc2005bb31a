// bap_internal.cuh -- device-side structures and building blocks of the nested Monte Carlo
// library (Doan et al., INRIA RR-6530, 2008).  Private to the library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bap.h"

namespace bap {

constexpr int MAXD = BAP_MAX_D;
constexpr int MAXF = MAXD + 1;            // CMC features: d prices + the payoff
constexpr int MAXDATES = BAP_MAX_DATES;
// Boundary coefficients: the full quadratic in d-1 <= 9 variables (55), or the full cubic in
// d-1 <= 5 variables (56; cubic boundaries are offered up to d = MAXD_CUBIC).
constexpr int MAXD_CUBIC = 6;
constexpr int MAXCOEF = 56;
constexpr int WARP = 32;

enum Purpose : uint32_t { P_IZ = 1, P_CMC = 2, P_TRAIN = 3, P_PRICE = 4 };
enum RuleKind : int { R_NONE = 0, R_IZ = 1, R_CMC = 2 };
// Bounds checks of the checked build (compiled with -DBAP_CHECKS, a debug aid in place of a
// sanitizer): bap_check(cond, code, buf) counts a failed condition in buf[0], keeps the first
// code in buf[1] and returns false so that the caller skips the access.  In the normal build it
// is the constant true and costs nothing.
#ifdef BAP_CHECKS
__device__ __forceinline__ bool bap_check(bool cond, int code, unsigned long long* buf) {
    if (!cond && buf) {
        atomicAdd(buf, 1ULL);
        atomicCAS(buf + 1, 0ULL, (unsigned long long)code);
    }
    return cond;
}
#else
__device__ __forceinline__ constexpr bool bap_check(bool, int, unsigned long long*) { return true; }
#endif

// Kernel selectors (not rule kinds): the cooperative kernel that runs all Newton passes of a date,
// and the I&Z kernels for cubic boundaries (one pass, cooperative).
constexpr int R_NEWTON_COOP = 3;
constexpr int R_IZ3 = 4;
constexpr int R_NEWTON_COOP3 = 5;
enum Mode : int { MODE_SUMS = 0, MODE_NEWTON = 1, MODE_LABEL = 2, MODE_TRACE = 3 };
enum ItemStatus : int { ST_OK = 0, ST_NOCONV = 1, ST_NOROOT = 2 };

// Market model in device memory: FP64 master values and the per-date stepping constants in
// log2 units, in FP32 and FP64 (Section 2.2: correlated GBM, rate r, yields delta_i).
struct DevModel {
    int d, n_dates, payoff, uniform_dates;
    double r, K;
    double S0[MAXD], sigma[MAXD], delta[MAXD], w[MAXD];
    double t[MAXDATES + 1];
    double L[MAXD * MAXD];                 // lower Cholesky factor of rho, FP64
    double drift2[MAXDATES + 1][MAXD];     // (r - delta_q - sigma_q^2/2) (t_k - t_{k-1}) / ln 2
    double vol2[MAXDATES + 1][MAXD];       // sigma_q sqrt(t_k - t_{k-1}) / ln 2
};

// Iteration state of a Newton loop whose passes are decided on the device: the index of the
// next pass.
struct IterState {
    int iter;
    int pad[3];
};

// Newton state of one I&Z boundary point (FP64, the Newton iterations of Section 2.3).
struct ItemState {
    double x, lo, hi, dx_old, dx;
    int iters, status, done, pivot;
};

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds; multipliers 0xD2511F53 and
// 0xCD9E8D57; Weyl key increments 0x9E3779B9 and 0xBB67AE85.  Round keys are precomputed once
// per launch (key = (lo32(seed), hi32(seed) ^ purpose << 24 ^ m)).

struct RoundKeys {
    uint32_t k0[10], k1[10];
};

__host__ __device__ inline RoundKeys make_round_keys(uint64_t seed, uint32_t purpose, uint32_t m) {
    RoundKeys rk;
    uint32_t a = (uint32_t)(seed & 0xffffffffu);
    uint32_t b = (uint32_t)(seed >> 32) ^ (purpose << 24) ^ m;
    for (int r = 0; r < 10; ++r) {
        rk.k0[r] = a;
        rk.k1[r] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return rk;
}

// 32 x 32 -> 64-bit product in one instruction (both halves of the Philox multiply).
__device__ __forceinline__ void mulhilo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
    uint64_t p;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        const RoundKeys& rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0, hi0, lo1, hi1;
        mulhilo(0xD2511F53u, c0, hi0, lo0);
        mulhilo(0xCD9E8D57u, c2, hi1, lo1);
        uint32_t n0 = hi1 ^ c1 ^ rk.k0[r];
        uint32_t n2 = hi0 ^ c3 ^ rk.k1[r];
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// ---------------------------------------------------------------------------------------------
// Single-precision hardware approximations (PTX .approx instructions) and their FP64
// counterparts, selected by the path arithmetic type.

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <typename Real> struct PathMath;

template <> struct PathMath<float> {
    __device__ __forceinline__ static float exp2r(float x) { return ex2_approx(x); }
    // Box-Muller pair from two Philox words: u1 = (v0 + 1) 2^-23, u2 = v1 2^-23.  The angle is
    // taken as 2 pi (u2 - 1/2) in [-pi, pi) (the hardware sine's accurate range) and the sign
    // folded into the radius: cos(2 pi u2) = -cos(2 pi (u2 - 1/2)), same for sin.
    __device__ __forceinline__ static void box_muller(uint32_t w0, uint32_t w1, float& z0,
                                                      float& z1) {
        // 1 + v 2^-23 as a bit pattern: the exponent of 1.0 plus the 23-bit v (no carry; an
        // add of the shifted word, one instruction)
        float u1 = __uint_as_float((w0 >> 9) + 0x3f800000u) - 0.99999988079071044921875f;
        float r = -sqrt_approx(-1.3862943611198906f * lg2_approx(u1));   // -sqrt(-2 ln u1)
        // a = 2 pi (u2 - 1/2) from the bit pattern 1 + u2 in one fused multiply-add
        float a = fmaf(__uint_as_float((w1 >> 9) + 0x3f800000u), 6.283185307179586f,
                       -9.42477796076938f);
        z0 = r * __cosf(a);
        z1 = r * __sinf(a);
    }
};

template <> struct PathMath<double> {
    __device__ __forceinline__ static double exp2r(double x) { return exp2(x); }
    __device__ __forceinline__ static void box_muller(uint32_t w0, uint32_t w1, double& z0,
                                                      double& z1) {
        double u1 = (double)((w0 >> 9) + 1u) * (1.0 / 8388608.0);
        double u2 = (double)(w1 >> 9) * (1.0 / 8388608.0);
        double r = sqrt(-2.0 * log(u1));
        double s, c;
        sincospi(2.0 * u2, &s, &c);
        z0 = r * c;
        z1 = r * s;
    }
};

// The D normals of counter prefix (w0, w1, 4*step): Philox call c gives normals 4c..4c+3,
// words (0,1) -> (cos, sin) pair 0 and words (2,3) -> pair 1.
template <int D, typename Real>
__device__ __forceinline__ void normals(uint32_t w0, uint32_t w1, uint32_t step,
                                        const RoundKeys& rk, Real (&z)[D]) {
#pragma unroll
    for (int c = 0; c < (D + 3) / 4; ++c) {
        uint4 x = philox(w0, w1, 4u * step + (uint32_t)c, 0u, rk);
        Real a, b;
        if (4 * c < D) {
            PathMath<Real>::box_muller(x.x, x.y, a, b);
            z[4 * c] = a;
            if (4 * c + 1 < D) z[4 * c + 1] = b;
        }
        if (4 * c + 2 < D) {
            PathMath<Real>::box_muller(x.z, x.w, a, b);
            z[4 * c + 2] = a;
            if (4 * c + 3 < D) z[4 * c + 3] = b;
        }
    }
}

__host__ __device__ inline int n_basis(int s, int degree) {
    int n = 1;
    if (degree >= 1) n += s;
    if (degree >= 2) n += s * (s + 1) / 2;
    if (degree >= 3) n += s * (s + 1) * (s + 2) / 6;
    return n;
}

// Staged I&Z boundary block for the path kernel: always the full quadratic in all d prices,
// with zero terms for the boundary's pivot asset (lower degrees carry zero coefficients), so
// that the kernel evaluates it on the prices without reordering them; padded to a multiple of 4
// values so that a block is read with 16-byte vector loads.
__host__ __device__ constexpr int iz_stage_stride(int d) {
    return ((1 + d + d * (d + 1) / 2) + 3) & ~3;
}

// The same for a cubic boundary: the full cubic in the d-1 other assets, nested for Horner
// evaluation (see stage_iz_one), padded to a multiple of 4.
__host__ __device__ constexpr int iz_stage_stride3(int d) {
    return ((1 + (d - 1) + (d - 1) * d / 2 + (d - 1) * d * (d + 1) / 6) + 3) & ~3;
}

// Staged stride of a boundary of this degree.
__host__ __device__ constexpr int iz_stride(int d, int degree) {
    return degree >= 3 ? iz_stage_stride3(d) : iz_stage_stride(d);
}

// CMC staged rule record per date (floats or doubles; integers stored as bit patterns):
// [0] F0 = sum of the constant stumps' votes, [1] the overflow mask (bit f: feature f has more
// than CMC_SLOTS - 1 distinct thresholds), [2..3] spare, then one fixed block of 2 CMC_SLOTS
// values per feature f at CMC_HEAD + 2 CMC_SLOTS f: its distinct sorted thresholds t_f[0..U-1]
// padded with +inf to CMC_SLOTS, then the step table T_f[0..U] (padded with T_f[U]), where
// T_f[c] is the sum of the feature's stump votes at a value above exactly c of its distinct
// thresholds.  F(S) = F0 + sum_f T_f[#{t_f < x_f}]; the count is a fixed five-level binary search
// within the block, so every value read sits at a constant offset from the record.  A feature
// with U >= CMC_SLOTS distinct thresholds keeps in its block [offset, U] (its first two
// values) and its thresholds and U + 1 steps in the overflow area after the blocks.
// Length: the blocks, and at most 2 U + 1 <= 2 n_f + 1 overflow values per feature; odd, so that
// the records of different dates start in different shared-memory banks.
// An integer stored in a float or double record slot as a bit pattern, and read back.
__device__ __forceinline__ void put_int_as(float* p, int v) { *p = __int_as_float(v); }
__device__ __forceinline__ void put_int_as(double* p, int v) { *p = __longlong_as_double((long long)v); }
__device__ __forceinline__ int get_int_as(float v) { return __float_as_int(v); }
__device__ __forceinline__ int get_int_as(double v) { return (int)__double_as_longlong(v); }

constexpr int CMC_SLOTS = 32;
constexpr int CMC_HEAD = 4;
__host__ __device__ inline int cmc_record_len(int nF, int max_stumps) {
    return (CMC_HEAD + 2 * CMC_SLOTS * nF + 2 * max_stumps + nF) | 1;
}
// The part of a record a path kernel stages in shared memory: the head and the fixed blocks
// (the overflow area stays in global memory), padded to an odd row length.
__host__ __device__ constexpr int cmc_staged_len(int nF) {
    return (CMC_HEAD + 2 * CMC_SLOTS * nF) | 1;
}

}  // namespace bap
