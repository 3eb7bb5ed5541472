// pair_physics.cuh -- per-pair arithmetic of the method used by the pair
// kernels: pair smoothing length, the transport-velocity limiter (Eq. 15),
// one neighbour's contribution to the pressure (Eq. 3, 5-6) and viscous
// (Eq. 7) accelerations and to the residual of Eq. 14 in the FP64 form (the
// FP32 form is pair_force32 in k_pair32.cu), and the block reduction of the
// FP64 diagnostics partials.
//
// Readings of the paper: e_ij points from i to j (Riemann states U_l, U_r);
// grad W_ij is grad_i W_ij = W'(r) (x_i - x_j)/r; V_j = m_j / rho_j;
// rho_bar = (rho_i + rho_j)/2, c_bar = c; a wall neighbour stands in with
// rho_j = rho_i, p_j = p_i (so V_j = m_j / rho_i) and its prescribed velocity.
#pragma once

#include "common.cuh"

namespace sphtv {

template <typename Real>
__device__ __forceinline__ Real pair_h(const Consts<Real>& K, Real hi, Real hj)
{
    return K.h_pair_max ? (hi > hj ? hi : hj) : Real(0.5) * (hi + hj);
}

template <typename Real>
__device__ __forceinline__ Real tv_limiter(const Consts<Real>& K, Real s)
{
    if (K.tv_mode == SPH_TV_OFF) return Real(0);
    if (K.tv_mode == SPH_TV_UNLIMITED || K.tv_mode == SPH_TV_BACKGROUND) return Real(1);
    if (s > K.tv_thresh) {
        Real t = K.tv_C * s;
        return t < Real(1) ? t : Real(1);
    }
    return Real(0);
}

// Per-particle values of i shared by all pairs of i in the FP64 force pass.
// C is a constant factor of W'/r that the pass takes out of the pair sums
// (-5 a_D h^-(D+2) at uniform resolution, where W'/r = C t^3; else 1).
struct PairI64 {
    double w;          // rho_i - rho0
    double inv_rho;    // 1 / rho_i
    double hp;         // p_i / 2 = (c^2 / 2) w_i
    double crho;       // (c/2)(rho0 + w_i / 2): (c/2) rho_bar = crho + (c/4) w_j
    double m2_ir;      // -2 C / rho_i
    double eta_ir;     // 2 eta C / rho_i
};

__device__ __forceinline__ PairI64 pair_i64(const Consts<double>& K, double w, double inv_rho, double C)
{
    PairI64 I;
    I.w = w;
    I.inv_rho = inv_rho;
    I.hp = (0.5 * K.c2) * w;
    I.crho = (0.5 * K.c) * (K.rho0 + 0.5 * w);
    I.m2_ir = (-2.0 * C) * inv_rho;
    I.eta_ir = (K.two_eta * C) * inv_rho;
    return I;
}

// min(max(x, 0), 1) by the sign and order of the binary64 bit pattern (the
// order of non-negative doubles is that of their patterns): integer selects
// instead of two FP64 comparisons.
__device__ __forceinline__ double clamp01(double x)
{
    const long long b = __double_as_longlong(x);
    if (b < 0) return 0.0;
    if (b >= 0x3ff0000000000000LL) return 1.0;
    return x;
}

// w = +inf marks a wall particle in the velocity record (a bit test: no
// FP64 comparison).
__device__ __forceinline__ bool is_wall(double w)
{
    return (__double_as_longlong(w) & 0x7fffffffffffffffLL) == 0x7ff0000000000000LL;
}

// Contribution of neighbour j to a_i and R_i in the FP64 form: Eq. 3
// (pressure, with P* of Eq. 5-6), Eq. 7 (viscous) and the residual of
// Eq. 14, arranged for the FP64 pipe (1/74 of the FP32 rate here): P* from
// the density deviations (p_i + p_j = c^2 (w_i + w_j), rho_bar = rho0 +
// (w_i + w_j)/2), the limiter's clamp on the integer ALU, and one product
// V_j g that the pressure, viscous and residual terms share.  rv = x_i -
// x_j, inv_r = 1/r, g = W'(r, h_ij) / (r C); w_j = rho_j - rho0 and V_j =
// m_j / rho_j, for a wall neighbour w_i and m_j / rho_i (the caller
// substitutes them).  acc_R collects R_i / C.
template <int DIM>
__device__ __forceinline__ void pair_force64(const Consts<double>& K, const PairI64& I, const double* rv,
                                             double inv_r, double g, const double* vi, const double* vj,
                                             double w_j, double V_j, PlainD* acc_a, PlainD* acc_R)
{
    double dv[3] = {0.0, 0.0, 0.0};
    double dvr = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        dv[d] = vi[d] - vj[d];
        dvr += dv[d] * rv[d];
    }
    const double du = -dvr * inv_r;                                   // U_l - U_r
    const double beta = clamp01((K.beta_slope * K.inv_c) * du);
    const double hpsum = fma(0.5 * K.c2, w_j, I.hp);                   // (p_i + p_j) / 2
    const double crhobar = fma(0.25 * K.c, w_j, I.crho);               // (c/2) rho_bar
    const double pstar = fma(beta * du, crhobar, hpsum);
    const double vw = V_j * g;                                        // V_j W'/(r C)
    const double cpw = I.m2_ir * (vw * pstar);                        // -2 m_j P* / (rho_i rho_j) W'/r
    const double cv = I.eta_ir * vw;                                  // 2 eta m_j / (rho_i rho_j) W'/r
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        acc_a[d].s = fma(cpw, rv[d], acc_a[d].s);
        acc_a[d].s = fma(cv, dv[d], acc_a[d].s);
        acc_R[d].s = fma(vw, rv[d], acc_R[d].s);
    }
}

// Free-stream forcing rate of the fringe region technique (Nordstrom, Nordin
// & Henningson 1999): lambda(x) = lambda_max [S((x - x0)/rise) - S((x -
// x1)/fall + 1)] with the smooth step S(t) = 1/(1 + exp(1/(t - 1) + 1/t)) on
// (0, 1), 0 below, 1 above; the acceleration gets lambda(x) (U_inf - v).
template <typename Real>
__device__ __forceinline__ Real fringe_step(Real t)
{
    if (t <= Real(0)) return Real(0);
    if (t >= Real(1)) return Real(1);
    return Real(1) / (Real(1) + exp(Real(1) / (t - Real(1)) + Real(1) / t));
}

template <typename Real>
__device__ __forceinline__ Real fringe_rate(const Consts<Real>& K, Real x)
{
    return K.fr_lambda *
           (fringe_step<Real>((x - K.fr_x[0]) / K.fr_x[2]) - fringe_step<Real>((x - K.fr_x[1]) / K.fr_x[3] + Real(1)));
}

// Block reduction of the diagnostics partials into out_block (layout: 0
// mass, 1-3 momentum, 4 KE, 5 n_chi, 6 max|v|, 7 max|v + dr/dt|, 8 max|dr|,
// 9-11 the fluid's momentum rate from its pair terms, sum m_i (a_i - g -
// forcing), whose negative is the force on the walls; zero unless the pass
// computes it).  FIRST: per-particle values of a pair pass, with
// slot 5 a 0/1 flag and slots 6-8 the SQUARES of the magnitudes: the square
// root of the largest square is the largest magnitude (both correctly
// rounded), so one root per block replaces one per particle.  Otherwise:
// rows of partials to fold.  The sums are FP64 shuffle trees in a fixed
// order.  With FIRST the flags are counted with a ballot and the maxima of
// the non-negative squares are integer maxima of their bit patterns (a NaN
// counts as 0, as fmax ignores it), which keeps both off the FP64 pipe
// (1/74 of the FP32 rate on this part).  sums = false (the same for every
// thread of the grid) when the caller's sums are all zero: they are skipped.
template <bool FIRST>
__device__ __forceinline__ void block_partials(double* vals, double* out_block, bool sums = true, bool body = false)
{
    __shared__ double sh[32][kNPart];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    constexpr int kSums = FIRST ? 5 : 9;
    if (FIRST && !sums) {
        // the caller's sums are all zero (uniform over the grid): skip them
        if (lane == 0)
            for (int k = 0; k < 5; ++k) sh[w][k] = 0.0;
    } else if (FIRST) {
        // the five sums as a transposing reduction: at each of the first three
        // levels a lane keeps half of its values and adds its partner's copy
        // of them (4 + 2 + 1 additions instead of 5 per level), then the last
        // two levels reduce one value per group of four lanes; value g ends in
        // lane 4 g (eight slots, the last three zero)
        double v8[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v8[k] = k < 5 ? vals[k] : 0.0;
        const bool hi16 = lane & 16, hi8 = lane & 8, hi4 = lane & 4;
        double a4[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const double send = hi16 ? v8[j] : v8[4 + j];
            const double keep = hi16 ? v8[4 + j] : v8[j];
            a4[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
        double a2[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const double send = hi8 ? a4[j] : a4[2 + j];
            const double keep = hi8 ? a4[2 + j] : a4[j];
            a2[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
        double a1;
        {
            const double send = hi4 ? a2[0] : a2[1];
            const double keep = hi4 ? a2[1] : a2[0];
            a1 = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
        a1 += __shfl_xor_sync(0xffffffffu, a1, 2);
        a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
        const int g = (lane >> 2);   // value index held by this group of four lanes
        if ((lane & 3) == 0 && g < 5) sh[w][g] = a1;
    } else {
#pragma unroll
        for (int k = 0; k < kSums; ++k) {
            double x = vals[k];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                double y = __shfl_down_sync(0xffffffffu, x, off);
                x = (k >= 6 && k <= 8) ? fmax(x, y) : x + y;
            }
            if (lane == 0) sh[w][k] = x;
        }
    }
    // slots 9-11 (uniform over the grid: body is the same for every thread)
    if (body || !FIRST) {
#pragma unroll
        for (int k = 9; k < 12; ++k) {
            double x = vals[k];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
            if (lane == 0) sh[w][k] = x;
        }
    } else if (lane == 0) {
        for (int k = 9; k < 12; ++k) sh[w][k] = 0.0;
    }
    if (FIRST) {
        const unsigned flags = __ballot_sync(0xffffffffu, __double_as_longlong(vals[5]) != 0);
        if (lane == 0) sh[w][5] = (double)__popc(flags);
#pragma unroll
        for (int k = 6; k <= 8; ++k) {
            long long b = __double_as_longlong(vals[k]);
            if ((b & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL) b = 0;      // NaN
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) b = max(b, __shfl_down_sync(0xffffffffu, b, off));
            if (lane == 0) sh[w][k] = __longlong_as_double(b);
        }
    }
    __syncthreads();
    if (threadIdx.x < kNPart) {
        const int k = threadIdx.x;
        double x = sh[0][k];
        for (int t = 1; t < nw; ++t) x = (k >= 6 && k <= 8) ? fmax(x, sh[t][k]) : x + sh[t][k];
        if (FIRST && k >= 6 && k <= 8) x = sqrt(x);
        out_block[k] = x;
    }
}


}  // namespace sphtv
