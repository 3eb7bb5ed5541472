// pair_physics.cuh -- the per-pair arithmetic of the method, shared by the
// FP64 and FP32 pair kernels: pair smoothing length, the transport-velocity
// limiter (Eq. 15), one neighbour's contribution to the pressure (Eq. 3,
// 5-6) and viscous (Eq. 7) accelerations and to the residual of Eq. 14, and
// the block reduction of the FP64 diagnostics partials.
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

// Contribution of neighbour j to a_i and R_i (rv = x_i - x_j, inv_r = 1/r,
// dwr = W'(r, h_ij)/r, inv_rho_i = 1/rho_i, inv_rho_j = 1/rho_j computed
// once per particle by the density pass, unused for a wall j).  Adds into
// the caller's accumulators.  The one reciprocal of each density serves both
// V_j and 1/(rho_i rho_j) (FP64 division is costly on this GPU); products of
// constants (eta_R / c, c / 2) are written so that the compiler takes them
// out of the neighbour loop.
template <typename Real, int DIM, typename Acc>
__device__ __forceinline__ void pair_force(const Consts<Real>& K, const Real* rv, Real inv_r, Real dwr,
                                           const Real* vi, Real rho_i, Real inv_rho_i, Real p_i, const Real* vj,
                                           Real w_j, Real m_j, Real inv_rho_jd, Acc* acc_a, Acc* acc_R)
{
    const bool wall = isinf(w_j);
    const Real rho_j = wall ? rho_i : K.rho0 + w_j;
    const Real inv_rho_j = wall ? inv_rho_i : inv_rho_jd;
    const Real p_j = wall ? p_i : K.c2 * w_j;
    // U_l - U_r = (v_i - v_j).e_ij with e_ij = -rv / r: one dot product with
    // the velocity difference, which the viscous term uses as well
    Real dv[3] = {Real(0), Real(0), Real(0)};
    Real dvr = Real(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        dv[d] = vi[d] - vj[d];
        dvr += dv[d] * rv[d];
    }
    const Real du = -dvr * inv_r;
    Real beta = (K.beta_slope * K.inv_c) * du;
    beta = beta > Real(0) ? beta : Real(0);
    beta = beta < Real(1) ? beta : Real(1);
    const Real rhobar = Real(0.5) * (rho_i + rho_j);
    const Real pstar = Real(0.5) * (p_i + p_j) + (Real(0.5) * K.c) * (beta * rhobar * du);
    const Real mr = m_j * (inv_rho_i * inv_rho_j);         // m_j / (rho_i rho_j)
    const Real cpw = Real(-2) * mr * pstar * dwr;          // pressure: cp W'/r
    const Real cv = K.two_eta * mr * dwr;                  // viscous
    const Real vw = m_j * inv_rho_j * dwr;                 // residual: V_j W'/r
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        acc_a[d].add(cpw * rv[d] + cv * dv[d]);
        acc_R[d].add(vw * rv[d]);
    }
}

// Block reduction of the diagnostics partials into out_block (layout: 0
// mass, 1-3 momentum, 4 KE, 5 n_chi, 6 max|v|, 7 max|v + dr/dt|, 8 max|dr|,
// 9 unused, written 0).  FIRST: per-particle values of a pair pass, with
// slot 5 a 0/1 flag and slots 6-8 the SQUARES of the magnitudes: the square
// root of the largest square is the largest magnitude (both correctly
// rounded), so one root per block replaces one per particle.  Otherwise:
// rows of partials to fold.  The sums are FP64 shuffle trees in a fixed
// order.  With FIRST the flags are counted with a ballot and the maxima of
// the non-negative squares are integer maxima of their bit patterns (a NaN
// counts as 0, as fmax ignores it), which keeps both off the FP64 pipe
// (1/64 of the FP32 rate on this part).  sums = false (the same for every
// thread of the grid) when the caller's sums are all zero: they are skipped.
template <bool FIRST>
__device__ __forceinline__ void block_partials(double* vals, double* out_block, bool sums = true)
{
    __shared__ double sh[32][kNPart];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    constexpr int kSums = FIRST ? 5 : 9;
    if (FIRST && !sums) {
        // the caller's sums are all zero (uniform over the grid): skip them
        if (lane == 0)
            for (int k = 0; k < 5; ++k) sh[w][k] = 0.0;
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
    if (threadIdx.x < 9) {
        const int k = threadIdx.x;
        double x = sh[0][k];
        for (int t = 1; t < nw; ++t) x = (k >= 6 && k <= 8) ? fmax(x, sh[t][k]) : x + sh[t][k];
        if (FIRST && k >= 6) x = sqrt(x);
        out_block[k] = x;
    } else if (threadIdx.x == 9) {
        out_block[9] = 0.0;
    }
}


}  // namespace sphtv
