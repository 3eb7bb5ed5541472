// k_adjoint.cu -- reverse-mode adjoint of the libsphtv step (not in the
// paper; derivatives of Eq. 2-8 and 14-16 taken by hand), with each step's
// neighbour set and step size frozen.
//
// One reverse step, in the cell-sorted order of the forward step it undoes
// (forward values come from a per-step tape), cotangents kept in FP64 in the
// caller's particle order:
//   k_adj_prep    : A_i = abar'_i + dt/2 vbar'_i (the closing kick), and the
//                   cotangent of the residual R_i from that of the
//                   displacement dr_i = xi chi(s) H^2 R_i, s = H^2 |R_i|^2
//   k_adj_pairs   : gather form of the pair terms: particle k collects the
//                   derivatives of its own sums (k as i) and of each fluid
//                   neighbour's sums (k as j), so no atomics are needed;
//                   also the density cotangent and d/d(eta) partials
//   k_adj_density : the density sum rho_k = rho0 sum_j W_kj / sigma0_k, then
//                   the reverse of the drift and the opening kick; its first
//                   block adds the step's d/d(eta) (fixed-order reduction)
//
// Subgradients: d beta/d dU = eta_R / c inside 0 < eta_R dU / c < 1, else 0
// (Eq. 6); d chi/d s = C inside thresh < s < 1/C, else 0 (Eq. 15).
#include <type_traits>

#include "common.cuh"
#include "launch.h"
#include "pair_physics.cuh"
#include "pair_walk.cuh"

namespace sphtv {

template <typename Real>
using AccOf = typename std::conditional<sizeof(Real) == 4, KSum, PlainD>::type;

// The cotangents Abar_k and Rbar_k of a particle as one record of
// kAbStride<DIM> values ({Abar, Rbar}, padded to a whole number of 16-byte
// vectors in the FP32 form), so that the pair kernel gathers a neighbour's
// with one or two vector loads.
template <int DIM> constexpr int kAbStride = DIM == 3 ? 8 : 4;

template <typename Real, int DIM>
__device__ __forceinline__ void load_ab(const Real* __restrict__ AR, int k, Real* Ab, Real* Rb)
{
    const Real* p = AR + (size_t)k * kAbStride<DIM>;
    if constexpr (sizeof(Real) == 4) {
        const float4 a = *(const float4*)p;
        if (DIM == 2) {
            Ab[0] = a.x; Ab[1] = a.y; Rb[0] = a.z; Rb[1] = a.w;
        } else {
            const float4 b = *(const float4*)(p + 4);
            Ab[0] = a.x; Ab[1] = a.y; Ab[2] = a.z; Rb[0] = a.w; Rb[1] = b.x; Rb[2] = b.y;
        }
    } else {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            Ab[d] = p[d];
            Rb[d] = p[DIM + d];
        }
    }
}

// Forward values of one step.
template <typename Real>
struct Tape {
    const int32_t* id;
    const int8_t* kind;
    const double* x;       // [DIM][n] positions after the drift (FP64)
    const double* h;
    const double* m;
    const double* s0;
    const typename Vec4<Real>::T* vr;   // {half-step v, rho - rho0 (+inf: wall)}
    const Real* R;         // [DIM][n] residual
    const int32_t* start;  // cell ranges
    const float4* pos4;    // FP32 form: cell-relative positions
    const int32_t* cell;   // FP32 form: cell of each particle
    const double* dt;      // step size of the step
    const uint32_t* nbl;   // FP32 form: the step's force-neighbour list (transposed), or null
    const int32_t* nbc;    // and its counts
};

// Visit the neighbours j != k of particle k with 0 < r < 2 h_kj, decided
// exactly as the forward pass decided them: f(j, rv[3] = x_k - x_j, r, 1/r)
// (FP32 form: 1/r from rsqrt and r = r^2/r, as the forward force pass takes
// them; FP64 form: r = sqrt(r^2), 1/r = 1/r).
template <typename Real, int DIM, typename F>
__device__ __forceinline__ void adj_visit(int n, int k, const Grid& G, const Consts<Real>& K, const Tape<Real>& T,
                                          F& f)
{
    if constexpr (sizeof(Real) == 4) {
        const float4 pk = T.pos4[k];
        const float ok[3] = {pk.x, pk.y, pk.z};
        const int cnt = T.nbl ? T.nbc[k] : 0;
        if (T.nbl && cnt <= list_capacity(DIM)) {
            // FP32 form: the forward density pass's list of the step, which
            // holds exactly the pairs its walk accepted, in the walk's order;
            // the pair vector and r^2 with the walk's arithmetic
            const float ex = G.edgef[0], ey = G.edgef[1], ez = G.edgef[2];
            // the entry two ahead and the neighbour's position one ahead in flight
            const uint32_t* lp = T.nbl + k;
            uint32_t e_n = cnt > 0 ? lp[0] : 0u;
            uint32_t e_nn = cnt > 1 ? lp[n] : 0u;
            float4 p_n = T.pos4[e_n >> kCodeBits];
            lp += 2 * (size_t)n;
            for (int q = 0; q < cnt; ++q, lp += n) {
                const uint32_t e = e_n;
                const float4 pj = p_n;
                e_n = e_nn;
                if (q + 1 < cnt) p_n = T.pos4[e_n >> kCodeBits];
                e_nn = q + 2 < cnt ? *lp : 0u;
                const int j = (int)(e >> kCodeBits);
                const uint32_t code = e & ((1u << kCodeBits) - 1u);
                const int dx = (int)(code % kSide) - kStencilR, dy = (int)((code / kSide) % kSide) - kStencilR,
                          dz = (int)(code / (kSide * kSide)) - kStencilR;
                const float2 rxy = __fadd2_rn(__ffma2_rn(make_float2(pj.x, pj.y), make_float2(-1.f, -1.f),
                                                         make_float2(ok[0], ok[1])),
                                              make_float2(-(float)dx * ex, -(float)dy * ey));
                const float2 qq = __fmul2_rn(rxy, rxy);
                float r2 = qq.x + qq.y;
                float rz = 0.f;
                if (DIM == 3) {
                    rz = (ok[2] - pj.z) + -(float)dz * ez;
                    r2 = fmaf(rz, rz, r2);
                }
                const Real rv[3] = {rxy.x, rxy.y, rz};
                const float inv_r = rsqrtf(r2);
                f(j, rv, r2 * inv_r, inv_r);
            }
            return;
        }
        // more neighbours than the list holds (or no list): the clipped row
        // walk of the forward density pass, with its arithmetic for r^2, so
        // the pairs are exactly the forward's (same order as the cell scan
        // below)
        const float hk = (float)T.h[k];
        const float reach = K.uniform_h ? 2.f * K.h_u : 2.f * pair_h(K, hk, K.h_u);
        auto g = [&](int j, uint32_t, const float4&, float r2, float rx, float ry, float rz) {
            float lim;
            if (K.uniform_h) lim = K.four_h2_u;
            else {
                const float hh = pair_h(K, hk, (float)T.h[j]);
                lim = 4.f * hh * hh;
            }
            if (!(r2 < lim) || !(r2 > 0.f)) return;
            const Real rv[3] = {rx, ry, rz};
            const float inv_r = rsqrtf(r2);
            f(j, rv, r2 * inv_r, inv_r);
        };
        for_candidates_rows<DIM, false>(ok, reach, T.cell[k], G, T.start, T.cell, T.pos4, g);
    } else {
        // FP64 form: the exact test of the forward pass (minimum image,
        // sqrt(r^2) < 2 h_kj)
        const int SR = G.R, zr = DIM == 3 ? SR : 0;
        int c[3];
        for (int d = 0; d < 3; ++d) c[d] = d < DIM ? cell_coord(G, T.x[(size_t)d * n + k], d) : 0;
        for (int dz = -zr; dz <= zr; ++dz) {
            int cz = DIM == 3 ? cell_step(G, c[2], dz, 2) : 0;
            if (cz < 0) continue;
            for (int dy = -SR; dy <= SR; ++dy) {
                int cy = cell_step(G, c[1], dy, 1);
                if (cy < 0) continue;
                for (int dx = -SR; dx <= SR; ++dx) {
                    int cx = cell_step(G, c[0], dx, 0);
                    if (cx < 0) continue;
                    const int cell = cx + G.nc[0] * (cy + G.nc[1] * cz);
                    for (int j = T.start[cell]; j < T.start[cell + 1]; ++j) {
                        if (j == k) continue;
                        Real rv[3] = {0, 0, 0};
                        double r2 = 0.0;
                        for (int d = 0; d < DIM; ++d) {
                            rv[d] = min_image(G, T.x[(size_t)d * n + k], T.x[(size_t)d * n + j], d);
                            r2 += rv[d] * rv[d];
                        }
                        const double r = sqrt(r2);
                        const double hij = pair_h(K, T.h[k], T.h[j]);
                        if (!(r < 2.0 * hij) || r == 0.0) continue;
                        f(j, rv, (Real)r, Real(1) / (Real)r);
                    }
                }
            }
        }
    }
}

// Reverse of one pair term of a_i (Eq. 3, 5-7) and R_i (Eq. 14) for the pair
// (i, j), given the cotangents Ai of a_i and Rbi of R_i.  rv = x_i - x_j,
// r = |rv|, inv_r = 1/r, w = W'(r), w2 = W''(r); rho_j, p_j and vj are the
// stand-ins of a wall neighbour when j is a wall; inv_rho_i, inv_rho_j are
// the reciprocals of the densities (each division once per pair or per
// particle, not six times per call).  Outputs: rb (cotangent of rv), dvb
// (of v_i - v_j), rho_ib, rho_jb (of rho_i, rho_j), etab (of eta).
template <typename Real, int DIM>
__device__ __forceinline__ void pair_adjoint(const Consts<Real>& K, const Real* rv, Real r, Real inv_r, Real w,
                                             Real w2, const Real* vi, Real rho_i, Real inv_rho_i, Real p_i,
                                             const Real* vj, Real rho_j, Real inv_rho_j, Real p_j, Real m_j,
                                             const Real* Ai, const Real* Rbi, Real* rb, Real* dvb, Real& rho_ib,
                                             Real& rho_jb, Real& etab)
{
    Real u[3] = {0, 0, 0}, dv[3] = {0, 0, 0};
    Real udv = 0, Au = 0, Adv = 0, Ru = 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        u[d] = rv[d] * inv_r;
        dv[d] = vi[d] - vj[d];
        udv += u[d] * dv[d];
        Au += Ai[d] * u[d];
        Adv += Ai[d] * dv[d];
        Ru += Rbi[d] * u[d];
    }
    const Real dU = -udv;                               // U_l - U_r
    const Real slope = K.beta_slope * K.inv_c;
    const Real braw = slope * dU;
    const Real beta = braw > Real(0) ? (braw < Real(1) ? braw : Real(1)) : Real(0);
    const Real dbeta = (braw > Real(0) && braw < Real(1)) ? slope : Real(0);
    const Real rbar = Real(0.5) * (rho_i + rho_j);
    const Real pstar = Real(0.5) * (p_i + p_j) + Real(0.5) * beta * rbar * K.c * dU;
    const Real Kf = m_j * (inv_rho_i * inv_rho_j);      // m_j / (rho_i rho_j)
    const Real Vj = m_j * inv_rho_j;
    const Real wq = w * inv_r;
    const Real Pb = Real(-2) * Kf * w * Au;
    const Real Kb = Real(-2) * pstar * w * Au + K.two_eta * wq * Adv;
    const Real wb = Real(-2) * Kf * pstar * Au + Vj * Ru;
    const Real wqb = K.two_eta * Kf * Adv;
    etab = Real(2) * Kf * wq * Adv;
    const Real dUb = Pb * Real(0.5) * rbar * K.c * (beta + dU * dbeta);
    const Real rbarb = Pb * Real(0.5) * beta * K.c * dU;
    rho_ib = -Kf * inv_rho_i * Kb + Real(0.5) * rbarb + K.c2 * Real(0.5) * Pb;
    rho_jb = -Kf * inv_rho_j * Kb + Real(0.5) * rbarb + K.c2 * Real(0.5) * Pb - Vj * inv_rho_j * w * Ru;
    Real ub[3] = {0, 0, 0};
    Real uu = 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        ub[d] = Real(-2) * Kf * pstar * w * Ai[d] + Vj * w * Rbi[d] - dUb * dv[d];
        dvb[d] = K.two_eta * Kf * wq * Ai[d] - dUb * u[d];
        uu += ub[d] * u[d];
    }
    const Real radial = w2 * wb + (w2 * inv_r - w * inv_r * inv_r) * wqb;
#pragma unroll
    for (int d = 0; d < DIM; ++d) rb[d] = (ub[d] - uu * u[d]) * inv_r + radial * u[d];
}

// 1/x: rcp.approx in the FP32 form (as its forward pass takes reciprocals),
// the correctly rounded division in the FP64 form.
__device__ __forceinline__ float recip(float x) { return rcp_approx(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

template <typename Real>
__device__ __forceinline__ Real inv_pair_h(const Consts<Real>& K, const Tape<Real>& T, int k, int j)
{
    if constexpr (sizeof(Real) == 4) {
        if (K.uniform_h) return K.inv_h_u;
        return 1.f / pair_h(K, (float)T.h[k], (float)T.h[j]);
    } else {
        return 1.0 / pair_h(K, T.h[k], T.h[j]);
    }
}

// ------------------------------------------------------------------- prep

template <typename Real, int DIM>
__global__ void __launch_bounds__(256) k_adj_prep(int n, Tape<Real> T, Consts<Real> K, int step_mode,
                                                  const double* __restrict__ vc, const double* __restrict__ ac,
                                                  const double* __restrict__ drc, Real* __restrict__ AR)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = T.id[k];
    Real* const ar = AR + (size_t)k * kAbStride<DIM>;
    if (T.kind[k]) {
        for (int q = 0; q < kAbStride<DIM>; ++q) ar[q] = Real(0);
        return;
    }
    const double hdt = step_mode ? 0.5 * *T.dt : 0.0;
    const Real H = K.tv_h_particle ? (Real)T.h[k] : K.h_min;
    const Real H2 = H * H;
    Real R[3] = {0, 0, 0}, D[3] = {0, 0, 0};
    Real s = 0, DR = 0;
    for (int d = 0; d < DIM; ++d) {
        R[d] = T.R[(size_t)d * n + k];
        D[d] = (Real)drc[(size_t)d * n + i];
        s += R[d] * R[d];
        DR += D[d] * R[d];
    }
    s *= H2;
    const Real chi = tv_limiter(K, s);
    const Real dchi = (K.tv_mode == SPH_TV_LIMITED && s > K.tv_thresh && K.tv_C * s < Real(1)) ? K.tv_C : Real(0);
    for (int d = 0; d < DIM; ++d) {
        ar[d] = (Real)(ac[(size_t)d * n + i] + hdt * vc[(size_t)d * n + i]);
        ar[DIM + d] = K.tv_xi * H2 * (chi * D[d] + dchi * DR * Real(2) * H2 * R[d]);
    }
    for (int q = 2 * DIM; q < kAbStride<DIM>; ++q) ar[q] = Real(0);
}

// ------------------------------------------------------------------ pairs

template <typename Real, int DIM>
__global__ void __launch_bounds__(128) k_adj_pairs(int n, Tape<Real> T, Grid G, Consts<Real> K,
                                                   const Real* __restrict__ AR,
                                                   Real* __restrict__ xbp, Real* __restrict__ vbp,
                                                   Real* __restrict__ sigb, double* __restrict__ partials)
{
    using Acc = AccOf<Real>;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double part[kNPart];
#pragma unroll
    for (int q = 0; q < kNPart; ++q) part[q] = 0.0;
    if (k < n && !T.kind[k]) {
        const auto mk = T.vr[k];
        const Real vk[3] = {mk.x, mk.y, mk.z};
        const Real rho_k = K.rho0 + mk.w;
        const Real p_k = K.c2 * mk.w;
        const Real inv_rho_k = Real(1) / rho_k;
        const Real m_k = (Real)T.m[k];
        Real Ak[3] = {0, 0, 0}, Rk[3] = {0, 0, 0};
        load_ab<Real, DIM>(AR, k, Ak, Rk);
        Acc ax[DIM], av[DIM], arho;
        double eta_acc = 0.0;
        auto pair = [&](int j, const Real* rv, Real r, Real inv_r) {
            const Real inv_h = inv_pair_h(K, T, k, j);
            const Real w = wendland_dW<DIM, Real>(r, inv_h);
            const Real w2 = wendland_d2W<DIM, Real>(r, inv_h);
            const auto mj = T.vr[j];
            const Real vj[3] = {mj.x, mj.y, mj.z};
            const bool wall = isinf(mj.w);
            const Real rho_j = wall ? rho_k : K.rho0 + mj.w;
            const Real inv_rho_j = wall ? inv_rho_k : recip(rho_j);
            const Real p_j = wall ? p_k : K.c2 * mj.w;
            Real rb[3], dvb[3], rib, rjb, eb;
            // k's own sums (k as i)
            pair_adjoint<Real, DIM>(K, rv, r, inv_r, w, w2, vk, rho_k, inv_rho_k, p_k, vj, rho_j, inv_rho_j, p_j,
                                    (Real)T.m[j], Ak, Rk, rb, dvb, rib, rjb, eb);
            for (int d = 0; d < DIM; ++d) {
                ax[d].add(rb[d]);
                av[d].add(dvb[d]);
            }
            arho.add(wall ? rib + rjb : rib);
            eta_acc += (double)eb;
            if (wall) return;
            // the fluid neighbour's sums (j as i, k as j): r_jk = -r_kj
            Real Aj[3] = {0, 0, 0}, Rj[3] = {0, 0, 0}, mrv[3] = {0, 0, 0};
            load_ab<Real, DIM>(AR, j, Aj, Rj);
            for (int d = 0; d < DIM; ++d) mrv[d] = -rv[d];
            pair_adjoint<Real, DIM>(K, mrv, r, inv_r, w, w2, vj, rho_j, inv_rho_j, p_j, vk, rho_k, inv_rho_k, p_k,
                                    m_k, Aj, Rj, rb, dvb, rib, rjb, eb);
            for (int d = 0; d < DIM; ++d) {
                ax[d].add(-rb[d]);
                av[d].add(-dvb[d]);
            }
            arho.add(rjb);
        };
        adj_visit<Real, DIM>(n, k, G, K, T, pair);
        for (int d = 0; d < DIM; ++d) {
            xbp[(size_t)d * n + k] = ax[d].value();
            vbp[(size_t)d * n + k] = av[d].value();
        }
        sigb[k] = arho.value() * K.rho0 / (Real)T.s0[k];
        part[0] = eta_acc;
    } else if (k < n) {
        for (int d = 0; d < DIM; ++d) xbp[(size_t)d * n + k] = vbp[(size_t)d * n + k] = Real(0);
        sigb[k] = Real(0);
    }
    block_partials<true>(part, partials + (size_t)blockIdx.x * kNPart);
}

// ------------------------------------------------- density + drift / kick

template <typename Real, int DIM>
__global__ void __launch_bounds__(128) k_adj_density(int n, Tape<Real> T, Grid G, Consts<Real> K,
                                                     const Real* __restrict__ sigb, const Real* __restrict__ xbp,
                                                     const Real* __restrict__ vbp, int step_mode,
                                                     double* __restrict__ xc, double* __restrict__ vc,
                                                     double* __restrict__ ac, double* __restrict__ drc,
                                                     const double* __restrict__ partials, int nblocks,
                                                     double* __restrict__ eta)
{
    using Acc = AccOf<Real>;
    if (blockIdx.x == 0) {
        // block 0 first adds the pair kernel's per-block d/d(eta) partials to
        // eta (a fixed order: strided per thread, then the warps, then the
        // block's warps by thread 0)
        __shared__ double wsum[32];
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[(size_t)b * kNPart];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += wsum[w];
            *eta += t;
        }
    }
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = T.id[k];
    if (T.kind[k]) {
        if (step_mode)
            for (int d = 0; d < 3; ++d) {
                const size_t o = (size_t)d * n + i;
                xc[o] = vc[o] = ac[o] = drc[o] = 0.0;
            }
        return;
    }
    const Real sk = sigb[k];
    Acc acc[DIM];
    auto pair = [&](int j, const Real* rv, Real r, Real inv_r) {
        const Real inv_h = inv_pair_h(K, T, k, j);
        const Real w = wendland_dW<DIM, Real>(r, inv_h);
        const Real sj = T.kind[j] ? Real(0) : sigb[j];
        const Real g = sizeof(Real) == 4 ? (sk + sj) * w * inv_r : (sk + sj) * w / r;
        for (int d = 0; d < DIM; ++d) acc[d].add(g * rv[d]);
    };
    adj_visit<Real, DIM>(n, k, G, K, T, pair);
    const double dt = step_mode ? *T.dt : 0.0;
    const double hdt = 0.5 * dt;
    for (int d = 0; d < DIM; ++d) {
        const size_t o = (size_t)d * n + i, so = (size_t)d * n + k;
        const double xb = xc[o] + (double)xbp[so] + (double)acc[d].value();   // cotangent of x'
        double vh = vc[o] + (double)vbp[so];                                  // of the half-step v
        if (step_mode) {
            drc[o] = xb;              // x' = x + dt v_h + dr
            vh += dt * xb;
            ac[o] = hdt * vh;         // v_h = v + dt/2 a
        }
        xc[o] = xb;
        vc[o] = vh;
    }
}

// ----------------------------------------------------- cotangent layouts

__global__ void k_aos_to_soa(int n, const double* __restrict__ src3, double* __restrict__ dst)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int d = 0; d < 3; ++d) dst[(size_t)d * n + i] = src3[3 * (size_t)i + d];
}

__global__ void k_soa_to_aos(int n, const double* __restrict__ src, double* __restrict__ dst3)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int d = 0; d < 3; ++d) dst3[3 * (size_t)i + d] = src[(size_t)d * n + i];
}

// -------------------------------------------------------------- launchers

cudaError_t launch_aos_to_soa(int n, const double* src3, double* dst, cudaStream_t st)
{
    k_aos_to_soa<<<(n + 255) / 256, 256, 0, st>>>(n, src3, dst);
    return cudaGetLastError();
}

cudaError_t launch_soa_to_aos(int n, const double* src, double* dst3, cudaStream_t st)
{
    k_soa_to_aos<<<(n + 255) / 256, 256, 0, st>>>(n, src, dst3);
    return cudaGetLastError();
}

static inline int nblk(int n, int t) { return (n + t - 1) / t; }

int adj_pair_blocks(int n) { return nblk(n, 128); }

template <typename Real>
static Tape<Real> make_tape(const TapeView& V)
{
    Tape<Real> T;
    T.id = V.id; T.kind = V.kind; T.x = V.x; T.h = V.h; T.m = V.m; T.s0 = V.s0;
    T.vr = (const typename Vec4<Real>::T*)V.vr;
    T.R = (const Real*)V.R;
    T.start = V.start; T.pos4 = V.pos4; T.cell = V.cell; T.dt = V.dt;
    T.nbl = V.nbl; T.nbc = V.nbc;
    return T;
}

template <typename Real, int DIM>
static void adjoint_step_t(int n, const TapeView& V, const Grid& G, const Consts<Real>& K, const AdjView& A,
                           int step_mode, cudaStream_t st)
{
    Tape<Real> T = make_tape<Real>(V);
    k_adj_prep<Real, DIM><<<nblk(n, 256), 256, 0, st>>>(n, T, K, step_mode, A.vc, A.ac, A.drc, (Real*)A.AR);
    k_adj_pairs<Real, DIM><<<nblk(n, 128), 128, 0, st>>>(n, T, G, K, (const Real*)A.AR,
                                                         (Real*)A.xbp, (Real*)A.vbp, (Real*)A.sigb, A.partials);
    k_adj_density<Real, DIM><<<nblk(n, 128), 128, 0, st>>>(n, T, G, K, (const Real*)A.sigb, (const Real*)A.xbp,
                                                           (const Real*)A.vbp, step_mode, A.xc, A.vc, A.ac, A.drc,
                                                           A.partials, nblk(n, 128), A.eta);
}

cudaError_t launch_adjoint_step(int prec, int dim, int n, const TapeView& V, const Grid& G, const void* K,
                                const AdjView& A, int step_mode, cudaStream_t st)
{
    if (prec == 64) {
        const Consts<double>& k = *(const Consts<double>*)K;
        if (dim == 2) adjoint_step_t<double, 2>(n, V, G, k, A, step_mode, st);
        else adjoint_step_t<double, 3>(n, V, G, k, A, step_mode, st);
    } else {
        const Consts<float>& k = *(const Consts<float>*)K;
        if (dim == 2) adjoint_step_t<float, 2>(n, V, G, k, A, step_mode, st);
        else adjoint_step_t<float, 3>(n, V, G, k, A, step_mode, st);
    }
    return cudaGetLastError();
}

}  // namespace sphtv
