// k_pair.cu -- the pair passes of libsphtv, one thread per cell-sorted
// particle, neighbours from the (2R+1)^D block of cells around it.
//
//   k_density : sigma_i = sum_j W(r_ij, h_ij) (self and walls included),
//               rho_i = rho0 sigma_i / sigma0_i (Eq. 8), stored as
//               rho_i - rho0 beside the half-step velocity (p = c^2 (rho -
//               rho0), Eq. 2, is formed where it is used).
//   k_forces  : for every fluid i, over j != i:
//                 Riemann interface pressure P* with the dissipation
//                 limiter (Eq. 5-6), pressure acceleration (Eq. 3),
//                 viscous acceleration (Eq. 7), residual R_i = sum_j V_j
//                 grad_i W_ij (Eq. 14); then the limiter chi_i (Eq. 15), the
//                 displacement dr_i = xi chi_i h^2 R_i (Eq. 16), the closing
//                 half kick, and FP64 block partials of the diagnostics.
//   k_finalize: reduces the partials in a fixed order, computes the next
//               step size min(dt_ad, dt_ac) (Eq. 9-11, h = h_min).
//
// Readings: e_ij points from i to j (Riemann states); grad W_ij is
// grad_i W_ij = W'(r) (x_i - x_j)/r; V_j = m_j / rho_j; rho_bar is the mean
// density, c_bar = c; h_ij = (h_i + h_j)/2 (or max); a wall j stands in with
// rho_j = rho_i, p_j = p_i, V_j = m_j / rho_i and its prescribed velocity.
//
// FP64 form (this file): absolute FP64 positions, the nearest periodic
// image of each pair (fixed by the stencil step of its cell), plain sums;
// 1/rho_i once per particle.  FP32 form: k_pair32.cu.
#include "common.cuh"
#include "launch.h"
#include "pair_physics.cuh"
#include "pair_walk.cuh"

namespace sphtv {

// ============================================================== FP64 form

// Candidates come from the clipped FP32 row walk over the cell-relative
// positions (pos4); a loose FP32 test drops the far ones and the exact FP64
// test (minimum image, sqrt(r2) < 2 h_ij) decides the rest.  The walk visits
// candidates in the order of the cell scan (cells by dz, dy, dx, then index),
// so sigma is summed in the same order as a plain scan would.  With nbl
// non-null it also writes the particle's neighbour list (j != i,
// 0 < r < 2 h_ij), transposed (entry k at nbl[k * n + i] = j << kCodeBits),
// and the count (which may exceed cap); the FP64 force pass walks it.
template <int DIM>
__global__ void __launch_bounds__(256) k_density_f64(int n, StateSet<double> S, const int32_t* __restrict__ start,
                                                     Grid G, Consts<double> K, double4_32a* __restrict__ vr,
                                                     const float4* __restrict__ pos4,
                                                     const int32_t* __restrict__ cell_of, uint32_t* __restrict__ nbl,
                                                     int32_t* __restrict__ nbc, int cap, double* __restrict__ vol)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double xi[3] = {0, 0, 0}, vi[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        xi[d] = S.x[(size_t)d * n + i];
        vi[d] = S.v[(size_t)d * n + i];
    }
    if (S.kind[i]) {
        vr[i] = make_double4_32a(vi[0], vi[1], vi[2], __longlong_as_double(0x7ff0000000000000ll));
        if (nbc) nbc[i] = 0;
        return;
    }
    const double hi = S.h[i];
    const float4 pi = pos4[i];
    const float oi[3] = {pi.x, pi.y, pi.z};
    const int cell_i = cell_of[i];
    int ci[3];
    cell_decode(G, cell_i, ci);
    // reach of the walk: the largest support radius 2 h_ij of i (h_j <= h_max)
    const float reach = (float)(2.0 * pair_h(K, hi, K.h_u));
    // uniform resolution: h_ij = h for every pair, so the support, the
    // prefilter bound and a_D h^-D are constants (the same values, computed
    // once instead of per candidate on the FP64 pipe)
    const bool uni = K.uniform_h != 0;
    const double two_hu = 2.0 * K.h_u;
    const float lim_u = (float)two_hu;
    const float lim2_u = lim_u * lim_u * 1.0001f;
    const double wnorm_u = kernel_norm<DIM, double>() * pow_dim<DIM, double>(K.inv_h_u);
    const double half_inv_hu = 0.5 * K.inv_h_u, two_inv_hu = 2.0 * K.inv_h_u;
    // sigma; at uniform resolution the sum of W / (a_D h^-D), the constant
    // applied once at the end
    double sigma = 0.0;
    // the exact FP64 test of a candidate that passed the FP32 prefilter: adds
    // W to sigma; true for a force neighbour (j != i, 0 < r < 2 h_ij).  The
    // comparisons of non-negative doubles are made on their bit patterns
    // (same order) by the integer ALU, off the FP64 pipe.
    auto exact = [&](int j, uint32_t code, double hij) {
        // x_i - x_j with the periodic image of the stencil step (the nearest
        // image of every neighbour: the same operations as min_image)
        const int step[3] = {(int)(code % kSide) - kStencilR, (int)((code / kSide) % kSide) - kStencilR,
                             (int)(code / (kSide * kSide)) - kStencilR};
        double r2 = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            double t = __dsub_rn(xi[d], S.x[(size_t)d * n + j]);
            if (G.periodic[d]) {
                const int sc = ci[d] + step[d];
                if (sc >= G.nc[d]) t = __dsub_rn(t, G.L[d]);
                else if (sc < 0) t = __dadd_rn(t, G.L[d]);
            }
            r2 += t * t;
        }
        const double r = sqrt(r2);
        // r < 2 h_ij (a NaN has a pattern above every finite value's)
        if (!((unsigned long long)__double_as_longlong(r) <
              (unsigned long long)__double_as_longlong(uni ? two_hu : 2.0 * hij)))
            return false;
        if (uni) {
            // t = 1 - q/2 and 2q + 1 with q = r/h, each one fused operation
            const double t = fma(-half_inv_hu, r, 1.0);
            const double t2 = t * t;
            sigma = fma(t2 * t2, fma(two_inv_hu, r, 1.0), sigma);
        } else {
            sigma += wendland_W<DIM, double>(r, 1.0 / hij);
        }
        return j != i && __double_as_longlong(r2) != 0;               // r2 >= +0
    };
    // FP32 prefilter bound (1e-4 margin) of the pair (i, j); pj_w = (float)h_j
    // when h varies
    const float hi_f = (float)hi;
    auto prefilter2 = [&](float pj_w) {
        if (uni) return lim2_u;
        const float lim = 2.f * (K.h_pair_max ? fmaxf(hi_f, pj_w) : 0.5f * (hi_f + pj_w));
        return lim * lim * 1.0001f;
    };
    int cnt = 0;
    // one pass: the exact test inside the walk (the lanes whose candidate
    // passed the prefilter run it while the others wait)
    auto visit = [&](int j, uint32_t code, const float4&, float r2f, float, float, float) {
        double hij = K.h_u;
        float lim2 = lim2_u;
        if (!uni) {
            hij = pair_h(K, hi, S.h[j]);
            const float lim = (float)(2.0 * hij);
            lim2 = lim * lim * 1.0001f;
        }
        if (!(r2f <= lim2)) return;                      // FP32 prefilter, 1e-4 margin
        if (exact(j, code, hij) && nbl) {
            if (cnt < cap) nbl[(size_t)cnt * n + i] = ((uint32_t)j << kCodeBits) | code;
            ++cnt;
        }
    };
    bool staged = false;
    if (nbl) {
        // two passes: the walk stages the candidates that pass the prefilter
        // in the particle's list, then the exact FP64 test runs over them
        // with every lane busy (the FP64 pipe serves a warp instruction
        // whole, however few of its lanes are active), and the list is
        // compacted in place to the force neighbours.  Same tests, in the
        // same order, as the one pass.
        int nf = 0;
        uint32_t* lp = nbl + i;
        auto stage = [&](int j, uint32_t code, const float4& pj, float r2f, float, float, float) {
            if (!(r2f <= prefilter2(pj.w))) return;
            if (nf < cap) {
                *lp = ((uint32_t)j << kCodeBits) | code;
                lp += n;
            }
            ++nf;
        };
        for_candidates_rows<DIM, false>(oi, reach, cell_i, G, start, cell_of, pos4, stage);
        if (nf <= cap) {
            staged = true;
            for (int k = 0; k < nf; ++k) {
                const uint32_t e = nbl[(size_t)k * n + i];
                const int j = (int)(e >> kCodeBits);
                const double hij = uni ? K.h_u : pair_h(K, hi, S.h[j]);
                if (exact(j, e & ((1u << kCodeBits) - 1u), hij)) {
                    if (cnt != k) nbl[(size_t)cnt * n + i] = e;     // entries before a rejected one stay in place
                    ++cnt;
                }
            }
        }
    }
    if (!staged) for_candidates_rows<DIM, false>(oi, reach, cell_i, G, start, cell_of, pos4, visit);
    if (nbc) nbc[i] = cnt;
    if (uni) sigma *= wnorm_u;
    double rho = __ddiv_rn(__dmul_rn(K.rho0, sigma), S.s0[i]);
    const double w = __dsub_rn(rho, K.rho0);
    vr[i] = make_double4_32a(vi[0], vi[1], vi[2], w);
    // V_i = m_i / rho_i for the force pass, once per particle instead of once
    // per pair
    if (vol) vol[i] = S.m[i] / (K.rho0 + w);
}

template <int DIM>
__global__ void __launch_bounds__(256, 2) k_forces_f64(int n, StateSet<double> S, const int32_t* __restrict__ start,
                                                    Grid G, Consts<double> K, const double4_32a* __restrict__ vr,
                                                    const uint32_t* __restrict__ nbl, const int32_t* __restrict__ nbc,
                                                    int cap, const double* __restrict__ dt_ptr, int kick_on,
                                                    int write_ad, double* __restrict__ Rout,
                                                    double* __restrict__ chi_out, double* __restrict__ partials,
                                                    const double* __restrict__ vol)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double part[kNPart];
#pragma unroll
    for (int k = 0; k < kNPart; ++k) part[k] = 0.0;
    const double dt = *dt_ptr;
    const double hdt = kick_on ? 0.5 * dt : 0.0;
    if (i < n && S.kind[i] == 0) {
        double xi[3] = {0, 0, 0}, vi[3] = {0, 0, 0};
        double4_32a me = vr[i];
        vi[0] = me.x; vi[1] = me.y; vi[2] = me.z;
#pragma unroll
        for (int d = 0; d < DIM; ++d) xi[d] = S.x[(size_t)d * n + i];
        const double hi = S.h[i];
        const double rho_i = K.rho0 + me.w;
        const double inv_rho_i = 1.0 / rho_i;
        PlainD acc_a[DIM], acc_R[DIM];
        // uniform resolution: h_ij = h for every pair, so the support bounds
        // and -5 a_D h^-(D+2) are constants
        const bool uni = K.uniform_h != 0;
        const double far_u = 4.0 * K.h_u * K.h_u * (1.0 + 1e-12), two_hu = 2.0 * K.h_u;
        const double dwrnorm_u = -5.0 * kernel_norm<DIM, double>() * pow_dim<DIM, double>(K.inv_h_u) * K.inv_h_u *
                                 K.inv_h_u;
        // the cell of i (as the sort computed it from these positions)
        const int ci[3] = {cell_coord(G, xi[0], 0), cell_coord(G, xi[1], 1), DIM == 3 ? cell_coord(G, xi[2], 2) : 0};
        // W'/r = C t^3 at uniform resolution (t = 1 - r / 2h): C leaves the sums
        const double C = uni ? dwrnorm_u : 1.0;
        const double half_inv_h = 0.5 * K.inv_h_u;
        const PairI64 I = pair_i64(K, me.w, inv_rho_i, C);
        // a neighbour j (0 < r < 2 h_ij) at rv = x_i - x_j, r2 = |rv|^2
        auto body = [&](int j, const double* rv, double r2) {
            const double inv_r = rsqrt(r2);
            const double r = r2 * inv_r;
            double g;
            if (uni) {
                const double t = fma(-half_inv_h, r, 1.0);
                g = t * t * t;
            } else {
                g = wendland_dW<DIM, double>(r, 1.0 / pair_h(K, hi, S.h[j])) * inv_r;
            }
            const double4_32a oj = vr[j];
            const double vj[3] = {oj.x, oj.y, oj.z};
            double w_j = oj.w, V_j = vol[j];
            const bool wall = is_wall(w_j);
            if (__any_sync(__activemask(), wall)) {
                // a wall stands in with rho_j = rho_i: w_j = w_i, V_j = m_j / rho_i
                if (wall) {
                    w_j = me.w;
                    V_j = S.m[j] * inv_rho_i;
                }
            }
            pair_force64<DIM>(K, I, rv, inv_r, g, vi, vj, w_j, V_j, acc_a, acc_R);
        };
        const int cnt = nbl ? nbc[i] : cap + 1;
        if (cnt <= cap) {
            // the density pass's list: exactly the pairs with 0 < r < 2 h_ij
            // (its exact FP64 test), in the order of the cell scan below, so
            // no test is repeated here.  The stencil step of j's cell fixes
            // the periodic image (the nearest one for every neighbour: the
            // same operations as min_image).
            for (int k = 0; k < cnt; ++k) {
                const uint32_t e = nbl[(size_t)k * n + i];
                const int j = (int)(e >> kCodeBits);
                const int code = (int)(e & ((1u << kCodeBits) - 1u));
                const int step[3] = {code % kSide - kStencilR, (code / kSide) % kSide - kStencilR,
                                     code / (kSide * kSide) - kStencilR};
                double rv[3] = {0, 0, 0};
                double r2 = 0.0;
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    double t = __dsub_rn(xi[d], S.x[(size_t)d * n + j]);
                    if (G.periodic[d]) {
                        const int sc = ci[d] + step[d];
                        if (sc >= G.nc[d]) t = __dsub_rn(t, G.L[d]);
                        else if (sc < 0) t = __dadd_rn(t, G.L[d]);
                    }
                    rv[d] = t;
                    r2 += t * t;
                }
                body(j, rv, r2);
            }
        } else {
            // no list (or more neighbours than it holds): scan the cells with
            // the minimum image and the support test
            const int SR = G.R, zr = DIM == 3 ? SR : 0;
            for (int dz = -zr; dz <= zr; ++dz) {
                int cz = DIM == 3 ? cell_step(G, ci[2], dz, 2) : 0;
                if (cz < 0) continue;
                for (int dy = -SR; dy <= SR; ++dy) {
                    int cy = cell_step(G, ci[1], dy, 1);
                    if (cy < 0) continue;
                    for (int dx = -SR; dx <= SR; ++dx) {
                        int cx = cell_step(G, ci[0], dx, 0);
                        if (cx < 0) continue;
                        int cell = cx + G.nc[0] * (cy + G.nc[1] * cz);
                        for (int j = start[cell]; j < start[cell + 1]; ++j) {
                            if (j == i) continue;
                            double rv[3] = {0, 0, 0};
                            double r2 = 0.0;
#pragma unroll
                            for (int d = 0; d < DIM; ++d) {
                                rv[d] = min_image(G, xi[d], S.x[(size_t)d * n + j], d);
                                r2 += rv[d] * rv[d];
                            }
                            const double hij = uni ? K.h_u : pair_h(K, hi, S.h[j]);
                            if (r2 > (uni ? far_u : 4.0 * hij * hij * (1.0 + 1e-12))) continue;
                            if (!(r2 > 0.0)) continue;
                            if (!(sqrt(r2) < (uni ? two_hu : 2.0 * hij))) continue;
                            body(j, rv, r2);
                        }
                    }
                }
            }
        }
        double a[3] = {0, 0, 0}, R[3] = {0, 0, 0};
        double R2 = 0.0;
        const double m_i = S.m[i];
        // free-stream forcing lambda(x) (U_inf - v) of the fringe region
        const double lam = K.fr_on ? fringe_rate<double>(K, xi[0]) : 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const double pair_a = acc_a[d].value();
            // the fluid's momentum rate from its pair terms: minus the force on the walls
            if (K.body_force) part[9 + d] = m_i * pair_a;
            a[d] = K.g[d] + pair_a;
            if (K.fr_on) a[d] += lam * (K.fr_u[d] - vi[d]);
            R[d] = C * acc_R[d].value();
            R2 += R[d] * R[d];
        }
        const double htv = K.tv_h_particle ? hi : K.h_min;
        const double htv2 = htv * htv;
        const double chi = tv_limiter(K, htv2 * R2);
        // Eq. 12 (background pressure p0 = rho0 c^2): dr = dt^2/2 a_bg = -(dt^2 p0 / rho_i) R_i
        const bool bgmode = K.tv_mode == SPH_TV_BACKGROUND;
        const double bg = bgmode ? -(dt * dt * (K.rho0 * K.c2) / rho_i) : 0.0;
        double v2 = 0.0, vt2 = 0.0, dr2 = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            size_t o = (size_t)d * n + i;
            double dr = bgmode ? bg * R[d] : K.tv_xi * chi * htv2 * R[d];
            double vn = __dadd_rn(vi[d], __dmul_rn(hdt, a[d]));
            if (write_ad) {
                S.a[o] = a[d];
                S.dr[o] = dr;
            }
            S.v[o] = vn;
            Rout[o] = R[d];
            part[1 + d] = m_i * vn;
            v2 += vn * vn;
            dr2 += dr * dr;
            double vt = dt > 0.0 ? vn + dr / dt : vn;
            vt2 += vt * vt;
        }
        chi_out[i] = chi;
        part[0] = m_i;
        part[4] = 0.5 * m_i * v2;
        part[5] = chi > 0.0 ? 1.0 : 0.0;
        part[6] = v2;                 // squares: block_partials takes the roots
        part[7] = vt2;
        part[8] = dr2;
    } else if (i < n) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            if (write_ad) {
                S.a[(size_t)d * n + i] = 0.0;
                S.dr[(size_t)d * n + i] = 0.0;
            }
            Rout[(size_t)d * n + i] = 0.0;
        }
        chi_out[i] = 0.0;
    }
    block_partials<true>(part, partials + (size_t)blockIdx.x * kNPart, true, K.body_force != 0);
}

// ================================================ diagnostics only

// FP64 partials of the diagnostics from the stored v and dr (no pair work):
// used when the caller supplied a and dr, so no force pass is needed.
template <typename Real, int DIM>
__global__ void __launch_bounds__(256) k_diag_only(int n, StateSet<Real> S, double* __restrict__ partials)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double part[kNPart];
#pragma unroll
    for (int k = 0; k < kNPart; ++k) part[k] = 0.0;
    if (i < n && S.kind[i] == 0) {
        const double m_i = S.m[i];
        double v2 = 0.0, dr2 = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            double v = (double)S.v[(size_t)d * n + i];
            double dr = (double)S.dr[(size_t)d * n + i];
            part[1 + d] = m_i * v;
            v2 += v * v;
            dr2 += dr * dr;
        }
        part[0] = m_i;
        part[4] = 0.5 * m_i * v2;
        part[6] = v2;                 // squares: block_partials takes the roots
        part[7] = v2;
        part[8] = dr2;
    }
    block_partials<true>(part, partials + (size_t)blockIdx.x * kNPart);
}

// =========================================================== finalize

// First level of the diagnostics reduction: block b folds rows
// [b * chunk, (b + 1) * chunk) of the per-block partials into row b of out,
// in a fixed order (the result does not depend on timing).
__global__ void __launch_bounds__(256) k_reduce_rows(int nrows, int chunk, const double* __restrict__ in,
                                                     double* __restrict__ out)
{
    double acc[kNPart];
#pragma unroll
    for (int k = 0; k < kNPart; ++k) acc[k] = 0.0;
    const int r0 = blockIdx.x * chunk, r1 = min(nrows, r0 + chunk);
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const double* p = in + (size_t)r * kNPart;
#pragma unroll
        for (int k = 0; k < kNPart; ++k) acc[k] = (k >= 6 && k <= 8) ? fmax(acc[k], p[k]) : acc[k] + p[k];
    }
    block_partials<false>(acc, out + (size_t)blockIdx.x * kNPart);
}

struct DtConsts {
    double eta, rho0, h_min, u_ref, cfl_ad, cfl_ac, c, fixed_dt;
};

__global__ void __launch_bounds__(256) k_finalize(int nblocks, const double* __restrict__ partials, DtConsts D,
                                                  double* __restrict__ diag, double* __restrict__ dt_ptr,
                                                  int count_step)
{
    double acc[kNPart];
#pragma unroll
    for (int k = 0; k < kNPart; ++k) acc[k] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const double* p = partials + (size_t)b * kNPart;
#pragma unroll
        for (int k = 0; k < kNPart; ++k) acc[k] = (k >= 6 && k <= 8) ? fmax(acc[k], p[k]) : acc[k] + p[k];
    }
    __shared__ double out[kNPart];
    block_partials<false>(acc, out);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double vmax = out[6];
        const double dt_used = *dt_ptr;
        // Eq. 9-11 with h = h_min
        const double nu = D.eta / D.rho0;
        const double vad = fmax(vmax, fmax(nu / D.h_min, D.u_ref));
        const double dt_ad = D.cfl_ad * D.h_min / vad;
        const double dt_ac = D.cfl_ac * D.h_min / (vmax + D.c);
        const double dt_next = D.fixed_dt > 0.0 ? D.fixed_dt : fmin(dt_ad, dt_ac);
        diag[DG_MASS] = out[0];
        diag[DG_MOM + 0] = out[1];
        diag[DG_MOM + 1] = out[2];
        diag[DG_MOM + 2] = out[3];
        diag[DG_KE] = out[4];
        diag[DG_NCHI] = out[5];
        diag[DG_VMAX] = vmax;
        diag[DG_VTMAX] = out[7];
        diag[DG_DRMAX] = out[8];
        diag[DG_DT] = count_step ? dt_used : 0.0;
        diag[DG_DTNEXT] = dt_next;
        diag[DG_STEPS] = count_step ? diag[DG_STEPS] + 1.0 : 0.0;
        for (int d = 0; d < 3; ++d) diag[DG_FBODY + d] = -out[9 + d];    // force on the walls
        // simulated time and the body's impulse since sph_build_cells (the time
        // integral of the force over the steps, each step's force times its dt)
        for (int d = 0; d < 3; ++d) diag[DG_IMPULSE + d] = count_step ? diag[DG_IMPULSE + d] - out[9 + d] * dt_used : 0.0;
        diag[DG_TIME] = count_step ? diag[DG_TIME] + dt_used : 0.0;
        *dt_ptr = dt_next;
    }
}

// ============================================================ launchers

static inline int nblk(int n, int t) { return (n + t - 1) / t; }

// Threads per block of the pair passes: 256 (FP64) or 128 (FP32) when the
// particles fill every SM at that size; smaller blocks (down to one warp)
// when they do not, so that a small problem still spreads over all SMs
// instead of queueing its FP64 work on a few.
int pair_threads(int prec, int n, int sms)
{
    const int full = prec == 64 ? 256 : 128;
    if (sms <= 0) sms = 152;
    if ((int64_t)n >= (int64_t)sms * full) return full;
    int t = ((n + sms - 1) / sms + 31) / 32 * 32;
    return t < 32 ? 32 : (t > full ? full : t);
}

int pair_blocks(int prec, int n, int sms) { return nblk(n, pair_threads(prec, n, sms)); }

cudaError_t launch_density(int prec, int dim, int n, void* S, const int32_t* start, const Grid& G, const void* K,
                           void* vr, const float4* pos4, const int32_t* cell_of, uint32_t* nbl, int32_t* nbc,
                           cudaStream_t st, double* vol, const float4* pos4c, int tiles)
{
    const int T = pair_threads(prec, n, G.sms);
    if (prec == 32) return launch_density32(dim, n, S, start, G, K, vr, pos4, cell_of, nbl, nbc, st, pos4c, tiles);
    auto s = *(StateSet<double>*)S;
    auto k = *(const Consts<double>*)K;
    const int cap = nbl_capacity(dim);
    if (dim == 2)
        k_density_f64<2><<<nblk(n, T), T, 0, st>>>(n, s, start, G, k, (double4_32a*)vr, pos4, cell_of, nbl, nbc, cap,
                                                   vol);
    else
        k_density_f64<3><<<nblk(n, T), T, 0, st>>>(n, s, start, G, k, (double4_32a*)vr, pos4, cell_of, nbl, nbc, cap,
                                                   vol);
    return cudaGetLastError();
}

cudaError_t launch_forces(int prec, int dim, int n, void* S, const int32_t* start, const Grid& G, const void* K,
                          const float* mf, const void* vr, const float4* pos4, const int32_t* cell_of,
                          const uint32_t* nbl, const int32_t* nbc, const double* dt, int kick_on, int write_ad,
                          void* Rout, void* chi, double* partials, cudaStream_t st, const double* vol)
{
    const int T = pair_threads(prec, n, G.sms);
    if (prec == 32)
        return launch_forces32(dim, n, S, start, G, K, mf, vr, pos4, cell_of, nbl, nbc, dt, kick_on, write_ad, Rout,
                               chi, partials, st);
    auto s = *(StateSet<double>*)S;
    auto k = *(const Consts<double>*)K;
    const int cap = nbl_capacity(dim);
    if (dim == 2)
        k_forces_f64<2><<<nblk(n, T), T, 0, st>>>(n, s, start, G, k, (const double4_32a*)vr, nbl, nbc, cap, dt,
                                                  kick_on, write_ad, (double*)Rout, (double*)chi, partials, vol);
    else
        k_forces_f64<3><<<nblk(n, T), T, 0, st>>>(n, s, start, G, k, (const double4_32a*)vr, nbl, nbc, cap, dt,
                                                  kick_on, write_ad, (double*)Rout, (double*)chi, partials, vol);
    return cudaGetLastError();
}

cudaError_t launch_diag_only(int prec, int dim, int n, void* S, double* partials, int sms, cudaStream_t st)
{
    const int T = pair_threads(prec, n, sms);   // one partials row per block of the force pass
    if (prec == 64) {
        auto s = *(StateSet<double>*)S;
        if (dim == 2) k_diag_only<double, 2><<<nblk(n, T), T, 0, st>>>(n, s, partials);
        else k_diag_only<double, 3><<<nblk(n, T), T, 0, st>>>(n, s, partials);
    } else {
        auto s = *(StateSet<float>*)S;
        if (dim == 2) k_diag_only<float, 2><<<nblk(n, T), T, 0, st>>>(n, s, partials);
        else k_diag_only<float, 3><<<nblk(n, T), T, 0, st>>>(n, s, partials);
    }
    return cudaGetLastError();
}

int reduce_rows_blocks() { return 256; }

int launch_reduce_rows(int nblocks, const double* partials, double* rows, cudaStream_t st)
{
    const int G = reduce_rows_blocks();
    if (nblocks <= 4 * G) return 0;
    const int chunk = (nblocks + G - 1) / G;
    k_reduce_rows<<<G, 256, 0, st>>>(nblocks, chunk, partials, rows);
    return G;
}

cudaError_t launch_finalize(int nblocks, const double* partials, double* rows, const sph_params& P, double* diag,
                            double* dt, int count_step, cudaStream_t st)
{
    DtConsts D{P.eta, P.rho0, P.h_min, P.u_ref, P.cfl_ad, P.cfl_ac, P.c0, P.fixed_dt};
    const int G = reduce_rows_blocks();
    if (nblocks > 4 * G) {
        const int chunk = (nblocks + G - 1) / G;
        k_reduce_rows<<<G, 256, 0, st>>>(nblocks, chunk, partials, rows);
        k_finalize<<<1, 256, 0, st>>>(G, rows, D, diag, dt, count_step);
    } else {
        k_finalize<<<1, 256, 0, st>>>(nblocks, partials, D, diag, dt, count_step);
    }
    return cudaGetLastError();
}

}  // namespace sphtv
