// k_pair.cu -- the pair passes of libsphtv, one thread per cell-sorted
// particle, neighbours from the 3^D block of cells around it.
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
// FP64 form: absolute FP64 positions, minimum image per pair, plain sums.
// FP32 form: FP32 positions relative to the cell origin plus a per
// neighbour-cell shift, Kahan-compensated FP32 pair sums, FP64 partials.
#include "common.cuh"
#include "launch.h"

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
    if (K.tv_mode == SPH_TV_UNLIMITED) return Real(1);
    if (s > K.tv_thresh) {
        Real t = K.tv_C * s;
        return t < Real(1) ? t : Real(1);
    }
    return Real(0);
}

// Contribution of neighbour j to a_i and R_i (rv = x_i - x_j, r = |rv|,
// dw = W'(r, h_ij)).  Adds into the caller's accumulators.
template <typename Real, int DIM, typename Acc>
__device__ __forceinline__ void pair_force(const Consts<Real>& K, const Real* rv, Real r, Real dw, const Real* vi,
                                           Real rho_i, Real p_i, const Real* vj, Real w_j, Real m_j, Acc* acc_a,
                                           Acc* acc_R)
{
    const bool wall = isinf(w_j);
    const Real rho_j = wall ? rho_i : K.rho0 + w_j;
    const Real p_j = wall ? p_i : K.c2 * w_j;
    const Real inv_r = Real(1) / r;
    Real ul = Real(0), ur = Real(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        Real e = -rv[d] * inv_r;
        ul += vi[d] * e;
        ur += vj[d] * e;
    }
    Real du = ul - ur;
    Real beta = K.beta_slope * (du * K.inv_c);
    beta = beta > Real(0) ? beta : Real(0);
    beta = beta < Real(1) ? beta : Real(1);
    const Real rhobar = Real(0.5) * (rho_i + rho_j);
    const Real pstar = Real(0.5) * (p_i + p_j) + Real(0.5) * beta * rhobar * K.c * du;
    const Real inv_rr = Real(1) / (rho_i * rho_j);
    const Real cp = Real(-2) * m_j * pstar * inv_rr;
    const Real cv = K.two_eta * m_j * inv_rr * dw * inv_r;
    const Real V_j = m_j / rho_j;
    const Real dwr = dw * inv_r;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        Real gw = dwr * rv[d];
        acc_a[d].add(cp * gw + cv * (vi[d] - vj[d]));
        acc_R[d].add(V_j * gw);
    }
}

// Block reduction of the FP64 partials: 6 sums then 3 maxima.
__device__ __forceinline__ void block_partials(double* vals, double* out_block)
{
    __shared__ double sh[32][kNPart];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < kNPart; ++k) {
        double x = vals[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            double y = __shfl_down_sync(0xffffffffu, x, off);
            x = (k >= 6 && k <= 8) ? fmax(x, y) : x + y;
        }
        if (lane == 0) sh[w][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < kNPart) {
        int k = threadIdx.x;
        double x = sh[0][k];
        for (int t = 1; t < nw; ++t) x = (k >= 6 && k <= 8) ? fmax(x, sh[t][k]) : x + sh[t][k];
        out_block[k] = x;
    }
}
// partial layout: 0 mass, 1-3 momentum, 4 KE, 5 n_chi, 6 vmax, 7 vt_max, 8 dr_max, 9 unused

// ============================================================== FP64 form

template <int DIM>
__global__ void __launch_bounds__(256) k_density_f64(int n, StateSet<double> S, const int32_t* __restrict__ start,
                                                     Grid G, Consts<double> K, double4_32a* __restrict__ vr)
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
        return;
    }
    const double hi = S.h[i];
    int c[3] = {cell_coord(G, xi[0], 0), cell_coord(G, xi[1], 1), DIM == 3 ? cell_coord(G, xi[2], 2) : 0};
    double sigma = 0.0;
    const int zr = DIM == 3 ? 1 : 0;
    for (int dz = -zr; dz <= zr; ++dz) {
        int cz = DIM == 3 ? cell_step(G, c[2], dz, 2) : 0;
        if (cz < 0) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            int cy = cell_step(G, c[1], dy, 1);
            if (cy < 0) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                int cx = cell_step(G, c[0], dx, 0);
                if (cx < 0) continue;
                int cell = cx + G.nc[0] * (cy + G.nc[1] * cz);
                for (int j = start[cell]; j < start[cell + 1]; ++j) {
                    double r2 = 0.0;
#pragma unroll
                    for (int d = 0; d < DIM; ++d) {
                        double t = min_image(G, xi[d], S.x[(size_t)d * n + j], d);
                        r2 += t * t;
                    }
                    double r = sqrt(r2);
                    double hij = pair_h(K, hi, S.h[j]);
                    if (r < 2.0 * hij) sigma += wendland_W<DIM, double>(r, 1.0 / hij);
                }
            }
        }
    }
    double rho = __ddiv_rn(__dmul_rn(K.rho0, sigma), S.s0[i]);
    vr[i] = make_double4_32a(vi[0], vi[1], vi[2], __dsub_rn(rho, K.rho0));
}

template <int DIM>
__global__ void __launch_bounds__(256) k_forces_f64(int n, StateSet<double> S, const int32_t* __restrict__ start,
                                                    Grid G, Consts<double> K, const double4_32a* __restrict__ vr,
                                                    const double* __restrict__ dt_ptr, int kick_on, int write_ad,
                                                    double* __restrict__ Rout, double* __restrict__ chi_out,
                                                    double* __restrict__ partials)
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
        const double p_i = K.c2 * me.w;
        PlainD acc_a[DIM], acc_R[DIM];
        int c[3] = {cell_coord(G, xi[0], 0), cell_coord(G, xi[1], 1), DIM == 3 ? cell_coord(G, xi[2], 2) : 0};
        const int zr = DIM == 3 ? 1 : 0;
        for (int dz = -zr; dz <= zr; ++dz) {
            int cz = DIM == 3 ? cell_step(G, c[2], dz, 2) : 0;
            if (cz < 0) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                int cy = cell_step(G, c[1], dy, 1);
                if (cy < 0) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    int cx = cell_step(G, c[0], dx, 0);
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
                        double r = sqrt(r2);
                        double hij = pair_h(K, hi, S.h[j]);
                        if (!(r < 2.0 * hij) || r == 0.0) continue;
                        double dw = wendland_dW<DIM, double>(r, 1.0 / hij);
                        double4_32a oj = vr[j];
                        double vj[3] = {oj.x, oj.y, oj.z};
                        pair_force<double, DIM, PlainD>(K, rv, r, dw, vi, rho_i, p_i, vj, oj.w, S.m[j], acc_a, acc_R);
                    }
                }
            }
        }
        double a[3] = {0, 0, 0}, R[3] = {0, 0, 0};
        double R2 = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            a[d] = K.g[d] + acc_a[d].value();
            R[d] = acc_R[d].value();
            R2 += R[d] * R[d];
        }
        const double htv = K.tv_h_particle ? hi : K.h_min;
        const double htv2 = htv * htv;
        const double chi = tv_limiter(K, htv2 * R2);
        const double m_i = S.m[i];
        double v2 = 0.0, vt2 = 0.0, dr2 = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            size_t o = (size_t)d * n + i;
            double dr = K.tv_xi * chi * htv2 * R[d];
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
        part[6] = sqrt(v2);
        part[7] = sqrt(vt2);
        part[8] = sqrt(dr2);
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
    block_partials(part, partials + (size_t)blockIdx.x * kNPart);
}

// ============================================================== FP32 form

template <int DIM, typename Acc>
__global__ void __launch_bounds__(256) k_density_f32(int n, const float4* __restrict__ pos4,
                                                     const int32_t* __restrict__ cell_of,
                                                     const int32_t* __restrict__ start, Grid G, Consts<float> K,
                                                     StateSet<float> S, float4* __restrict__ vr)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float vi[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int d = 0; d < DIM; ++d) vi[d] = S.v[(size_t)d * n + i];
    if (S.kind[i]) {
        vr[i] = make_float4(vi[0], vi[1], vi[2], __int_as_float(0x7f800000));
        return;
    }
    const float4 pi = pos4[i];
    const float oi[3] = {pi.x, pi.y, pi.z};
    const float hi = pi.w;
    int c[3];
    cell_decode(G, cell_of[i], c);
    Acc sigma;
    const int zr = DIM == 3 ? 1 : 0;
    for (int dz = -zr; dz <= zr; ++dz) {
        int cz = DIM == 3 ? cell_step(G, c[2], dz, 2) : 0;
        if (cz < 0) continue;
        float shz = -(float)dz * G.edgef[2];
        for (int dy = -1; dy <= 1; ++dy) {
            int cy = cell_step(G, c[1], dy, 1);
            if (cy < 0) continue;
            float shy = -(float)dy * G.edgef[1];
            for (int dx = -1; dx <= 1; ++dx) {
                int cx = cell_step(G, c[0], dx, 0);
                if (cx < 0) continue;
                float shx = -(float)dx * G.edgef[0];
                int cell = cx + G.nc[0] * (cy + G.nc[1] * cz);
                for (int j = start[cell]; j < start[cell + 1]; ++j) {
                    float4 pj = pos4[j];
                    float rx = (oi[0] - pj.x) + shx;
                    float ry = (oi[1] - pj.y) + shy;
                    float r2 = rx * rx + ry * ry;
                    if (DIM == 3) {
                        float rz = (oi[2] - pj.z) + shz;
                        r2 += rz * rz;
                    }
                    float hij = pair_h(K, hi, pj.w);
                    if (r2 < 4.f * hij * hij) sigma.add(wendland_W<DIM, float>(sqrtf(r2), 1.f / hij));
                }
            }
        }
    }
    // rho - rho0 = rho0 (sigma - sigma0) / sigma0; sigma - sigma0 is exact in FP32
    const float s0 = (float)S.s0[i];
    const float w = K.rho0 * (sigma.value() - s0) / s0;
    vr[i] = make_float4(vi[0], vi[1], vi[2], w);
}

template <int DIM, typename Acc>
__global__ void __launch_bounds__(256) k_forces_f32(int n, const float4* __restrict__ pos4,
                                                    const int32_t* __restrict__ cell_of,
                                                    const int32_t* __restrict__ start, Grid G, Consts<float> K,
                                                    StateSet<float> S, const float4* __restrict__ vr,
                                                    const double* __restrict__ dt_ptr, int kick_on, int write_ad,
                                                    float* __restrict__ Rout, float* __restrict__ chi_out,
                                                    double* __restrict__ partials)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double part[kNPart];
#pragma unroll
    for (int k = 0; k < kNPart; ++k) part[k] = 0.0;
    const double dt = *dt_ptr;
    const double hdt = kick_on ? 0.5 * dt : 0.0;
    if (i < n && S.kind[i] == 0) {
        const float4 pi = pos4[i];
        const float oi[3] = {pi.x, pi.y, pi.z};
        const float hi = pi.w;
        const float4 me = vr[i];
        const float vi[3] = {me.x, me.y, me.z};
        const float rho_i = K.rho0 + me.w;
        const float p_i = K.c2 * me.w;
        Acc acc_a[DIM], acc_R[DIM];
        int c[3];
        cell_decode(G, cell_of[i], c);
        const int zr = DIM == 3 ? 1 : 0;
        for (int dz = -zr; dz <= zr; ++dz) {
            int cz = DIM == 3 ? cell_step(G, c[2], dz, 2) : 0;
            if (cz < 0) continue;
            float shz = -(float)dz * G.edgef[2];
            for (int dy = -1; dy <= 1; ++dy) {
                int cy = cell_step(G, c[1], dy, 1);
                if (cy < 0) continue;
                float shy = -(float)dy * G.edgef[1];
                for (int dx = -1; dx <= 1; ++dx) {
                    int cx = cell_step(G, c[0], dx, 0);
                    if (cx < 0) continue;
                    float shx = -(float)dx * G.edgef[0];
                    int cell = cx + G.nc[0] * (cy + G.nc[1] * cz);
                    for (int j = start[cell]; j < start[cell + 1]; ++j) {
                        if (j == i) continue;
                        float4 pj = pos4[j];
                        float rv[3] = {(oi[0] - pj.x) + shx, (oi[1] - pj.y) + shy, 0.f};
                        float r2 = rv[0] * rv[0] + rv[1] * rv[1];
                        if (DIM == 3) {
                            rv[2] = (oi[2] - pj.z) + shz;
                            r2 += rv[2] * rv[2];
                        }
                        float hij = pair_h(K, hi, pj.w);
                        if (!(r2 < 4.f * hij * hij) || r2 == 0.f) continue;
                        float r = sqrtf(r2);
                        float dw = wendland_dW<DIM, float>(r, 1.f / hij);
                        float4 oj = vr[j];
                        float vj[3] = {oj.x, oj.y, oj.z};
                        pair_force<float, DIM, Acc>(K, rv, r, dw, vi, rho_i, p_i, vj, oj.w, (float)S.m[j], acc_a,
                                                    acc_R);
                    }
                }
            }
        }
        float a[3] = {0, 0, 0}, R[3] = {0, 0, 0};
        float R2 = 0.f;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            a[d] = K.g[d] + acc_a[d].value();
            R[d] = acc_R[d].value();
            R2 += R[d] * R[d];
        }
        const float htv = K.tv_h_particle ? hi : K.h_min;
        const float htv2 = htv * htv;
        const float chi = tv_limiter(K, htv2 * R2);
        const double m_i = S.m[i];
        double v2 = 0.0, vt2 = 0.0, dr2 = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            size_t o = (size_t)d * n + i;
            float dr = K.tv_xi * chi * htv2 * R[d];
            float vn = __fadd_rn(vi[d], __fmul_rn((float)hdt, a[d]));
            if (write_ad) {
                S.a[o] = a[d];
                S.dr[o] = dr;
            }
            S.v[o] = vn;
            Rout[o] = R[d];
            part[1 + d] = m_i * (double)vn;
            v2 += (double)vn * vn;
            dr2 += (double)dr * dr;
            double vt = dt > 0.0 ? (double)vn + (double)dr / dt : (double)vn;
            vt2 += vt * vt;
        }
        chi_out[i] = chi;
        part[0] = m_i;
        part[4] = 0.5 * m_i * v2;
        part[5] = chi > 0.f ? 1.0 : 0.0;
        part[6] = sqrt(v2);
        part[7] = sqrt(vt2);
        part[8] = sqrt(dr2);
    } else if (i < n) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            if (write_ad) {
                S.a[(size_t)d * n + i] = 0.f;
                S.dr[(size_t)d * n + i] = 0.f;
            }
            Rout[(size_t)d * n + i] = 0.f;
        }
        chi_out[i] = 0.f;
    }
    block_partials(part, partials + (size_t)blockIdx.x * kNPart);
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
        part[6] = sqrt(v2);
        part[7] = sqrt(v2);
        part[8] = sqrt(dr2);
    }
    block_partials(part, partials + (size_t)blockIdx.x * kNPart);
}

// =========================================================== finalize

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
    block_partials(acc, out);
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
        *dt_ptr = dt_next;
    }
}

// ============================================================ launchers

static inline int nblk(int n, int t) { return (n + t - 1) / t; }

int pair_blocks(int n) { return nblk(n, 256); }

cudaError_t launch_density(int prec, int dim, int n, void* S, const int32_t* start, const Grid& G, const void* K,
                           void* vr, const float4* pos4, const int32_t* cell_of, cudaStream_t st)
{
    const int T = 256;
    if (prec == 64) {
        auto s = *(StateSet<double>*)S;
        auto k = *(const Consts<double>*)K;
        if (dim == 2) k_density_f64<2><<<nblk(n, T), T, 0, st>>>(n, s, start, G, k, (double4_32a*)vr);
        else k_density_f64<3><<<nblk(n, T), T, 0, st>>>(n, s, start, G, k, (double4_32a*)vr);
    } else {
        auto s = *(StateSet<float>*)S;
        auto k = *(const Consts<float>*)K;
        if (k.kahan) {
            if (dim == 2) k_density_f32<2, KSum><<<nblk(n, T), T, 0, st>>>(n, pos4, cell_of, start, G, k, s, (float4*)vr);
            else k_density_f32<3, KSum><<<nblk(n, T), T, 0, st>>>(n, pos4, cell_of, start, G, k, s, (float4*)vr);
        } else {
            if (dim == 2) k_density_f32<2, PlainF><<<nblk(n, T), T, 0, st>>>(n, pos4, cell_of, start, G, k, s, (float4*)vr);
            else k_density_f32<3, PlainF><<<nblk(n, T), T, 0, st>>>(n, pos4, cell_of, start, G, k, s, (float4*)vr);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_forces(int prec, int dim, int n, void* S, const int32_t* start, const Grid& G, const void* K,
                          const void* vr, const float4* pos4, const int32_t* cell_of, const double* dt, int kick_on,
                          int write_ad, void* Rout, void* chi, double* partials, cudaStream_t st)
{
    const int T = 256;
    if (prec == 64) {
        auto s = *(StateSet<double>*)S;
        auto k = *(const Consts<double>*)K;
        if (dim == 2)
            k_forces_f64<2><<<nblk(n, T), T, 0, st>>>(n, s, start, G, k, (const double4_32a*)vr, dt, kick_on, write_ad,
                                                      (double*)Rout, (double*)chi, partials);
        else
            k_forces_f64<3><<<nblk(n, T), T, 0, st>>>(n, s, start, G, k, (const double4_32a*)vr, dt, kick_on, write_ad,
                                                      (double*)Rout, (double*)chi, partials);
    } else {
        auto s = *(StateSet<float>*)S;
        auto k = *(const Consts<float>*)K;
#define SPH_F32_FORCES(D, A)                                                                                  \
    k_forces_f32<D, A><<<nblk(n, T), T, 0, st>>>(n, pos4, cell_of, start, G, k, s, (const float4*)vr, dt, kick_on, write_ad, \
                                                 (float*)Rout, (float*)chi, partials)
        if (k.kahan) {
            if (dim == 2) SPH_F32_FORCES(2, KSum);
            else SPH_F32_FORCES(3, KSum);
        } else {
            if (dim == 2) SPH_F32_FORCES(2, PlainF);
            else SPH_F32_FORCES(3, PlainF);
        }
#undef SPH_F32_FORCES
    }
    return cudaGetLastError();
}

cudaError_t launch_diag_only(int prec, int dim, int n, void* S, double* partials, cudaStream_t st)
{
    const int T = 256;
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

cudaError_t launch_finalize(int nblocks, const double* partials, const sph_params& P, double* diag, double* dt,
                            int count_step, cudaStream_t st)
{
    DtConsts D{P.eta, P.rho0, P.h_min, P.u_ref, P.cfl_ad, P.cfl_ac, P.c0, P.fixed_dt};
    k_finalize<<<1, 256, 0, st>>>(nblocks, partials, D, diag, dt, count_step);
    return cudaGetLastError();
}

}  // namespace sphtv
