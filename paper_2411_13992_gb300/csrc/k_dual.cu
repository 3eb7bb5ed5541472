// k_dual.cu -- the dual-criteria time stepping of libsphtv (Sec. 2.4).
//
// One advection step (size Dt_ad, Eq. 9-10) follows the cell sort and the
// density pass; the density pass writes each particle's neighbour list, and
// that list stays frozen for the whole advection step (W' is evaluated at the
// current distance, so a pair that leaves the support stops contributing):
//   k_dual_begin      : Dt_ad, |v|_ad and the first substep size (Eq. 9-11)
//   k_dual_advect     : viscous acceleration (Eq. 7), held for the step, and
//                       the transport correction dr (Eq. 14-16, or Eq. 12
//                       with p0 = 7 rho0 |v|_ad^2 of Eq. 13)
// then acoustic substeps dt = min(dt_ac, Dt_ad - t) (Eq. 11), each
//   k_dual_first_half : rho += dt/2 drho (after completing the previous
//                       substep's second half), x += dr (first substep of the
//                       advection step only), x += dt/2 v
//   k_dual_pressure   : Riemann pressure force (Eq. 3 row 2, Eq. 5-6) + the
//                       held viscous force + g; v += dt a
//   k_dual_drift      : x += dt/2 v
//   k_dual_continuity : drho_i = 2 rho_i sum_j V_j (U* - U_l) dW/dr (Eq. 3
//                       row 1, U* of Eq. 5 row 1), diagnostics partials
//   k_dual_finalize   : reduction; the next substep size; marks the
//                       advection step done after its last substep
// and, once per advection step, k_dual_complete: rho += dt/2 drho of the last
// substep.  Every substep kernel returns at once when the advection step is
// done, so the host launches a few substeps more than it expects and waits
// for the stream once per advection step.
//
// Readings (as in the kick-drift-kick passes): e_ij points from i to j;
// grad W_ij = W'(r) (x_i - x_j)/r; V_j = m_j / rho_j; rho_bar is the mean
// density, c_bar = c; U* uses p_l, p_r for the p_L, p_R of Eq. 5 and no
// limiter; a wall j stands in with rho_j = rho_i, p_j = p_i and its
// prescribed velocity.  The density lives as w = rho - rho0 beside the
// velocity (vr), so the FP32 form keeps the digits of the deviation.
#include <type_traits>

#include "common.cuh"
#include "launch.h"
#include "pair_physics.cuh"

namespace sphtv {

namespace {

template <typename Real> struct V4;
template <> struct V4<float> {
    using T = float4;
    __device__ static T make(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
};
template <> struct V4<double> {
    using T = double4_32a;
    __device__ static T make(double a, double b, double c, double d) { return make_double4_32a(a, b, c, d); }
};

template <typename Real>
struct DualK {
    int n, cap;
    StateSet<Real> S;
    typename V4<Real>::T* vr;
    float4* pos4;            // cell-relative offsets (the FP32 form's drifts keep them current), m or h
    const float* mf;         // FP32 form: masses
    const uint32_t* nbl;
    const int32_t* nbc;
    Real* anu;               // [DIM][n] viscous acceleration held for the advection step
    Real* R;                 // [DIM][n] residual
    Real* chi;               // [n] limiter
    double* du;              // DU_* state
    double* partials;
    uint32_t* err;
};

constexpr int kTPB64 = 256;
constexpr int kTPB32 = 128;
template <typename Real> constexpr int tpb() { return sizeof(Real) == 8 ? kTPB64 : kTPB32; }

__device__ __forceinline__ bool dual_done(const double* du) { return du[DU_DONE] != 0.0; }

// Shared table of the FP32 stencil shifts (FP32 form only).
template <typename Real>
__device__ __forceinline__ void fill_shift_table(const Grid& G, float4* tab)
{
    if (sizeof(Real) == 4) {
        for (int t = threadIdx.x; t < kCodes; t += blockDim.x) {
            float sh[3];
            code_shift(G, (uint32_t)t, sh);
            tab[t] = make_float4(sh[0], sh[1], sh[2], 0.f);
        }
    }
    __syncthreads();
}

// Visit the frozen neighbour list of particle i: f(j, rv, r2, wj, oj) with
// rv the pair vector x_i - x_j at the current positions, wj = pos4[j].w (FP32
// form: m or h) and oj = vr[j].  The FP32 walk keeps the list entries four
// ahead and the neighbour data two ahead in flight.
template <typename Real, int DIM, typename F>
__device__ __forceinline__ void for_list(const DualK<Real>& A, const Grid& G, const float4* tab, int i, int cnt, F& f)
{
    const int n = A.n;
    if constexpr (std::is_same<Real, double>::value) {
        double xi[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int d = 0; d < DIM; ++d) xi[d] = A.S.x[(size_t)d * n + i];
        for (int k = 0; k < cnt; ++k) {
            const int j = (int)(A.nbl[(size_t)k * n + i] >> kCodeBits);
            double rv[3] = {0.0, 0.0, 0.0};
            double r2 = 0.0;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                rv[d] = min_image(G, xi[d], A.S.x[(size_t)d * n + j], d);
                r2 += rv[d] * rv[d];
            }
            f(j, rv, r2, 0.f, A.vr[j]);
        }
    } else {
        const float4 pi = A.pos4[i];
        const float oi[3] = {pi.x, pi.y, pi.z};
        const uint32_t* lp = A.nbl + i;
        auto one = [&](uint32_t ec, const float4& pj, const float4& oj) {
            const float4 sh = tab[ec & ((1u << kCodeBits) - 1u)];
            float rv[3] = {0.f, 0.f, 0.f};
            rv[0] = (oi[0] - pj.x) + sh.x;
            rv[1] = (oi[1] - pj.y) + sh.y;
            float r2 = rv[0] * rv[0] + rv[1] * rv[1];
            if (DIM == 3) {
                rv[2] = (oi[2] - pj.z) + sh.z;
                r2 += rv[2] * rv[2];
            }
            f((int)(ec >> kCodeBits), rv, r2, pj.w, oj);
        };
        // two pairs per iteration, in list order: the next iteration's two
        // pairs of neighbour data and the entries of the one after in flight,
        // the entries through a pointer that advances by two rows
        uint32_t e0 = cnt > 0 ? lp[0] : 0u;
        uint32_t e1 = cnt > 1 ? lp[(size_t)n] : 0u;
        uint32_t e2 = cnt > 2 ? lp[2 * (size_t)n] : 0u;
        uint32_t e3 = cnt > 3 ? lp[3 * (size_t)n] : 0u;
        float4 p0 = A.pos4[e0 >> kCodeBits], o0 = A.vr[e0 >> kCodeBits];
        float4 p1 = A.pos4[e1 >> kCodeBits], o1 = A.vr[e1 >> kCodeBits];
        int k = 0;
        const uint32_t* lq = lp + 4 * (size_t)n;
        const size_t n2 = 2 * (size_t)n;
        for (; k + 1 < cnt; k += 2, lq += n2) {
            const float4 p2 = A.pos4[e2 >> kCodeBits], o2 = A.vr[e2 >> kCodeBits];
            const float4 p3 = A.pos4[e3 >> kCodeBits], o3 = A.vr[e3 >> kCodeBits];
            const uint32_t e4 = k + 4 < cnt ? lq[0] : 0u;
            const uint32_t e5 = k + 5 < cnt ? lq[n] : 0u;
            one(e0, p0, o0);
            one(e1, p1, o1);
            p0 = p2; o0 = o2; p1 = p3; o1 = o3;
            e0 = e2; e1 = e3; e2 = e4; e3 = e5;
        }
        if (k < cnt) one(e0, p0, o0);
    }
}

// Smoothing length and mass of particle j (wj = pos4[j].w in the FP32 form).
template <typename Real, bool UNIFORM>
__device__ __forceinline__ void h_m_of(const DualK<Real>& A, const Consts<Real>& K, int j, float wj, Real& h, Real& m)
{
    if constexpr (std::is_same<Real, double>::value) {
        h = A.S.h[j];
        m = A.S.m[j];
    } else {
        h = UNIFORM ? K.h_u : wj;
        m = UNIFORM ? wj : A.mf[j];
    }
}

// 1/r, r and W'(r, h_ij)/r of a pair, zero at and beyond the support 2 h_ij
// (the list is frozen while the particles move).  FP64: IEEE operations;
// FP32: rsqrt and W'/r = coef t^3, t = max(1 - r/(2h), 0).
template <typename Real>
struct PairGeo {
    Real inv_r, r, dwr;
};

template <typename Real, int DIM, bool UNIFORM>
__device__ __forceinline__ PairGeo<Real> pair_geo(const Consts<Real>& K, Real r2, Real hi, Real hj)
{
    PairGeo<Real> g;
    if constexpr (std::is_same<Real, double>::value) {
        g.r = sqrt(r2);
        g.inv_r = 1.0 / g.r;
        const double h = pair_h(K, hi, hj);
        g.dwr = g.r < 2.0 * h ? wendland_dW<DIM, double>(g.r, 1.0 / h) * g.inv_r : 0.0;
    } else {
        g.inv_r = rsqrtf(r2);
        g.r = r2 * g.inv_r;
        float inv_h, coef;
        if (UNIFORM) {
            inv_h = K.inv_h_u;
            coef = K.dwr_coef_u;
        } else {
            inv_h = __frcp_rn(pair_h(K, hi, hj));
            coef = -5.f * kernel_norm<DIM, float>() * pow_dim<DIM, float>(inv_h) * inv_h * inv_h;
        }
        const float t = fmaxf(fmaf(-0.5f * inv_h, g.r, 1.f), 0.f);
        g.dwr = coef * (t * t * t);
    }
    return g;
}

template <typename Real>
__device__ __forceinline__ Real recip(Real x)
{
    if constexpr (std::is_same<Real, double>::value) return 1.0 / x;
    else return rcp_approx(x);
}

template <typename Real>
__device__ __forceinline__ Real fma_free_add(Real a, Real b);
template <> __device__ __forceinline__ double fma_free_add<double>(double a, double b) { return __dadd_rn(a, b); }
template <> __device__ __forceinline__ float fma_free_add<float>(float a, float b) { return __fadd_rn(a, b); }
template <typename Real>
__device__ __forceinline__ Real fma_free_mul(Real a, Real b);
template <> __device__ __forceinline__ double fma_free_mul<double>(double a, double b) { return __dmul_rn(a, b); }
template <> __device__ __forceinline__ float fma_free_mul<float>(float a, float b) { return __fmul_rn(a, b); }

}  // namespace

// ------------------------------------------------------------------ begin

struct DualConsts {
    double eta, rho0, h_min, u_ref, cfl_ad, cfl_ac, c;
};

// Eq. 9-11 with h = h_min from max |v| of the fluid (the diagnostics of the
// previous step or of sph_build_cells; the sort does not change v).
__global__ void k_dual_begin(DualConsts D, const double* __restrict__ diag, double* __restrict__ du)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double vmax = diag[DG_VMAX];
    const double nu = D.eta / D.rho0;
    const double vad = fmax(vmax, fmax(nu / D.h_min, D.u_ref));
    const double Dt = D.cfl_ad * D.h_min / vad;
    double dt = D.cfl_ac * D.h_min / (vmax + D.c);
    const double rem = Dt - 0.0;
    const int last = !(dt < rem);      // also ends the step on a non-finite size
    if (last) dt = rem;
    du[DU_DT_AD] = Dt;
    du[DU_VAD] = vad;
    du[DU_T] = 0.0;
    du[DU_DT] = dt;
    du[DU_HDT_PREV] = 0.0;
    du[DU_LAST] = last;
    du[DU_DONE] = 0.0;
    du[DU_K] = 0.0;
    du[DU_FIRST] = 1.0;
}

// ----------------------------------------------------------------- advect

template <typename Real, int DIM, typename Acc, bool UNIFORM>
__global__ void __launch_bounds__(sizeof(Real) == 8 ? 256 : 128) k_dual_advect(DualK<Real> A, Grid G, Consts<Real> K)
{
    __shared__ float4 tab[kCodes];
    fill_shift_table<Real>(G, tab);
    const int n = A.n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (A.S.kind[i]) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            A.anu[(size_t)d * n + i] = Real(0);
            A.R[(size_t)d * n + i] = Real(0);
            A.S.dr[(size_t)d * n + i] = Real(0);
        }
        A.chi[i] = Real(0);
        return;
    }
    int cnt = A.nbc[i];
    if (cnt > A.cap) {
        atomicOr(A.err, ERRB_OVERFLOW);
        cnt = A.cap;
    }
    const auto me = A.vr[i];
    const Real vi[3] = {me.x, me.y, me.z};
    const Real rho_i = K.rho0 + me.w;
    const Real inv_rho_i = recip(rho_i);
    Real hi, mi;
    {
        float wi = 0.f;
        if constexpr (!std::is_same<Real, double>::value) wi = A.pos4[i].w;
        h_m_of<Real, UNIFORM>(A, K, i, wi, hi, mi);
    }
    Acc acc_nu[DIM], acc_R[DIM];
    auto pair = [&](int j, const Real* rv, Real r2, float wj, const typename V4<Real>::T& oj) {
        if (!(r2 > Real(0))) return;
        Real hj, mj;
        h_m_of<Real, UNIFORM>(A, K, j, wj, hj, mj);
        const PairGeo<Real> g = pair_geo<Real, DIM, UNIFORM>(K, r2, hi, hj);
        const bool wall = isinf(oj.w);
        const Real inv_rho_j = wall ? inv_rho_i : recip(K.rho0 + oj.w);
        const Real cv = K.two_eta * mj * inv_rho_i * inv_rho_j * g.dwr;   // Eq. 7
        const Real vw = mj * inv_rho_j * g.dwr;                           // V_j W'/r
        const Real vj[3] = {oj.x, oj.y, oj.z};
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            acc_nu[d].add(cv * (vi[d] - vj[d]));
            acc_R[d].add(vw * rv[d]);
        }
    };
    for_list<Real, DIM>(A, G, tab, i, cnt, pair);
    Real R[3] = {0, 0, 0}, R2 = 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        R[d] = acc_R[d].value();
        R2 += R[d] * R[d];
        A.anu[(size_t)d * n + i] = acc_nu[d].value();
        A.R[(size_t)d * n + i] = R[d];
    }
    const Real htv = K.tv_h_particle ? hi : K.h_min;
    const Real chi = tv_limiter(K, htv * htv * R2);
    A.chi[i] = chi;
    // Eq. 12 with p0 = 7 rho0 |v|_ad^2 (Eq. 13): dr = -(Dt^2 p0 / rho_i) R_i
    const double Dt = A.du[DU_DT_AD], vad = A.du[DU_VAD];
    const double p0 = 7.0 * (double)K.rho0 * vad * vad;
    const double bg = -(Dt * Dt * p0 / (double)rho_i);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const Real dr = K.tv_mode == SPH_TV_BACKGROUND ? (Real)(bg * (double)R[d])
                                                       : K.tv_xi * chi * htv * htv * R[d];
        A.S.dr[(size_t)d * n + i] = dr;
    }
}

// ------------------------------------------------------------- substeps

template <typename Real, int DIM>
__global__ void __launch_bounds__(256) k_dual_first_half(DualK<Real> A, Grid G)
{
    if (dual_done(A.du)) return;
    const int n = A.n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || A.S.kind[i]) return;
    const double dt = A.du[DU_DT];
    const double hdt = 0.5 * dt;
    const bool first = A.du[DU_FIRST] != 0.0;
    auto me = A.vr[i];
    Real w = me.w;
    const Real dr = A.S.drho[i];
    if (!first) w = fma_free_add<Real>(w, fma_free_mul<Real>((Real)A.du[DU_HDT_PREV], dr));
    w = fma_free_add<Real>(w, fma_free_mul<Real>((Real)hdt, dr));
    me.w = w;
    A.vr[i] = me;
    // FP32 form: the cell-relative offsets take the same displacement in
    // FP32 (the permute recomputes them from the FP64 positions at the next
    // advection step), which keeps the FP64 origin arithmetic off the
    // substeps
    float4 p = sizeof(Real) == 4 ? A.pos4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    float of[3] = {p.x, p.y, p.z};
    const float hdtf = (float)hdt;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const size_t o = (size_t)d * n + i;
        const Real v = A.S.v[o];
        double x = A.S.x[o];
        if (first) {
            const Real drd = A.S.dr[o];
            x = __dadd_rn(x, (double)drd);
            of[d] = __fadd_rn(of[d], (float)drd);
        }
        x = __dadd_rn(x, __dmul_rn(hdt, (double)v));
        of[d] = __fmaf_rn(hdtf, (float)v, of[d]);
        A.S.x[o] = x;
    }
    if (sizeof(Real) == 4) A.pos4[i] = make_float4(of[0], of[1], of[2], p.w);
}

template <typename Real, int DIM, typename Acc, bool UNIFORM>
__global__ void __launch_bounds__(sizeof(Real) == 8 ? 256 : 128) k_dual_pressure(DualK<Real> A, Grid G, Consts<Real> K)
{
    __shared__ float4 tab[kCodes];
    if (dual_done(A.du)) return;
    fill_shift_table<Real>(G, tab);
    const int n = A.n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || A.S.kind[i]) return;
    const int cnt = min(A.nbc[i], A.cap);
    const double dt = A.du[DU_DT];
    const auto me = A.vr[i];
    const Real vi[3] = {me.x, me.y, me.z};
    const Real rho_i = K.rho0 + me.w;
    const Real inv_rho_i = recip(rho_i);
    const Real p_i = K.c2 * me.w;
    Real hi, mi;
    {
        float wi = 0.f;
        if constexpr (!std::is_same<Real, double>::value) wi = A.pos4[i].w;
        h_m_of<Real, UNIFORM>(A, K, i, wi, hi, mi);
    }
    Acc acc[DIM];
    auto pair = [&](int j, const Real* rv, Real r2, float wj, const typename V4<Real>::T& oj) {
        if (!(r2 > Real(0))) return;
        Real hj, mj;
        h_m_of<Real, UNIFORM>(A, K, j, wj, hj, mj);
        const PairGeo<Real> g = pair_geo<Real, DIM, UNIFORM>(K, r2, hi, hj);
        const bool wall = isinf(oj.w);
        const Real rho_j = wall ? rho_i : K.rho0 + oj.w;
        const Real inv_rho_j = wall ? inv_rho_i : recip(rho_j);
        const Real p_j = wall ? p_i : K.c2 * oj.w;
        Real dvr = (vi[0] - oj.x) * rv[0] + (vi[1] - oj.y) * rv[1];
        if (DIM == 3) dvr += (vi[2] - oj.z) * rv[2];
        const Real du = -dvr * g.inv_r;                        // U_l - U_r, e_ij from i to j
        Real beta = K.beta_slope * (du * K.inv_c);             // Eq. 6
        beta = beta > Real(0) ? beta : Real(0);
        beta = beta < Real(1) ? beta : Real(1);
        const Real rhobar = Real(0.5) * (rho_i + rho_j);
        const Real pstar = Real(0.5) * (p_i + p_j) + Real(0.5) * beta * rhobar * K.c * du;   // Eq. 5
        const Real cpw = Real(-2) * mj * inv_rho_i * inv_rho_j * pstar * g.dwr;           // Eq. 3
#pragma unroll
        for (int d = 0; d < DIM; ++d) acc[d].add(cpw * rv[d]);
    };
    for_list<Real, DIM>(A, G, tab, i, cnt, pair);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const size_t o = (size_t)d * n + i;
        const Real a = (acc[d].value() + A.anu[o]) + K.g[d];
        A.S.a[o] = a;
        A.S.v[o] = fma_free_add<Real>(A.S.v[o], fma_free_mul<Real>((Real)dt, a));
    }
}

template <typename Real, int DIM>
__global__ void __launch_bounds__(256) k_dual_drift(DualK<Real> A, Grid G)
{
    if (dual_done(A.du)) return;
    const int n = A.n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || A.S.kind[i]) return;
    const double hdt = 0.5 * A.du[DU_DT];
    const float hdtf = (float)hdt;
    float4 p = sizeof(Real) == 4 ? A.pos4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    float of[3] = {p.x, p.y, p.z};
    Real v[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const size_t o = (size_t)d * n + i;
        v[d] = A.S.v[o];
        A.S.x[o] = __dadd_rn(A.S.x[o], __dmul_rn(hdt, (double)v[d]));
        of[d] = __fmaf_rn(hdtf, (float)v[d], of[d]);    // the offsets follow in FP32 (k_dual_first_half)
    }
    const Real w = A.vr[i].w;
    A.vr[i] = V4<Real>::make(v[0], v[1], v[2], w);
    if (sizeof(Real) == 4) A.pos4[i] = make_float4(of[0], of[1], of[2], p.w);
}

template <typename Real, int DIM, typename Acc, bool UNIFORM>
__global__ void __launch_bounds__(sizeof(Real) == 8 ? 256 : 128) k_dual_continuity(DualK<Real> A, Grid G, Consts<Real> K)
{
    __shared__ float4 tab[kCodes];
    if (dual_done(A.du)) return;
    fill_shift_table<Real>(G, tab);
    const int n = A.n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double part[kNPart];
#pragma unroll
    for (int k = 0; k < kNPart; ++k) part[k] = 0.0;
    if (i < n && A.S.kind[i] == 0) {
        const int cnt = min(A.nbc[i], A.cap);
        const auto me = A.vr[i];
        const Real vi[3] = {me.x, me.y, me.z};
        const Real rho_i = K.rho0 + me.w;
        const Real inv_rho_i = recip(rho_i);
        const Real p_i = K.c2 * me.w;
        Real hi, mi;
        {
            float wi = 0.f;
            if constexpr (!std::is_same<Real, double>::value) wi = A.pos4[i].w;
            h_m_of<Real, UNIFORM>(A, K, i, wi, hi, mi);
        }
        Acc s;
        auto pair = [&](int j, const Real* rv, Real r2, float wj, const typename V4<Real>::T& oj) {
            if (!(r2 > Real(0))) return;
            Real hj, mj;
            h_m_of<Real, UNIFORM>(A, K, j, wj, hj, mj);
            const PairGeo<Real> g = pair_geo<Real, DIM, UNIFORM>(K, r2, hi, hj);
            const bool wall = isinf(oj.w);
            const Real rho_j = wall ? rho_i : K.rho0 + oj.w;
            const Real inv_rho_j = wall ? inv_rho_i : recip(rho_j);
            const Real p_j = wall ? p_i : K.c2 * oj.w;
            Real dvr = (vi[0] - oj.x) * rv[0] + (vi[1] - oj.y) * rv[1];
            if (DIM == 3) dvr += (vi[2] - oj.z) * rv[2];
            // U* - U_l = (U_r - U_l)/2 + (p_l - p_r) / (2 rho_bar c)   (Eq. 5, first row)
            const Real rhobar = Real(0.5) * (rho_i + rho_j);
            const Real dus = Real(0.5) * dvr * g.inv_r + Real(0.5) * (p_i - p_j) * recip(rhobar) * K.inv_c;
            // V_j (U* - U_l) dW/dr, dW/dr = (W'/r) r
            s.add(mj * inv_rho_j * dus * (g.dwr * g.r));
        };
        for_list<Real, DIM>(A, G, tab, i, cnt, pair);
        A.S.drho[i] = Real(2) * rho_i * s.value();
        // max |v| for the next substep size, from |v|^2 in the precision of v;
        // the other diagnostics (and |v|^2 in FP64 for the kinetic energy) only
        // after the last substep of the advection step (FP64 is 1/74 of the
        // FP32 rate)
        Real v2r = Real(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const Real v = A.S.v[(size_t)d * n + i];
            v2r += v * v;
        }
        part[6] = (double)v2r;        // squares: block_partials takes the roots
        if (A.du[DU_LAST] != 0.0) {
            double v2 = 0.0;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const double v = (double)A.S.v[(size_t)d * n + i];
                v2 += v * v;
            }
            part[6] = v2;
            const double inv_Dt = 1.0 / A.du[DU_DT_AD];
            const double m_i = A.S.m[i];
            double vt2 = 0.0, dr2 = 0.0;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const size_t o = (size_t)d * n + i;
                const double v = (double)A.S.v[o];
                const double dr = (double)A.S.dr[o];
                part[1 + d] = m_i * v;
                dr2 += dr * dr;
                const double vt = v + dr * inv_Dt;
                vt2 += vt * vt;
            }
            part[0] = m_i;
            part[4] = 0.5 * m_i * v2;
            part[5] = A.chi[i] > Real(0) ? 1.0 : 0.0;
            part[7] = vt2;
            part[8] = dr2;
        }
    } else if (i < n) {
        A.S.drho[i] = Real(0);
    }
    // the sums (mass, momentum, KE) only after the last substep: in the others
    // they are all zero, and their FP64 shuffles would cost every substep
    block_partials<true>(part, A.partials + (size_t)blockIdx.x * kNPart, A.du[DU_LAST] != 0.0);
}

// Reduce the substep's partials (in a fixed order); advance t; pick the next
// substep size, or finish the advection step and write the diagnostics.
__global__ void __launch_bounds__(256) k_dual_finalize(int nblocks, const double* __restrict__ partials, DualConsts D,
                                                       double* __restrict__ du, double* __restrict__ diag,
                                                       double* __restrict__ dt_ptr)
{
    if (dual_done(du)) return;
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
    if (threadIdx.x != 0) return;
    const double vmax = out[6];
    const double dt = du[DU_DT];
    const double t = du[DU_T] + dt;
    const double k = du[DU_K] + 1.0;
    du[DU_T] = t;
    du[DU_K] = k;
    du[DU_HDT_PREV] = 0.5 * dt;
    du[DU_FIRST] = 0.0;
    if (du[DU_LAST] != 0.0) {
        const double Dt = du[DU_DT_AD];
        const double nu = D.eta / D.rho0;
        const double vad = fmax(vmax, fmax(nu / D.h_min, D.u_ref));
        diag[DG_MASS] = out[0];
        diag[DG_MOM + 0] = out[1];
        diag[DG_MOM + 1] = out[2];
        diag[DG_MOM + 2] = out[3];
        diag[DG_KE] = out[4];
        diag[DG_NCHI] = out[5];
        diag[DG_VMAX] = vmax;
        diag[DG_VTMAX] = out[7];
        diag[DG_DRMAX] = out[8];
        diag[DG_DT] = Dt;
        diag[DG_DTNEXT] = D.cfl_ad * D.h_min / vad;
        diag[DG_STEPS] = diag[DG_STEPS] + 1.0;
        diag[DG_SUBSTEPS] = k;
        *dt_ptr = Dt;
        du[DU_DONE] = 1.0;
        return;
    }
    double dtn = D.cfl_ac * D.h_min / (vmax + D.c);
    const double rem = du[DU_DT_AD] - t;
    const int last = !(dtn < rem);     // also ends the step on a non-finite size
    if (last) dtn = rem;
    du[DU_DT] = dtn;
    du[DU_LAST] = last;
}

// Second half of the last substep's density update: rho += dt/2 drho.
template <typename Real>
__global__ void __launch_bounds__(256) k_dual_complete(DualK<Real> A)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n || A.S.kind[i]) return;
    auto me = A.vr[i];
    me.w = fma_free_add<Real>(me.w, fma_free_mul<Real>((Real)A.du[DU_HDT_PREV], A.S.drho[i]));
    A.vr[i] = me;
}

// ============================================================ launchers

namespace {

inline int nblk(int n, int t) { return (n + t - 1) / t; }

template <typename Real>
DualK<Real> dual_k(const DualArgs& a)
{
    DualK<Real> k;
    k.n = a.n;
    k.cap = a.cap;
    k.S = *(const StateSet<Real>*)a.S;
    k.vr = (typename V4<Real>::T*)a.vr;
    k.pos4 = a.pos4;
    k.mf = a.mf;
    k.nbl = a.nbl;
    k.nbc = a.nbc;
    k.anu = (Real*)a.anu;
    k.R = (Real*)a.R;
    k.chi = (Real*)a.chi;
    k.du = a.du;
    k.partials = a.partials;
    k.err = a.err;
    return k;
}

DualConsts dual_consts(const sph_params& P)
{
    return DualConsts{P.eta, P.rho0, P.h_min, P.u_ref, P.cfl_ad, P.cfl_ac, P.c0};
}

// Pair kernel dispatch: precision, dimension, compensated sums (FP32) and
// uniform resolution (FP32) are template arguments.
template <template <typename, int, typename, bool> class Kern> struct Dispatch;

#define SPH_DUAL_PAIR_KERNEL(name)                                                                         \
    template <typename Real, int DIM, typename Acc, bool U>                                                \
    struct name##_t {                                                                                      \
        static void run(const DualK<Real>& A, const Grid& G, const Consts<Real>& K, cudaStream_t st)     \
        {                                                                                                  \
            const int T = pair_threads(sizeof(Real) == 8 ? 64 : 32, A.n, G.sms);                            \
            name<Real, DIM, Acc, U><<<nblk(A.n, T), T, 0, st>>>(A, G, K);                                    \
        }                                                                                                  \
    };
SPH_DUAL_PAIR_KERNEL(k_dual_advect)
SPH_DUAL_PAIR_KERNEL(k_dual_pressure)
SPH_DUAL_PAIR_KERNEL(k_dual_continuity)
#undef SPH_DUAL_PAIR_KERNEL

template <template <typename, int, typename, bool> class KT>
void run_pair(int prec, int dim, const DualArgs& a, const Grid& G, const void* Kp, cudaStream_t st)
{
    if (prec == 64) {
        const auto A = dual_k<double>(a);
        const auto& K = *(const Consts<double>*)Kp;
        if (dim == 2) KT<double, 2, PlainD, false>::run(A, G, K, st);
        else KT<double, 3, PlainD, false>::run(A, G, K, st);
        return;
    }
    const auto A = dual_k<float>(a);
    const auto& K = *(const Consts<float>*)Kp;
    const bool u = K.uniform_h != 0, ks = K.kahan != 0;
    if (dim == 2) {
        if (ks) u ? KT<float, 2, KSum, true>::run(A, G, K, st) : KT<float, 2, KSum, false>::run(A, G, K, st);
        else u ? KT<float, 2, PlainF, true>::run(A, G, K, st) : KT<float, 2, PlainF, false>::run(A, G, K, st);
    } else {
        if (ks) u ? KT<float, 3, KSum, true>::run(A, G, K, st) : KT<float, 3, KSum, false>::run(A, G, K, st);
        else u ? KT<float, 3, PlainF, true>::run(A, G, K, st) : KT<float, 3, PlainF, false>::run(A, G, K, st);
    }
}

template <typename Real>
void run_elem(int dim, const DualArgs& a, const Grid& G, int which, cudaStream_t st)
{
    const auto A = dual_k<Real>(a);
    const int T = 256, B = nblk(A.n, T);
    if (which == 0) {
        if (dim == 2) k_dual_first_half<Real, 2><<<B, T, 0, st>>>(A, G);
        else k_dual_first_half<Real, 3><<<B, T, 0, st>>>(A, G);
    } else if (which == 1) {
        if (dim == 2) k_dual_drift<Real, 2><<<B, T, 0, st>>>(A, G);
        else k_dual_drift<Real, 3><<<B, T, 0, st>>>(A, G);
    } else {
        k_dual_complete<Real><<<B, T, 0, st>>>(A);
    }
}

}  // namespace

int dual_pair_blocks(int prec, int n, int sms) { return pair_blocks(prec, n, sms); }

cudaError_t launch_dual_begin(const sph_params& P, const double* diag, double* du, cudaStream_t st)
{
    k_dual_begin<<<1, 32, 0, st>>>(dual_consts(P), diag, du);
    return cudaGetLastError();
}

cudaError_t launch_dual_advect(int prec, int dim, const DualArgs& a, const Grid& G, const void* K, cudaStream_t st)
{
    run_pair<k_dual_advect_t>(prec, dim, a, G, K, st);
    return cudaGetLastError();
}

cudaError_t launch_dual_substep(int prec, int dim, const DualArgs& a, const Grid& G, const void* K,
                                const sph_params& P, double* diag, double* dt_ptr, cudaStream_t st,
                                int64_t* launches)
{
    if (prec == 64) run_elem<double>(dim, a, G, 0, st);
    else run_elem<float>(dim, a, G, 0, st);
    run_pair<k_dual_pressure_t>(prec, dim, a, G, K, st);
    if (prec == 64) run_elem<double>(dim, a, G, 1, st);
    else run_elem<float>(dim, a, G, 1, st);
    run_pair<k_dual_continuity_t>(prec, dim, a, G, K, st);
    const int nb = dual_pair_blocks(prec, a.n, G.sms);
    const int rows = launch_reduce_rows(nb, a.partials, a.rows, st);
    k_dual_finalize<<<1, 256, 0, st>>>(rows ? rows : nb, rows ? a.rows : a.partials, dual_consts(P), a.du, diag,
                                       dt_ptr);
    *launches += rows ? 6 : 5;
    return cudaGetLastError();
}

cudaError_t launch_dual_complete(int prec, const DualArgs& a, cudaStream_t st)
{
    if (prec == 64) run_elem<double>(2, a, Grid{}, 2, st);
    else run_elem<float>(2, a, Grid{}, 2, st);
    return cudaGetLastError();
}

}  // namespace sphtv
