// k_pair32.cu -- FP32 pair passes of libsphtv (density and fused forces),
// one thread per cell-sorted particle.
//
// The density pass scans the 5^D cells around each particle (cell-relative
// FP32 positions; lanes that share a cell load the same candidate at the
// same time), sums sigma, and records the particle's force neighbours in a
// transposed list in HBM (entry k of particle i at k * n + i, so a warp's
// list reads are coalesced).  The force pass then runs the pair body over
// that list only: about 80 neighbours per particle in 3-D instead of about
// 275 candidates, and no lane waits on another lane's candidate tests.  A
// particle with more neighbours than the list holds scans its cells again.
//
// Pair vectors keep full FP32 precision: r_ij = (o_i - o_j) + s, where o are
// offsets from each particle's cell origin and s = -(cell step) x edge is
// exact in FP32.
//
// Method (see k_pair.cu for the FP64 form and pair_physics.cuh for the
// readings of the paper): density Eq. 8 with Eq. 2; pressure Eq. 3, 5, 6;
// viscous Eq. 7; residual, limiter and displacement Eq. 14-16.
#include "common.cuh"
#include "launch.h"
#include "pair_physics.cuh"
#include "pair_walk.cuh"

namespace sphtv {

constexpr int kTPB32 = 128;      // threads per block of the FP32 pair kernels

// Support radius squared of a pair: 4 h_ij^2.
template <bool UNIFORM>
__device__ __forceinline__ float support2(const Consts<float>& K, float hi, float hj)
{
    if (UNIFORM) return K.four_h2_u;
    float h = pair_h(K, hi, hj);
    return 4.f * h * h;
}

// The force pass's sums a_i and R_i (DIM components each).  Generic form:
// one accumulator per component.
template <int DIM, typename Acc>
struct PairSums {
    Acc a[DIM], R[DIM];
    __device__ __forceinline__ void add(const float* xa, const float* xR)
    {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            a[d].add(xa[d]);
            R[d].add(xR[d]);
        }
    }
    __device__ __forceinline__ float a_value(int d) const { return a[d].value(); }
    __device__ __forceinline__ float R_value(int d) const { return R[d].value(); }
};

// Compensated form: the same Kahan steps as KSum, component by component,
// taken two components at a time in packed FP32x2 arithmetic (each lane of a
// packed operation is the IEEE operation of KSum, so the sums are bit for
// bit those of six KSum accumulators).  Components: (a0, a1), (a2, R0),
// (R1, R2) in 3-D; (a0, a1), (R0, R1) in 2-D.
struct KSum2 {
    float2 s, c;
    __device__ __forceinline__ KSum2() : s(make_float2(0.f, 0.f)), c(make_float2(0.f, 0.f)) {}
    __device__ __forceinline__ void add(float2 x)
    {
        const float2 m1 = make_float2(-1.f, -1.f);
        const float2 y = __ffma2_rn(c, m1, x);      // x - c
        const float2 t = __fadd2_rn(s, y);
        const float2 u = __ffma2_rn(s, m1, t);      // t - s
        c = __ffma2_rn(y, m1, u);                   // (t - s) - y
        s = t;
    }
};

template <int DIM>
struct PairSums<DIM, KSum> {
    KSum2 p[DIM];
    __device__ __forceinline__ void add(const float* xa, const float* xR)
    {
        if (DIM == 3) {
            p[0].add(make_float2(xa[0], xa[1]));
            p[1].add(make_float2(xa[2], xR[0]));
            p[2].add(make_float2(xR[1], xR[2]));
        } else {
            p[0].add(make_float2(xa[0], xa[1]));
            p[1].add(make_float2(xR[0], xR[1]));
        }
    }
    __device__ __forceinline__ float a_value(int d) const
    {
        return d == 0 ? p[0].s.x : (d == 1 ? p[0].s.y : p[1].s.x);
    }
    __device__ __forceinline__ float R_value(int d) const
    {
        if (DIM == 2) return d == 0 ? p[1].s.x : p[1].s.y;
        return d == 0 ? p[1].s.y : (d == 1 ? p[2].s.x : p[2].s.y);
    }
};

// One neighbour's contribution to a_i and R_i in the FP32 form, given
// rv = x_i - x_j, 1/r and dwr = W'(r)/r: the same formulas as pair_force64
// (Eq. 3, 5-7, 14) arranged for FP32 throughput -- W' only enters through
// W'/r, (U_l - U_r) = -(v_i - v_j).r_ij / r, and each density is inverted
// once (1/(rho_i rho_j) = (1/rho_i)(1/rho_j), V_j = m_j/rho_j).
template <int DIM, typename Acc>
__device__ __forceinline__ void pair_force32(const Consts<float>& K, const float* rv, float inv_r, float dwr,
                                             const float* vi, float rho_i, float inv_rho_i, float p_i,
                                             const float4& oj, float m_j, PairSums<DIM, Acc>& sums)
{
    const bool wall = isinf(oj.w);
    const float rho_j = wall ? rho_i : K.rho0 + oj.w;
    const float inv_rho_j = wall ? inv_rho_i : rcp_approx(rho_j);
    const float p_j = wall ? p_i : K.c2 * oj.w;
    const float dv[3] = {vi[0] - oj.x, vi[1] - oj.y, DIM == 3 ? vi[2] - oj.z : 0.f};
    float dvr = dv[0] * rv[0] + dv[1] * rv[1];
    if (DIM == 3) dvr += dv[2] * rv[2];
    const float du = -dvr * inv_r;                       // U_l - U_r, e_ij from i to j
    float beta = K.beta_slope * (du * K.inv_c);
    beta = fminf(fmaxf(beta, 0.f), 1.f);
    const float rhobar = 0.5f * (rho_i + rho_j);
    const float pstar = 0.5f * (p_i + p_j) + 0.5f * beta * rhobar * K.c * du;
    const float mr = m_j * inv_rho_i * inv_rho_j;        // m_j / (rho_i rho_j)
    const float cpw = -2.f * mr * pstar * dwr;           // pressure: cp * W'/r
    const float cv = K.two_eta * mr * dwr;               // viscous
    const float vw = m_j * inv_rho_j * dwr;              // residual: V_j W'/r
    float xa[DIM], xR[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        xa[d] = cpw * rv[d] + cv * dv[d];
        xR[d] = vw * rv[d];
    }
    sums.add(xa, xR);
}

// W'(r)/r for r < 2h: a_D h^-(D+2) (-5) t^3 with t = 1 - r/(2h).
template <int DIM>
__device__ __forceinline__ float dwr_of(float r, float inv_h, float coef)
{
    const float t = fmaf(-0.5f * inv_h, r, 1.f);
    return coef * (t * t * t);
}

// sigma_i's term of one candidate at uniform resolution: W(r) inside the
// support, 0 outside (t = 1 - q/2 set to 0).  Every candidate of the walk
// adds its term to the compensated sum, so no lane of a warp waits on
// another lane's accept branch for the kernel value; wnorm = a_D h^-D.
__device__ __forceinline__ float w_term_uniform(const Consts<float>& K, float wnorm, float r2)
{
    const bool in = r2 < K.four_h2_u;
    const float r = sqrt_approx(r2);
    float t = fmaf(-0.5f * K.inv_h_u, r, 1.f);
    t = in ? t : 0.f;
    const float t2 = t * t;
    return wnorm * (t2 * t2) * fmaf(2.f * K.inv_h_u, r, 1.f);
}

// One candidate's neighbour-list step, predicated (no branch): a force
// neighbour (0 < r^2 < 4h^2) takes slot cnt of the particle's transposed list
// (at base_i + cnt x the list's row stride) while the list has room, and is
// counted either way.  The entry is written once and read once (by the force
// pass): a streaming store.
__device__ __forceinline__ void list_take(const uint32_t* base_i, int& cnt, float r2, float four_h2, int cap,
                                          uint32_t entry, uint32_t stride_bytes)
{
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t.reg .u64 a;\n\t"
        "setp.lt.f32 p, %1, %2;\n\t"
        "setp.gt.and.f32 p, %1, 0f00000000, p;\n\t"
        "setp.lt.and.s32 q, %0, %3, p;\n\t"
        "mad.wide.u32 a, %0, %6, %5;\n\t"
        "@q st.global.cs.u32 [a], %4;\n\t"
        "@p add.s32 %0, %0, 1;\n\t}"
        : "+r"(cnt)
        : "f"(r2), "f"(four_h2), "r"(cap), "r"(entry), "l"(base_i), "r"(stride_bytes));
}

// The uniform-resolution density walk: the candidates, their order and their
// arithmetic are those of for_candidates_rows<DIM, true, true> with the
// density visit (rows by (dz, dy); each row cut to the sub-cells inside the
// half-chord, as one run of the sort order or, across a periodic x boundary,
// two; two candidates per iteration).  A run of odd length takes its last
// candidate with a second one whose distance is set far outside the support
// (no term of the sum, no list entry) instead of a separate one-candidate
// loop, and the list entry (j << 7) | code is formed as
// (j << 7) + dx + code of the row's dx = 0 cell.  A row that no lane of the
// warp needs is skipped by a vote; a lane that does not need a row the warp
// walks takes an empty run.  INNER: every particle of the warp lies R cells
// or more from both x ends of the grid, so that no row wraps or is clipped
// along x and the run bounds need no case analysis.
template <int DIM, typename Acc, bool INNER>
__device__ __forceinline__ void density_rows(const float* oi, const int* c, const Grid& G, const Consts<float>& K,
                                             float wnorm, const int32_t* __restrict__ rstart,
                                             const float4* __restrict__ pos4c, Acc& sigma, int& cnt,
                                             const uint32_t* base_i, int n, int cap)
{
    constexpr int R = kStencilR, zr = DIM == 3 ? R : 0;
    const unsigned mask = __activemask();
    const int ncx = G.nc[0];
    const float ex = G.edgef[0], ey = G.edgef[1], ez = G.edgef[2];
    const float inv_ex = 1.f / ex;
    const float reach = 2.f * K.h_u;
    const float reach2 = reach * reach;
    const int sh = G.sub_shift;
    const int nsx = ncx << sh;
    const float inv_exs = inv_ex * (float)(1 << sh);
    const float four_h2 = K.four_h2_u;
    const uint32_t stride = (uint32_t)n * (uint32_t)sizeof(uint32_t);
    const float2 oxy = make_float2(oi[0], oi[1]);
    auto dist2 = [&](const float4& pj, int dx, float shy, float shz, bool real) {
        const float shx = -(float)dx * ex;
        const float2 rxy = __fadd2_rn(__ffma2_rn(make_float2(pj.x, pj.y), make_float2(-1.f, -1.f), oxy),
                                      make_float2(shx, shy));
        const float2 q = __fmul2_rn(rxy, rxy);
        float r2 = q.x + q.y;
        if (DIM == 3) {
            const float rz = (oi[2] - pj.z) + shz;
            r2 = fmaf(rz, rz, r2);
        }
        return real ? r2 : 1.0e30f;
    };
    // candidates jb .. je - 1 of one run; kr = cell index of the run's dx = 0
    // cell (the candidate's dx is its cell index minus kr)
    auto run = [&](int jb, int je, int kr, float shy, float shz, uint32_t code0) {
        for (int j = jb; j < je; j += 2) {
            const bool two = j + 1 < je;
            const float4 p0 = pos4c[j];
            const float4 p1 = pos4c[two ? j + 1 : j];
            const int d0 = __float_as_int(p0.w) - kr, d1 = __float_as_int(p1.w) - kr;
            const float r20 = dist2(p0, d0, shy, shz, true);
            const float r21 = dist2(p1, d1, shy, shz, two);
            const uint32_t jv = (uint32_t)j << kCodeBits;
            sigma.add(w_term_uniform(K, wnorm, r20));
            list_take(base_i, cnt, r20, four_h2, cap, jv + code0 + (uint32_t)d0, stride);
            sigma.add_if(w_term_uniform(K, wnorm, r21), two);
            list_take(base_i, cnt, r21, four_h2, cap, jv + (1u << kCodeBits) + code0 + (uint32_t)d1, stride);
        }
    };
    for (int dz = -zr; dz <= zr; ++dz) {
        const int cz = DIM == 3 ? cell_step(G, c[2], dz, 2) : 0;
        float rz = 0.f;
        if (DIM == 3) {
            rz = dz > 0 ? dz * ez - oi[2] : (dz < 0 ? oi[2] + (-dz - 1) * ez : 0.f);
            rz = fmaxf(rz - 1e-3f * ez, 0.f);
        }
        const float wz2 = reach2 - rz * rz;
        const bool zok = cz >= 0 && wz2 > 0.f;
        if (!__any_sync(mask, zok)) continue;
        const float shz = -(float)dz * ez;
        // per row: dyf = dy, shy = -dy ey (exact steps of ey) and the code of
        // the row's dx = -R cell advance with dy; the nearest y distance of the
        // row is the larger of dy ey - o_y (dy > 0) and o_y + (-dy - 1) ey
        // (dy < 0), the other being negative, and 0 for dy = 0
        float dyf = (float)(-R), shy = (float)R * ey;
        uint32_t code0 = (uint32_t)(R + kSide * kSide * (dz + R));
        for (int dy = -R; dy <= R; ++dy, dyf += 1.f, shy -= ey, code0 += kSide) {
            const int cy = cell_step(G, c[1], dy, 1);
            const float ry = fmaxf(fmaxf(fmaf(dyf, ey, -oi[1]), fmaf(-dyf - 1.f, ey, oi[1])) - 1e-3f * ey, 0.f);
            const float w2 = wz2 - ry * ry;
            const float w = sqrt_approx(fmaxf(w2, 0.f)) + 1e-3f * ex;
            const int slo = max(__float2int_rd((oi[0] - w) * inv_exs), -(R << sh));
            const int shi = min(__float2int_rd((oi[0] + w) * inv_exs), ((R + 1) << sh) - 1);
            const bool ok = zok && cy >= 0 && w2 > 0.f && slo <= shi;
            if (!__any_sync(mask, ok)) continue;
            const int row = ncx * (cy + G.nc[1] * cz);
            const int rb = row << sh;                            // first sort bin of the row
            // sub-cells a .. b along the row (may leave [0, nsx) on a periodic axis)
            const int a = (c[0] << sh) + slo, b = (c[0] << sh) + shi;
            if (INNER) {
                int jb = 0, je = 0;
                if (ok) {
                    jb = rstart[rb + a];
                    je = rstart[rb + b + 1];
                }
                run(jb, je, row + c[0], shy, shz, code0);
                continue;
            }
            // runs lo .. hi (sub-cells of the row) with their dx = 0 cell
            int lo0 = a, hi0 = b, kr0 = row + c[0], lo1 = 0, hi1 = -1, kr1 = row + c[0];
            if (!G.periodic[0]) {
                lo0 = max(a, 0);
                hi0 = min(b, nsx - 1);
            } else if (a < 0) {
                lo0 = nsx + a;
                hi0 = min(nsx - 1, nsx + b);
                kr0 = row + c[0] + ncx;
                hi1 = b;
            } else if (a >= nsx) {
                lo0 = a - nsx;
                hi0 = b - nsx;
                kr0 = row + c[0] - ncx;
            } else if (b >= nsx) {
                hi0 = nsx - 1;
                hi1 = b - nsx;
                kr1 = row + c[0] - ncx;
            }
            int jb0 = 0, je0 = 0, jb1 = 0, je1 = 0;
            if (ok && lo0 <= hi0) {
                jb0 = rstart[rb + lo0];
                je0 = rstart[rb + hi0 + 1];
            }
            if (ok && lo1 <= hi1) {
                jb1 = rstart[rb + lo1];
                je1 = rstart[rb + hi1 + 1];
            }
            run(jb0, je0, kr0, shy, shz, code0);
            run(jb1, je1, kr1, shy, shz, code0);
        }
    }
}

// ---------------------------------------------------------------- density
//
// sigma_i over all neighbours (self included); also writes the particle's
// force neighbour list (j != i, 0 < r^2 < 4 h_ij^2) transposed into nbl:
// entry k of particle i at nbl[k * n + i] = (j << 7) | code, and the count
// (which may exceed cap: the force kernel then scans the cells itself).

// Blocks of 512 threads (16 warps of neighbouring particles, whose walks
// share the candidates' cache lines in L1), two per SM, with the register
// budget of 1,024 threads per SM (at most 64 registers; 56 used, no spills).
// The compiler's own choice, 48 registers with spills, ran the 128^3 pass
// 7 % longer early in the run and 25 % longer after step 400.
constexpr int kDensityTPB32 = 512;
template <int DIM, typename Acc, bool UNIFORM>
__global__ void __launch_bounds__(kDensityTPB32, 2) k_density32(int n, const float4* __restrict__ pos4,
                                                      const int32_t* __restrict__ cell_of,
                                                      const int32_t* __restrict__ start, Grid G, Consts<float> K,
                                                      StateSet<float> S, float4* __restrict__ vr,
                                                      uint32_t* __restrict__ nbl, int32_t* __restrict__ nbc, int cap,
                                                      const float4* __restrict__ pos4c)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // every load of the particle's own data first: they are independent
    const int8_t kind = S.kind[i];
    const float4 pi = pos4[i];
    const int cell_i = cell_of[i];
    const float s0 = (float)S.s0[i];
    float vi[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int d = 0; d < DIM; ++d) vi[d] = S.v[(size_t)d * n + i];
    if (kind) {
        vr[i] = make_float4(vi[0], vi[1], vi[2], __int_as_float(0x7f800000));
        nbc[i] = 0;
        return;
    }
    const float oi[3] = {pi.x, pi.y, pi.z};
    const float hi = UNIFORM ? K.h_u : pi.w;
    Acc sigma;
    int cnt = 0;
    uint32_t* lp = nbl + i;
    const float wnorm = kernel_norm<DIM, float>() * pow_dim<DIM, float>(K.inv_h_u);
    auto visit = [&](int j, uint32_t code, const float4& pj, float r2, float, float, float) {
        if (UNIFORM) {
            sigma.add(w_term_uniform(K, wnorm, r2));
            // the list write as predicated stores and a selected pointer step:
            // no branch for the warp to diverge on
            const bool take = r2 < K.four_h2_u && r2 > 0.f;
            const bool store = take && cnt < cap;
            if (store) __stcs(lp, ((uint32_t)j << kCodeBits) | code);   // read once, by the force pass
            lp += store ? n : 0;
            cnt += take ? 1 : 0;
        } else if (r2 < support2<UNIFORM>(K, hi, pj.w)) {
            const float inv_h = 1.f / pair_h(K, hi, pj.w);
            sigma.add(wendland_W<DIM, float>(sqrt_approx(r2), inv_h));
            if (r2 > 0.f) {
                if (cnt < cap) {
                    *lp = ((uint32_t)j << kCodeBits) | code;
                    lp += n;
                }
                ++cnt;
            }
        }
    };
    // reach: the largest support radius 2 h_ij of any pair of i (h_j <= h_max)
    const float reach = UNIFORM ? 2.f * K.h_u : 2.f * pair_h(K, hi, K.h_u);
    // at uniform resolution the walk reads the copy of the offsets that
    // carries each candidate's cell index in w (one load per candidate
    // instead of two)
    if (UNIFORM) {
        // warps whose particles all sit R cells or more from the x ends of
        // the grid take the walk without the periodic split and the clip
        int c[3];
        cell_decode(G, cell_i, c);
        const bool inner = c[0] >= kStencilR && c[0] < G.nc[0] - kStencilR;
        const int32_t* rstart = G.sub_shift ? G.sub_start : start;
        if (__all_sync(__activemask(), inner))
            density_rows<DIM, Acc, true>(oi, c, G, K, wnorm, rstart, pos4c, sigma, cnt, nbl + i, n, cap);
        else
            density_rows<DIM, Acc, false>(oi, c, G, K, wnorm, rstart, pos4c, sigma, cnt, nbl + i, n, cap);
    } else {
        for_candidates_rows<DIM>(oi, reach, cell_i, G, start, cell_of, pos4, visit);
    }
    nbc[i] = cnt;
    // rho - rho0 = rho0 (sigma - sigma0) / sigma0; sigma - sigma0 is exact in FP32
    const float w = K.rho0 * (sigma.value() - s0) / s0;
    vr[i] = make_float4(vi[0], vi[1], vi[2], w);
}

// ------------------------------------------------- density on cell-blocked tiles
//
// The same density pass at uniform resolution, one thread block per block of
// B0 x B1 (x B2) home cells.  The block first stages the offsets of every
// particle in the home cells and the R = 2 cells around them (the halo,
// H = B + 2R cells per axis, periodic images resolved) into shared memory,
// in halo x-major order, with the halo x index of each particle's cell in w.
// Then each thread walks its home particle's clipped 5^D stencil row by row
// over that tile: each (dy, dz) row of the stencil is one contiguous run of
// the tile (no periodic split, no per-row global loads), and the x step of a
// candidate is the difference of the halo x indices.  The visit order is the
// row walk's (rows by (dz, dy), cells by dx, particles by index within a
// cell) and the arithmetic is the same, so sigma and the neighbour list are
// bit for bit those of k_density32.  A block whose halo holds more particles
// than the tile takes the row walk over global memory instead.

template <int DIM> struct TileShape;
template <> struct TileShape<3> { static constexpr int B0 = 4, B1 = 4, B2 = 4; };
template <> struct TileShape<2> { static constexpr int B0 = 8, B1 = 8, B2 = 1; };

template <int DIM> struct TileDims {
    using S = TileShape<DIM>;
    static constexpr int R = kStencilR;
    static constexpr int H0 = S::B0 + 2 * R, H1 = S::B1 + 2 * R, H2 = DIM == 3 ? S::B2 + 2 * R : 1;
    static constexpr int NHC = H0 * H1 * H2;        // halo cells
    static constexpr int NHR = H1 * H2;             // halo rows along x
    static constexpr int NHOME = S::B1 * S::B2;     // home rows along x
};

// Threads per block: the per-thread tile walk and the cooperative pass.
template <int DIM> struct TileThreads { static constexpr int WALK = DIM == 3 ? 160 : 128, COOP = 128; };

// Coordinate of halo cell v (relative to the grid origin) along axis d:
// wrapped on periodic axes, -1 outside a non-periodic axis.
__device__ __forceinline__ int halo_coord(const Grid& G, int v, int d)
{
    const int nc = G.nc[d];
    if (G.periodic[d]) return ((v % nc) + nc) % nc;
    return (v >= 0 && v < nc) ? v : -1;
}

// In-place exclusive scan of a[0, len) by the T threads of the block, total
// in a[len].  s_warp holds T/32 + 1 ints.
template <int T>
__device__ __forceinline__ void block_exclusive_scan(int* a, int len, int* s_warp)
{
    static_assert(T % 32 == 0, "whole warps");
    const int ipt = (len + T - 1) / T;
    const int b = threadIdx.x * ipt;
    int sum = 0;
    for (int k = 0; k < ipt; ++k)
        if (b + k < len) sum += a[b + k];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int k = 0; k < T / 32; ++k) {
            const int t = s_warp[k];
            s_warp[k] = acc;
            acc += t;
        }
        s_warp[T / 32] = acc;
    }
    __syncthreads();
    int run = s_warp[w] + x - sum;
    for (int k = 0; k < ipt; ++k)
        if (b + k < len) {
            const int t = a[b + k];
            a[b + k] = run;
            run += t;
        }
    if (threadIdx.x == 0) a[len] = s_warp[T / 32];
    __syncthreads();
}

// Bytes of dynamic shared memory of a tile kernel for a tile of cap particles
// (plus extra bytes of per-block tables).
template <int DIM>
__host__ __device__ constexpr size_t tile_smem_bytes(int cap, size_t extra = 0)
{
    return (size_t)cap * (sizeof(float4) + sizeof(int)) + (size_t)(2 * TileDims<DIM>::NHC + 1) * sizeof(int) + extra;
}

// Shared-memory view of a staged block: the tile and its cell tables.
struct TileView {
    float4* pos;     // [cap] offsets, w = halo x index of the particle's cell
    int* gid;        // [cap] global particle index
    int* ts;         // [NHC + 1] tile start of each halo cell
    int* gs;         // [NHC] global start of each halo cell
    int* home;       // [NHOME + 1] prefix counts of the home particles by home row
    int bxn, byn, bzn;   // home cells of the block along each axis (edge blocks are partial)
    bool fits;       // the halo's particles fit the tile (else only the tables are set)
};

// Stage block b: counts and global starts of the halo cells, their scan, the
// particles' offsets (when they fit), and the home-row prefix counts.  Every
// thread of the block calls it; it ends with a barrier.
template <int DIM, int T>
__device__ __forceinline__ void stage_tile(TileView& V, const Grid& G, const int32_t* __restrict__ start,
                                           const float4* __restrict__ pos4c, int nb0, int nb1, int tile_cap,
                                           int* s_warp)
{
    using TD = TileDims<DIM>;
    using SH = TileShape<DIM>;
    constexpr int R = TD::R, H0 = TD::H0, H1 = TD::H1, NHC = TD::NHC;
    constexpr int Rz = DIM == 3 ? R : 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = blockIdx.x;
    const int bx = b % nb0, by = (b / nb0) % nb1, bz = b / (nb0 * nb1);
    const int cx0 = bx * SH::B0, cy0 = by * SH::B1, cz0 = bz * SH::B2;
    V.bxn = min(SH::B0, G.nc[0] - cx0);
    V.byn = min(SH::B1, G.nc[1] - cy0);
    V.bzn = DIM == 3 ? min(SH::B2, G.nc[2] - cz0) : 1;
    for (int c = tid; c < NHC; c += T) {
        const int hx = c % H0, hy = (c / H0) % H1, hz = c / (H0 * H1);
        const int gx = halo_coord(G, cx0 + hx - R, 0), gy = halo_coord(G, cy0 + hy - R, 1);
        const int gz = DIM == 3 ? halo_coord(G, cz0 + hz - R, 2) : 0;
        int cnt = 0, gs = 0;
        if (gx >= 0 && gy >= 0 && gz >= 0) {
            const int g = gx + G.nc[0] * (gy + G.nc[1] * gz);
            gs = start[g];
            cnt = start[g + 1] - gs;
        }
        V.gs[c] = gs;
        V.ts[c] = cnt;
    }
    __syncthreads();
    block_exclusive_scan<T>(V.ts, NHC, s_warp);
    V.fits = V.ts[NHC] <= tile_cap;
    // one warp per halo row: the particles of a row are one or two
    // contiguous runs of the cell-sorted offsets
    if (V.fits) {
        for (int r = warp; r < TD::NHR; r += T / 32) {
            const int c0 = r * H0;
            const int t1 = V.ts[c0 + H0];
            for (int t = V.ts[c0] + lane; t < t1; t += 32) {
                int lo = 0, hi = H0 - 1;           // the cell of t: last k with ts[c0 + k] <= t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (V.ts[c0 + mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
                const int c = c0 + lo;
                const int g = V.gs[c] + (t - V.ts[c]);
                float4 p = pos4c[g];
                p.w = __int_as_float(lo);
                V.pos[t] = p;
                V.gid[t] = g;
            }
        }
    }
    if (tid == 0) {
        int acc = 0;
        for (int k = 0; k < V.byn * V.bzn; ++k) {
            const int hy = R + k % V.byn, hz = Rz + k / V.byn;
            const int c = (hy + H1 * hz) * H0 + R;
            V.home[k] = acc;
            acc += V.ts[c + V.bxn] - V.ts[c];
        }
        V.home[V.byn * V.bzn] = acc;
    }
    __syncthreads();
}

// Home particle t of a staged block: its home row's halo coordinates, its
// tile index (valid when the tile fits) and its global index (home rows are
// runs of real cells, contiguous in the global order).
template <int DIM>
__device__ __forceinline__ void home_particle(const TileView& V, int t, int& hy, int& hz, int& s, int& g)
{
    using TD = TileDims<DIM>;
    constexpr int R = TD::R, H0 = TD::H0, H1 = TD::H1;
    int k = 0;
    while (V.home[k + 1] <= t) ++k;
    hy = R + k % V.byn;
    hz = (DIM == 3 ? R : 0) + k / V.byn;
    const int c_row = (hy + H1 * hz) * H0 + R;
    s = V.ts[c_row] + (t - V.home[k]);
    g = V.gs[c_row] + (t - V.home[k]);
}

// The clipped x extent [dxlo, dxhi] of stencil row (dy, dz) for a particle
// at cell-relative offset oi (the row walk's clipping: margins of 1e-3 of a
// cell edge); false if the row is out of reach.
template <int DIM>
__device__ __forceinline__ bool row_extent(const float* oi, int dy, int dz, float reach2, float ex, float ey, float ez,
                                           float inv_ex, int& dxlo, int& dxhi)
{
    constexpr int R = kStencilR;
    float rz = 0.f;
    if (DIM == 3) {
        rz = dz > 0 ? dz * ez - oi[2] : (dz < 0 ? oi[2] + (-dz - 1) * ez : 0.f);
        rz = fmaxf(rz - 1e-3f * ez, 0.f);
    }
    const float wz2 = reach2 - rz * rz;
    if (wz2 <= 0.f) return false;
    float ry = dy > 0 ? dy * ey - oi[1] : (dy < 0 ? oi[1] + (-dy - 1) * ey : 0.f);
    ry = fmaxf(ry - 1e-3f * ey, 0.f);
    const float w2 = wz2 - ry * ry;
    if (w2 <= 0.f) return false;
    const float w = sqrt_approx(w2) + 1e-3f * ex;
    dxlo = max(__float2int_rd((oi[0] - w) * inv_ex), -R);
    dxhi = min(__float2int_rd((oi[0] + w) * inv_ex), R);
    return dxlo <= dxhi;
}

// r^2 of a candidate from the tile, in the row walk's arithmetic (so the
// accept decisions, and the neighbour list, are those of the row walk).
template <int DIM>
__device__ __forceinline__ float tile_r2(const float* oi, int hx_i, const float4& pj, float ex, float shy, float shz)
{
    const float shx = -(float)(__float_as_int(pj.w) - hx_i) * ex;
    const float2 rxy = __fadd2_rn(__ffma2_rn(make_float2(pj.x, pj.y), make_float2(-1.f, -1.f),
                                             make_float2(oi[0], oi[1])),
                                  make_float2(shx, shy));
    const float2 q = __fmul2_rn(rxy, rxy);
    float r2 = q.x + q.y;
    if (DIM == 3) {
        const float rz_ = (oi[2] - pj.z) + shz;
        r2 = fmaf(rz_, rz_, r2);
    }
    return r2;
}

template <int DIM, typename Acc>
__global__ void __launch_bounds__(TileThreads<DIM>::WALK) k_density32_tile(
    int n, const float4* __restrict__ pos4c, const int32_t* __restrict__ cell_of, const int32_t* __restrict__ start,
    Grid G, Consts<float> K, StateSet<float> S, float4* __restrict__ vr, uint32_t* __restrict__ nbl,
    int32_t* __restrict__ nbc, int cap, int nb0, int nb1, int tile_cap)
{
    using TD = TileDims<DIM>;
    constexpr int T = TileThreads<DIM>::WALK, R = TD::R, H0 = TD::H0, H1 = TD::H1, NHC = TD::NHC;
    constexpr int Rz = DIM == 3 ? R : 0;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_warp[T / 32 + 1];
    __shared__ int s_home[TD::NHOME + 1];
    TileView V;
    V.pos = (float4*)smem;
    V.gid = (int*)(V.pos + tile_cap);
    V.ts = V.gid + tile_cap;
    V.gs = V.ts + NHC + 1;
    V.home = s_home;
    stage_tile<DIM, T>(V, G, start, pos4c, nb0, nb1, tile_cap, s_warp);
    const int nhome = V.home[V.byn * V.bzn];

    const float ex = G.edgef[0], ey = G.edgef[1], ez = G.edgef[2];
    const float inv_ex = 1.f / ex;
    const float reach = 2.f * K.h_u;
    const float reach2 = reach * reach;
    const float wnorm = kernel_norm<DIM, float>() * pow_dim<DIM, float>(K.inv_h_u);
    for (int t = threadIdx.x; t < nhome; t += T) {
        int hy_i, hz_i, s, i;
        home_particle<DIM>(V, t, hy_i, hz_i, s, i);
        const int8_t kind = S.kind[i];
        const float s0 = (float)S.s0[i];
        float vi[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int d = 0; d < DIM; ++d) vi[d] = S.v[(size_t)d * n + i];
        if (kind) {
            vr[i] = make_float4(vi[0], vi[1], vi[2], __int_as_float(0x7f800000));
            nbc[i] = 0;
            continue;
        }
        Acc sigma;
        int cnt = 0;
        uint32_t* lp = nbl + i;
        // every candidate adds its term (0 outside the support) as in the row
        // walk, so the compensated sums, too, are those of the row walk
        auto candidate = [&](float r2, uint32_t entry) {
            sigma.add(w_term_uniform(K, wnorm, r2));
            if (r2 < K.four_h2_u && r2 > 0.f) {
                if (cnt < cap) {
                    *lp = entry;
                    lp += n;
                }
                ++cnt;
            }
        };
        if (V.fits) {
            const float4 pi = V.pos[s];
            const float oi[3] = {pi.x, pi.y, pi.z};
            const int hx_i = __float_as_int(pi.w);
            for (int dz = -Rz; dz <= Rz; ++dz) {
                const float shz = -(float)dz * ez;
                for (int dy = -R; dy <= R; ++dy) {
                    int dxlo, dxhi;
                    if (!row_extent<DIM>(oi, dy, dz, reach2, ex, ey, ez, inv_ex, dxlo, dxhi)) continue;
                    const float shy = -(float)dy * ey;
                    const int rowc = (hy_i + dy + H1 * (hz_i + dz)) * H0 + hx_i;
                    const int tend = V.ts[rowc + dxhi + 1];
                    const uint32_t code_row =
                        (uint32_t)(R + kSide * (dy + R) + kSide * kSide * (dz + R)) - (uint32_t)hx_i;
                    auto one = [&](int tj, const float4& pj) {
                        const float r2 = tile_r2<DIM>(oi, hx_i, pj, ex, shy, shz);
                        candidate(r2, ((uint32_t)V.gid[tj] << kCodeBits) | (code_row + (uint32_t)__float_as_int(pj.w)));
                    };
                    int tj = V.ts[rowc + dxlo];
                    for (; tj + 1 < tend; tj += 2) {
                        const float4 p0 = V.pos[tj], p1 = V.pos[tj + 1];
                        one(tj, p0);
                        one(tj + 1, p1);
                    }
                    if (tj < tend) one(tj, V.pos[tj]);
                }
            }
        } else {
            // the halo does not fit the tile: the row walk over global memory
            const float4 pi = pos4c[i];
            const float oi[3] = {pi.x, pi.y, pi.z};
            auto visit = [&](int j, uint32_t code, const float4&, float r2, float, float, float) {
                candidate(r2, ((uint32_t)j << kCodeBits) | code);
            };
            for_candidates_rows<DIM, true, true>(oi, reach, cell_of[i], G, start, cell_of, pos4c, visit);
        }
        nbc[i] = cnt;
        const float w = K.rho0 * (sigma.value() - s0) / s0;
        vr[i] = make_float4(vi[0], vi[1], vi[2], w);
    }
}

// ------------------------------------ density on tiles, flattened row walk
//
// The tile walk with the rows of a particle's stencil walked as one sequence
// per lane: each lane first lists its particle's clipped row runs (tile
// start and length per stencil row, in shared memory, row-major so that the
// lanes of a warp read distinct banks), then steps through them two
// candidates at a time, moving to its next non-empty row when a run ends,
// while the other lanes of the warp are still inside theirs.  The warp then
// runs as many iterations as its longest particle has candidates, not the
// sum over rows of each row's longest run.  Same candidates, order and
// arithmetic as the row walk: the same sums and lists bit for bit.

constexpr int kFlatThreads3 = 160, kFlatThreads2 = 128;
template <int DIM> struct FlatShape {
    static constexpr int T = DIM == 3 ? kFlatThreads3 : kFlatThreads2;
    static constexpr int NR = DIM == 3 ? kSide * kSide : kSide;    // stencil rows
};

template <int DIM>
__host__ __device__ constexpr size_t flat_table_bytes()
{
    return (size_t)FlatShape<DIM>::NR * FlatShape<DIM>::T * sizeof(uint32_t);
}

template <int DIM, typename Acc>
__global__ void __launch_bounds__(FlatShape<DIM>::T) k_density32_flat(
    int n, const float4* __restrict__ pos4c, const int32_t* __restrict__ cell_of, const int32_t* __restrict__ start,
    Grid G, Consts<float> K, StateSet<float> S, float4* __restrict__ vr, uint32_t* __restrict__ nbl,
    int32_t* __restrict__ nbc, int cap, int nb0, int nb1, int tile_cap)
{
    using TD = TileDims<DIM>;
    constexpr int T = FlatShape<DIM>::T, NR = FlatShape<DIM>::NR, R = TD::R, H0 = TD::H0, H1 = TD::H1, NHC = TD::NHC;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_warp[T / 32 + 1];
    __shared__ int s_home[TD::NHOME + 1];
    __shared__ float4 s_rowc[NR];            // per stencil row: shy, shz, code of (dy, dz) with dx = -R, -
    uint32_t* runs = (uint32_t*)smem;        // [NR][T]: tile start | run length << 16
    TileView V;
    V.pos = (float4*)(smem + flat_table_bytes<DIM>());
    V.gid = (int*)(V.pos + tile_cap);
    V.ts = V.gid + tile_cap;
    V.gs = V.ts + NHC + 1;
    V.home = s_home;
    const float ex = G.edgef[0], ey = G.edgef[1], ez = G.edgef[2];
    for (int r = threadIdx.x; r < NR; r += T) {
        const int dy = r % kSide - R, dz = DIM == 3 ? r / kSide - R : 0;
        s_rowc[r] = make_float4(-(float)dy * ey, -(float)dz * ez,
                                __int_as_float(R + kSide * (dy + R) + kSide * kSide * (dz + R)), 0.f);
    }
    stage_tile<DIM, T>(V, G, start, pos4c, nb0, nb1, tile_cap, s_warp);
    const int nhome = V.home[V.byn * V.bzn];

    const float inv_ex = 1.f / ex;
    const float reach = 2.f * K.h_u;
    const float reach2 = reach * reach;
    const float wnorm = kernel_norm<DIM, float>() * pow_dim<DIM, float>(K.inv_h_u);
    for (int t = threadIdx.x; t < nhome; t += T) {
        int hy_i, hz_i, s, i;
        home_particle<DIM>(V, t, hy_i, hz_i, s, i);
        const int8_t kind = S.kind[i];
        const float s0 = (float)S.s0[i];
        float vi[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int d = 0; d < DIM; ++d) vi[d] = S.v[(size_t)d * n + i];
        if (kind) {
            vr[i] = make_float4(vi[0], vi[1], vi[2], __int_as_float(0x7f800000));
            nbc[i] = 0;
            continue;
        }
        Acc sigma;
        int cnt = 0;
        uint32_t* lp = nbl + i;
        auto candidate = [&](float r2, uint32_t entry) {
            sigma.add(w_term_uniform(K, wnorm, r2));
            const bool take = r2 < K.four_h2_u && r2 > 0.f;
            const bool store = take && cnt < cap;
            if (store) *lp = entry;
            lp += store ? n : 0;
            cnt += take ? 1 : 0;
        };
        if (V.fits) {
            const float4 pi = V.pos[s];
            const float oi[3] = {pi.x, pi.y, pi.z};
            const int hx_i = __float_as_int(pi.w);
            // this lane's row runs: tile start and length of each stencil row
            for (int r = 0; r < NR; ++r) {
                const int dy = r % kSide - R, dz = DIM == 3 ? r / kSide - R : 0;
                int dxlo, dxhi;
                uint32_t run = 0;
                if (row_extent<DIM>(oi, dy, dz, reach2, ex, ey, ez, inv_ex, dxlo, dxhi)) {
                    const int rowc = (hy_i + dy + H1 * (hz_i + dz)) * H0 + hx_i;
                    const int t0 = V.ts[rowc + dxlo];
                    run = (uint32_t)t0 | ((uint32_t)(V.ts[rowc + dxhi + 1] - t0) << 16);
                }
                runs[r * T + threadIdx.x] = run;
            }
            // the flattened walk: (row, position, end) of this lane
            int r = -1, tj = 0, tend = 0;
            float shy = 0.f, shz = 0.f;
            uint32_t code_row = 0;
            auto next_row = [&]() {
                while (tj >= tend && ++r < NR) {
                    const uint32_t run = runs[r * T + threadIdx.x];
                    tj = (int)(run & 0xffffu);
                    tend = tj + (int)(run >> 16);
                }
                if (r < NR) {
                    const float4 rc = s_rowc[r];
                    shy = rc.x;
                    shz = rc.y;
                    code_row = (uint32_t)__float_as_int(rc.z) - (uint32_t)hx_i;
                }
            };
            next_row();
            auto one = [&](int tq, const float4& pj) {
                const float r2 = tile_r2<DIM>(oi, hx_i, pj, ex, shy, shz);
                candidate(r2, ((uint32_t)V.gid[tq] << kCodeBits) | (code_row + (uint32_t)__float_as_int(pj.w)));
            };
            while (r < NR) {
                if (tj + 1 < tend) {
                    const float4 p0 = V.pos[tj], p1 = V.pos[tj + 1];
                    one(tj, p0);
                    one(tj + 1, p1);
                    tj += 2;
                } else {
                    one(tj, V.pos[tj]);
                    tj += 1;
                }
                if (tj >= tend) next_row();
            }
        } else {
            // the halo does not fit the tile: the row walk over global memory
            const float4 pi = pos4c[i];
            const float oi[3] = {pi.x, pi.y, pi.z};
            auto visit = [&](int j, uint32_t code, const float4&, float r2, float, float, float) {
                candidate(r2, ((uint32_t)j << kCodeBits) | code);
            };
            for_candidates_rows<DIM, true, true>(oi, reach, cell_of[i], G, start, cell_of, pos4c, visit);
        }
        nbc[i] = cnt;
        const float w = K.rho0 * (sigma.value() - s0) / s0;
        vr[i] = make_float4(vi[0], vi[1], vi[2], w);
    }
}

// ---------------------------------- density on tiles, lanes sharing a particle
//
// The same staged tile, walked cooperatively: a group of G lanes (8 in 3-D,
// 4 in 2-D) takes one home particle and splits its candidates, G at a time,
// in the row walk's order (stencil rows by (dz, dy), then the tile order of
// each row's clipped run).  Every lane of a warp tests a candidate in every
// iteration, whatever the lengths of the particle's row runs, so the walk
// does not lose lanes to the unequal runs of a disordered lattice.  Each
// lane keeps a compensated partial sum of sigma; the group combines them
// exactly pairwise (TwoSum) at the end.  Accepted neighbours go to the list
// in candidate order (ballot + prefix within the group), so the list and the
// count are those of the row walk; sigma differs from it only by the
// summation order.  The group's row table (exclusive prefix of the run
// lengths, tile start minus prefix, stencil code and shifts) lives in shared
// memory; a lane moves from row to row as its candidate index passes the
// prefixes.

template <int DIM> struct CoopShape {
    static constexpr int G = DIM == 3 ? 8 : 4;                 // lanes per particle
    static constexpr int NR = DIM == 3 ? kSide * kSide : kSide;  // stencil rows
    static constexpr int RPL = (NR + G - 1) / G;               // rows set up per lane
    static constexpr int NG = TileThreads<DIM>::COOP / G;      // groups per block
};

struct CoopRow {
    int base;        // tile start of the row's run minus the row's prefix: t = f + base
    uint32_t code;   // stencil code of the row minus hx_i: code = code + hx_j
    float shy, shz;  // FP32 shifts of the row
};

template <int DIM>
__host__ __device__ constexpr size_t coop_table_bytes()
{
    using C = CoopShape<DIM>;
    return (size_t)C::NG * (C::NR * sizeof(CoopRow) + (C::NR + 1) * sizeof(int));
}

// Compensated partial sums combined exactly: (s, c) holds s - c.
__device__ __forceinline__ void ksum_merge(float& s, float& c, float s2, float c2)
{
    const float t = __fadd_rn(s, s2);
    const float bb = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(s2, bb));   // s + s2 = t + e exactly
    c = __fsub_rn(__fadd_rn(c, c2), e);
    s = t;
}

template <typename Acc> struct PartialSum;
template <> struct PartialSum<KSum> {
    static __device__ __forceinline__ void get(const KSum& a, float& s, float& c) { s = a.s; c = a.c; }
    static constexpr bool compensated = true;
};
template <> struct PartialSum<PlainF> {
    static __device__ __forceinline__ void get(const PlainF& a, float& s, float& c) { s = a.s; c = 0.f; }
    static constexpr bool compensated = false;
};

template <int DIM, typename Acc>
__global__ void __launch_bounds__(TileThreads<DIM>::COOP, 4) k_density32_coop(
    int n, const float4* __restrict__ pos4c, const int32_t* __restrict__ cell_of, const int32_t* __restrict__ start,
    Grid G, Consts<float> K, StateSet<float> S, float4* __restrict__ vr, uint32_t* __restrict__ nbl,
    int32_t* __restrict__ nbc, int cap, int nb0, int nb1, int tile_cap)
{
    using TD = TileDims<DIM>;
    using C = CoopShape<DIM>;
    constexpr int T = TileThreads<DIM>::COOP, R = TD::R, H0 = TD::H0, H1 = TD::H1, NHC = TD::NHC;
    constexpr int GL = C::G, NR = C::NR, RPL = C::RPL, NG = C::NG;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_warp[T / 32 + 1];
    __shared__ int s_home[TD::NHOME + 1];
    TileView V;
    CoopRow* rows_all = (CoopRow*)smem;                              // [NG][NR]
    int* pref_all = (int*)(rows_all + NG * NR);                      // [NG][NR + 1]
    V.pos = (float4*)(smem + coop_table_bytes<DIM>());
    V.gid = (int*)(V.pos + tile_cap);
    V.ts = V.gid + tile_cap;
    V.gs = V.ts + NHC + 1;
    V.home = s_home;
    stage_tile<DIM, T>(V, G, start, pos4c, nb0, nb1, tile_cap, s_warp);
    const int nhome = V.home[V.byn * V.bzn];

    const float ex = G.edgef[0], ey = G.edgef[1], ez = G.edgef[2];
    const float inv_ex = 1.f / ex;
    const float reach = 2.f * K.h_u;
    const float reach2 = reach * reach;
    const float wnorm = kernel_norm<DIM, float>() * pow_dim<DIM, float>(K.inv_h_u);
    const int lane = threadIdx.x & 31, q = lane % GL;
    const int grp = threadIdx.x / GL;                   // group within the block
    const unsigned gshift = (unsigned)((lane / GL) * GL);
    const unsigned gmask = (GL == 32 ? 0xffffffffu : ((1u << GL) - 1u)) << gshift;
    CoopRow* rows = rows_all + grp * NR;
    int* pref = pref_all + grp * (NR + 1);

    if (!V.fits) {
        // the halo does not fit the tile: the row walk over global memory,
        // one thread per particle
        for (int t = threadIdx.x; t < nhome; t += T) {
            int hy_i, hz_i, s, i;
            home_particle<DIM>(V, t, hy_i, hz_i, s, i);
            const int8_t kind = S.kind[i];
            const float s0 = (float)S.s0[i];
            float vi[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int d = 0; d < DIM; ++d) vi[d] = S.v[(size_t)d * n + i];
            if (kind) {
                vr[i] = make_float4(vi[0], vi[1], vi[2], __int_as_float(0x7f800000));
                nbc[i] = 0;
                continue;
            }
            Acc sigma;
            int cnt = 0;
            uint32_t* lp = nbl + i;
            const float4 pi = pos4c[i];
            const float oi[3] = {pi.x, pi.y, pi.z};
            auto visit = [&](int j, uint32_t code, const float4&, float r2, float, float, float) {
                sigma.add(w_term_uniform(K, wnorm, r2));
                if (r2 < K.four_h2_u && r2 > 0.f) {
                    if (cnt < cap) {
                        *lp = ((uint32_t)j << kCodeBits) | code;
                        lp += n;
                    }
                    ++cnt;
                }
            };
            for_candidates_rows<DIM, true, true>(oi, reach, cell_of[i], G, start, cell_of, pos4c, visit);
            nbc[i] = cnt;
            vr[i] = make_float4(vi[0], vi[1], vi[2], K.rho0 * (sigma.value() - s0) / s0);
        }
        return;
    }

    // rounds of NG particles, one per group; every lane of the block runs the
    // same number of rounds (the warp-wide votes below need whole warps)
    const int rounds = (nhome + NG - 1) / NG;
    for (int round = 0; round < rounds; ++round) {
        const int t = round * NG + grp;
        int i = 0, total = 0;
        float oi[3] = {0.f, 0.f, 0.f};
        int hx_i = 0;
        float s0 = 1.f, vi[3] = {0.f, 0.f, 0.f};
        bool active = false;
        if (t < nhome) {
            int hy_i, hz_i, s;
            home_particle<DIM>(V, t, hy_i, hz_i, s, i);
            const float4 pi = V.pos[s];
            oi[0] = pi.x;
            oi[1] = pi.y;
            oi[2] = pi.z;
            hx_i = __float_as_int(pi.w);
            const int8_t kind = S.kind[i];
            s0 = (float)S.s0[i];
#pragma unroll
            for (int d = 0; d < DIM; ++d) vi[d] = S.v[(size_t)d * n + i];
            if (kind) {
                if (q == 0) {
                    vr[i] = make_float4(vi[0], vi[1], vi[2], __int_as_float(0x7f800000));
                    nbc[i] = 0;
                }
            } else {
                active = true;
                // this lane's stencil rows (RPL consecutive ones): their runs
                // go to the group's table first (tile start, length), then
                // get their prefixes
                int mine = 0;
#pragma unroll
                for (int k = 0; k < RPL; ++k) {
                    const int r = q * RPL + k;
                    if (r < NR) {
                        const int dy = r % kSide - R, dz = DIM == 3 ? r / kSide - R : 0;
                        int dxlo, dxhi, t0 = 0, l = 0;
                        if (row_extent<DIM>(oi, dy, dz, reach2, ex, ey, ez, inv_ex, dxlo, dxhi)) {
                            const int rowc = (hy_i + dy + H1 * (hz_i + dz)) * H0 + hx_i;
                            t0 = V.ts[rowc + dxlo];
                            l = V.ts[rowc + dxhi + 1] - t0;
                        }
                        rows[r].base = t0;
                        pref[r] = l;
                        mine += l;
                    }
                }
                // exclusive prefix of the rows over the group's lanes
                int incl = mine;
#pragma unroll
                for (int o = 1; o < GL; o <<= 1) {
                    const int y = __shfl_up_sync(gmask, incl, o, GL);
                    if (q >= o) incl += y;
                }
                int run = incl - mine;
#pragma unroll
                for (int k = 0; k < RPL; ++k) {
                    const int r = q * RPL + k;
                    if (r < NR) {
                        const int dy = r % kSide - R, dz = DIM == 3 ? r / kSide - R : 0;
                        const int l = pref[r];
                        pref[r] = run;
                        CoopRow rr;
                        rr.base = rows[r].base - run;
                        rr.code = (uint32_t)(R + kSide * (dy + R) + kSide * kSide * (dz + R)) - (uint32_t)hx_i;
                        rr.shy = -(float)dy * ey;
                        rr.shz = -(float)dz * ez;
                        rows[r] = rr;
                        run += l;
                    }
                }
                total = __shfl_sync(gmask, incl, GL - 1, GL);
                if (q == 0) pref[NR] = total;
            }
        }
        __syncwarp();
        Acc sigma;
        int cnt = 0;
        int r = 0;
        // candidate f = f0 + q of the group's particle, G at a time, until
        // every group of the warp is through its candidates
        for (int f0 = 0; __any_sync(0xffffffffu, active && f0 < total); f0 += GL) {
            const int f = f0 + q;
            bool take = false;
            float r2 = 0.f;
            uint32_t entry = 0;
            if (active && f < total) {
                while (f >= pref[r + 1]) ++r;
                const CoopRow rr = rows[r];
                const int tj = f + rr.base;
                const float4 pj = V.pos[tj];
                r2 = tile_r2<DIM>(oi, hx_i, pj, ex, rr.shy, rr.shz);
                sigma.add(w_term_uniform(K, wnorm, r2));
                if (r2 < K.four_h2_u) {
                    take = r2 > 0.f;
                    entry = ((uint32_t)V.gid[tj] << kCodeBits) | (rr.code + (uint32_t)__float_as_int(pj.w));
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, take) & gmask;
            if (take) {
                const int pos = cnt + __popc(m & ((1u << lane) - 1u));
                if (pos < cap) nbl[(size_t)pos * n + i] = entry;
            }
            cnt += __popc(m);
        }
        // combine the lanes' partial sums within the group
        float ps, pc;
        PartialSum<Acc>::get(sigma, ps, pc);
#pragma unroll
        for (int o = GL / 2; o >= 1; o >>= 1) {
            const float s2 = __shfl_xor_sync(0xffffffffu, ps, o, GL);
            const float c2 = __shfl_xor_sync(0xffffffffu, pc, o, GL);
            if (PartialSum<Acc>::compensated) ksum_merge(ps, pc, s2, c2);
            else ps += s2;
        }
        if (active && q == 0) {
            const float sig = PartialSum<Acc>::compensated ? __fsub_rn(ps, pc) : ps;
            nbc[i] = cnt;
            vr[i] = make_float4(vi[0], vi[1], vi[2], K.rho0 * (sig - s0) / s0);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ forces

// Register budget at uniform resolution: six blocks of 128 threads per SM
// (at most 85 registers; 80 used, no spills), for the three pairs of neighbour
// data in flight ahead of the three being computed.  The pass waits on these
// gathers (L1/L2 hits): with eight blocks and one pair of data ahead it ran
// 12 % longer early in a 128^3 run and 11 % longer after step 400; with three
// pairs per iteration at seven or eight blocks the registers spill (+35-75 %).
// Variable resolution keeps eight blocks (64 registers) and one pair ahead:
// at six blocks its pass ran 10 % longer.
template <int DIM, typename Acc, bool UNIFORM>
__global__ void __launch_bounds__(kTPB32, UNIFORM ? 6 : 8) k_forces32(int n, const float4* __restrict__ pos4,
                                                     const int32_t* __restrict__ cell_of,
                                                     const int32_t* __restrict__ start, Grid G, Consts<float> K,
                                                     StateSet<float> S, const float* __restrict__ mf,
                                                     const float4* __restrict__ vr, const uint32_t* __restrict__ nbl,
                                                     const int32_t* __restrict__ nbc, int cap,
                                                     const double* __restrict__ dt_ptr, int kick_on, int write_ad,
                                                     float* __restrict__ Rout, float* __restrict__ chi_out,
                                                     double* __restrict__ partials)
{
    __shared__ float4 tab[kCodes];
    for (int t = threadIdx.x; t < kCodes; t += blockDim.x) {
        float sh[3];
        code_shift(G, (uint32_t)t, sh);
        tab[t] = make_float4(sh[0], sh[1], sh[2], 0.f);
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double part[kNPart];
#pragma unroll
    for (int k = 0; k < kNPart; ++k) part[k] = 0.0;
    const double dt = *dt_ptr;
    const double hdt = kick_on ? 0.5 * dt : 0.0;
    if (i < n && S.kind[i] == 0) {
        const float4 pi = pos4[i];
        const float oi[3] = {pi.x, pi.y, pi.z};
        const float hi = UNIFORM ? K.h_u : pi.w;
        const float4 me = vr[i];
        const float vi[3] = {me.x, me.y, me.z};
        const float rho_i = K.rho0 + me.w;
        const float p_i = K.c2 * me.w;
        const float inv_rho_i = rcp_approx(rho_i);
        PairSums<DIM, Acc> sums;
        // W'/r = coef t^3, coef = -5 a_D h^-(D+2) (uniform h: one constant)
        const float norm = kernel_norm<DIM, float>();
        auto pair = [&](int j, const float4& pj, const float4& oj, const float* rv, float r2) {
            const float inv_r = rsqrtf(r2);
            const float r = r2 * inv_r;
            float inv_h, m_j;
            if (UNIFORM) {
                inv_h = K.inv_h_u;
                m_j = pj.w;
            } else {
                inv_h = __frcp_rn(pair_h(K, hi, pj.w));
                m_j = mf[j];
            }
            const float coef = UNIFORM ? K.dwr_coef_u : -5.f * norm * pow_dim<DIM, float>(inv_h) * inv_h * inv_h;
            const float dwr = dwr_of<DIM>(r, inv_h, coef);
            pair_force32<DIM, Acc>(K, rv, inv_r, dwr, vi, rho_i, inv_rho_i, p_i, oj, m_j, sums);
        };
        const int cnt = nbc[i];
        if (cnt <= cap) {
            // the neighbour list of the density pass: no candidate tests.
            // Software pipeline: the list entries six ahead and the
            // neighbour data three ahead are in flight while a pair is computed.
            const uint32_t* lp = nbl + i;
            auto one = [&](uint32_t ec, const float4& pj, const float4& oj) {
                const float4 sh = tab[ec & ((1u << kCodeBits) - 1u)];
                float rv[3];
                rv[0] = (oi[0] - pj.x) + sh.x;
                rv[1] = (oi[1] - pj.y) + sh.y;
                float r2 = rv[0] * rv[0] + rv[1] * rv[1];
                rv[2] = 0.f;
                if (DIM == 3) {
                    rv[2] = (oi[2] - pj.z) + sh.z;
                    r2 += rv[2] * rv[2];
                }
                pair((int)(ec >> kCodeBits), pj, oj, rv, r2);
            };
            // uniform resolution: three pairs per iteration, the next
            // iteration's three pairs of neighbour data and the entries of the
            // one after in flight (the entries read once, as streaming loads,
            // through a pointer that advances by three list rows per
            // iteration); the pairs in list order, so the sums are those of a
            // pair-by-pair walk
            if constexpr (UNIFORM) {
                uint32_t e[6];
#pragma unroll
                for (int t = 0; t < 6; ++t) e[t] = cnt > t ? __ldcs(lp + (size_t)t * n) : 0u;
                float4 pc[3], oc[3];
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    pc[t] = pos4[e[t] >> kCodeBits];
                    oc[t] = vr[e[t] >> kCodeBits];
                }
                int k = 0;
                const uint32_t* lq = lp + 6 * (size_t)n;
                const size_t n3 = 3 * (size_t)n;
                for (; k + 2 < cnt; k += 3, lq += n3) {
                    float4 pn[3], on[3];
#pragma unroll
                    for (int t = 0; t < 3; ++t) {
                        pn[t] = pos4[e[3 + t] >> kCodeBits];
                        on[t] = vr[e[3 + t] >> kCodeBits];
                    }
                    uint32_t en[3];
#pragma unroll
                    for (int t = 0; t < 3; ++t) en[t] = k + 6 + t < cnt ? __ldcs(lq + (size_t)t * n) : 0u;
#pragma unroll
                    for (int t = 0; t < 3; ++t) one(e[t], pc[t], oc[t]);
#pragma unroll
                    for (int t = 0; t < 3; ++t) {
                        pc[t] = pn[t];
                        oc[t] = on[t];
                        e[t] = e[3 + t];
                        e[3 + t] = en[t];
                    }
                }
                if (k < cnt) one(e[0], pc[0], oc[0]);
                if (k + 1 < cnt) one(e[1], pc[1], oc[1]);
            } else {
                // variable resolution (the pair's h per pair: more registers):
                // two pairs per iteration, the neighbour data one pair ahead
                uint32_t eA = cnt > 0 ? __ldcs(lp) : 0u;
                uint32_t eB = cnt > 1 ? __ldcs(lp + (size_t)n) : 0u;
                float4 pA = pos4[eA >> kCodeBits], oA = vr[eA >> kCodeBits];
                int k = 0;
                const uint32_t* lq = lp + 2 * (size_t)n;
                const size_t n2 = 2 * (size_t)n;
                for (; k + 1 < cnt; k += 2, lq += n2) {
                    const float4 pB = pos4[eB >> kCodeBits], oB = vr[eB >> kCodeBits];
                    const uint32_t eC = k + 2 < cnt ? __ldcs(lq) : 0u;
                    one(eA, pA, oA);
                    if (k + 2 < cnt) {
                        pA = pos4[eC >> kCodeBits];
                        oA = vr[eC >> kCodeBits];
                    }
                    const uint32_t eD = k + 3 < cnt ? __ldcs(lq + n) : 0u;
                    one(eB, pB, oB);
                    eA = eC;
                    eB = eD;
                }
                if (k < cnt) one(eA, pA, oA);
            }
        } else {
            // more neighbours than the list holds: scan the cells
            auto visit = [&](int j, uint32_t, const float4& pj, float r2, float rx, float ry, float rz) {
                if (r2 < support2<UNIFORM>(K, hi, pj.w) && r2 > 0.f) {
                    const float rv[3] = {rx, ry, rz};
                    pair(j, pj, vr[j], rv, r2);
                }
            };
            for_candidates<DIM>(oi, cell_of[i], G, start, pos4, visit);
        }
        float a[3] = {0, 0, 0}, R[3] = {0, 0, 0};
        float R2 = 0.f;
        const double m_i = S.m[i];
        // free-stream forcing lambda(x) (U_inf - v) of the fringe region,
        // at the particle's FP64 position along axis 0
        const float lam = K.fr_on ? fringe_rate<float>(K, (float)S.x[i]) : 0.f;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            // at uniform resolution the sums were taken without the factor C of W'/r
            const float pair_a = sums.a_value(d);
            // the fluid's momentum rate from its pair terms: minus the force on the walls
            if (K.body_force) part[9 + d] = m_i * (double)pair_a;
            a[d] = K.g[d] + pair_a;
            if (K.fr_on) a[d] = fmaf(lam, K.fr_u[d] - vi[d], a[d]);
            R[d] = sums.R_value(d);
            R2 += R[d] * R[d];
        }
        const float htv = K.tv_h_particle ? hi : K.h_min;
        const float htv2 = htv * htv;
        const float chi = tv_limiter(K, htv2 * R2);
        // Eq. 12 (background pressure p0 = rho0 c^2): dr = -(dt^2 p0 / rho_i) R_i
        // (its FP64 division only in that mode: FP64 is 1/74 of the FP32 rate)
        const bool bgmode = K.tv_mode == SPH_TV_BACKGROUND;
        const float bg = bgmode ? (float)(-(dt * dt * (double)(K.rho0 * K.c2)) / (double)rho_i) : 0.f;
        // momentum and kinetic energy in FP64; the maxima of the transport
        // speed |v + dr/dt| and of |dr| (diagnostics of the correction) from
        // FP32 squares, to keep this epilogue off the FP64 pipe
        const float inv_dt = dt > 0.0 ? 1.f / (float)dt : 0.f;
        const float hdtf = (float)hdt;
        double v2 = 0.0;
        float vt2 = 0.f, dr2 = 0.f;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const size_t o = (size_t)d * n + i;
            const float dr = bgmode ? bg * R[d] : K.tv_xi * chi * htv2 * R[d];
            const float vn = __fadd_rn(vi[d], __fmul_rn(hdtf, a[d]));
            if (write_ad) {
                S.a[o] = a[d];
                S.dr[o] = dr;
            }
            S.v[o] = vn;
            Rout[o] = R[d];
            part[1 + d] = m_i * (double)vn;
            v2 += (double)vn * vn;
            dr2 += dr * dr;
            const float vt = fmaf(dr, inv_dt, vn);
            vt2 += vt * vt;
        }
        chi_out[i] = chi;
        part[0] = m_i;
        part[4] = 0.5 * m_i * v2;
        part[5] = chi > 0.f ? 1.0 : 0.0;
        part[6] = v2;                 // squares: block_partials takes the roots
        part[7] = (double)vt2;
        part[8] = (double)dr2;
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
    block_partials<true>(part, partials + (size_t)blockIdx.x * kNPart, true, K.body_force != 0);
}

// --------------------------------------------------------------- launchers

static inline int nblk(int n, int t) { return (n + t - 1) / t; }

int nbl_capacity(int dim) { return list_capacity(dim); }

template <int DIM, typename Acc, bool U>
static void density_t(int n, const float4* pos4, const int32_t* cell_of, const int32_t* start, const Grid& G,
                      const Consts<float>& K, StateSet<float> S, float4* vr, uint32_t* nbl, int32_t* nbc,
                      cudaStream_t st, const float4* pos4c)
{
    const int T = n >= G.sms * kDensityTPB32 ? kDensityTPB32 : pair_threads(32, n, G.sms);
    k_density32<DIM, Acc, U><<<nblk(n, T), T, 0, st>>>(n, pos4, cell_of, start, G, K, S, vr, nbl, nbc,
                                                       nbl_capacity(DIM), pos4c);
}

// Particles the tile holds: the expected halo population (particles per
// cell x halo cells) with a margin, in whole warps, between 256 and 4096.
template <int DIM>
static int tile_capacity(int n, const Grid& G)
{
    const double per_cell = (double)n / (double)G.ncell;
    int cap = (int)(1.4 * per_cell * TileDims<DIM>::NHC) + 64;
    cap = (cap + 31) / 32 * 32;
    return cap < 256 ? 256 : (cap > 4096 ? 4096 : cap);
}

template <int DIM, typename Acc>
static cudaError_t density_tile_t(int mode, int n, const float4* pos4c, const int32_t* cell_of, const int32_t* start,
                                  const Grid& G, const Consts<float>& K, StateSet<float> S, float4* vr, uint32_t* nbl,
                                  int32_t* nbc, cudaStream_t st)
{
    using SH = TileShape<DIM>;
    const int nb0 = (G.nc[0] + SH::B0 - 1) / SH::B0, nb1 = (G.nc[1] + SH::B1 - 1) / SH::B1;
    const int nb2 = DIM == 3 ? (G.nc[2] + SH::B2 - 1) / SH::B2 : 1;
    const int cap = tile_capacity<DIM>(n, G);
    const int v = mode - 1;      // 0 tile walk, 1 cooperative, 2 flattened
    const size_t extra = v == 1 ? coop_table_bytes<DIM>() : (v == 2 ? flat_table_bytes<DIM>() : 0);
    const size_t smem = tile_smem_bytes<DIM>(cap, extra);
    auto kern = v == 1 ? k_density32_coop<DIM, Acc> : (v == 2 ? k_density32_flat<DIM, Acc> : k_density32_tile<DIM, Acc>);
    // opt in to more than 48 KB of dynamic shared memory once per kernel (and
    // again only for a larger size)
    static size_t opted[3] = {48 * 1024, 48 * 1024, 48 * 1024};
    if (smem > opted[v]) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        opted[v] = smem;
    }
    const int threads = v == 1 ? TileThreads<DIM>::COOP : (v == 2 ? FlatShape<DIM>::T : TileThreads<DIM>::WALK);
    kern<<<nb0 * nb1 * nb2, threads, smem, st>>>(n, pos4c, cell_of, start, G, K, S, vr, nbl, nbc, nbl_capacity(DIM),
                                                 nb0, nb1, cap);
    return cudaGetLastError();
}

template <int DIM, typename Acc, bool U>
static void forces_t(int n, const float4* pos4, const int32_t* cell_of, const int32_t* start, const Grid& G,
                     const Consts<float>& K, StateSet<float> S, const float* mf, const float4* vr,
                     const uint32_t* nbl, const int32_t* nbc, const double* dt, int kick_on, int write_ad,
                     float* Rout, float* chi, double* partials, cudaStream_t st)
{
    const int T = pair_threads(32, n, G.sms);
    k_forces32<DIM, Acc, U><<<nblk(n, T), T, 0, st>>>(n, pos4, cell_of, start, G, K, S, mf, vr, nbl, nbc,
                                                      nbl_capacity(DIM), dt, kick_on, write_ad, Rout, chi, partials);
}

#define SPH_DISPATCH32(FN, ...)                                                   \
    do {                                                                          \
        if (K.kahan) {                                                            \
            if (K.uniform_h) {                                                    \
                if (dim == 2) FN<2, KSum, true>(__VA_ARGS__);                     \
                else FN<3, KSum, true>(__VA_ARGS__);                              \
            } else {                                                              \
                if (dim == 2) FN<2, KSum, false>(__VA_ARGS__);                    \
                else FN<3, KSum, false>(__VA_ARGS__);                             \
            }                                                                     \
        } else {                                                                  \
            if (K.uniform_h) {                                                    \
                if (dim == 2) FN<2, PlainF, true>(__VA_ARGS__);                   \
                else FN<3, PlainF, true>(__VA_ARGS__);                            \
            } else {                                                              \
                if (dim == 2) FN<2, PlainF, false>(__VA_ARGS__);                  \
                else FN<3, PlainF, false>(__VA_ARGS__);                           \
            }                                                                     \
        }                                                                         \
    } while (0)

cudaError_t launch_density32(int dim, int n, void* Sv, const int32_t* start, const Grid& G, const void* Kv, void* vr,
                             const float4* pos4, const int32_t* cell_of, uint32_t* nbl, int32_t* nbc,
                             cudaStream_t st, const float4* pos4c, int tiles)
{
    const StateSet<float> S = *(StateSet<float>*)Sv;
    const Consts<float>& K = *(const Consts<float>*)Kv;
    if (K.uniform_h && !pos4c) return cudaErrorInvalidValue;   // the uniform walk reads the cell-tagged copy
    if (K.uniform_h && tiles) {
        float4* v4 = (float4*)vr;
        if (K.kahan) return dim == 2 ? density_tile_t<2, KSum>(tiles, n, pos4c, cell_of, start, G, K, S, v4, nbl, nbc, st)
                                     : density_tile_t<3, KSum>(tiles, n, pos4c, cell_of, start, G, K, S, v4, nbl, nbc, st);
        return dim == 2 ? density_tile_t<2, PlainF>(tiles, n, pos4c, cell_of, start, G, K, S, v4, nbl, nbc, st)
                        : density_tile_t<3, PlainF>(tiles, n, pos4c, cell_of, start, G, K, S, v4, nbl, nbc, st);
    }
    SPH_DISPATCH32(density_t, n, pos4, cell_of, start, G, K, S, (float4*)vr, nbl, nbc, st, pos4c);
    return cudaGetLastError();
}

cudaError_t launch_forces32(int dim, int n, void* Sv, const int32_t* start, const Grid& G, const void* Kv,
                            const float* mf, const void* vr, const float4* pos4, const int32_t* cell_of,
                            const uint32_t* nbl, const int32_t* nbc, const double* dt, int kick_on, int write_ad,
                            void* Rout, void* chi, double* partials, cudaStream_t st)
{
    const StateSet<float> S = *(StateSet<float>*)Sv;
    const Consts<float>& K = *(const Consts<float>*)Kv;
    SPH_DISPATCH32(forces_t, n, pos4, cell_of, start, G, K, S, mf, (const float4*)vr, nbl, nbc, dt, kick_on,
                   write_ad, (float*)Rout, (float*)chi, partials, st);
    return cudaGetLastError();
}

#undef SPH_DISPATCH32

}  // namespace sphtv
