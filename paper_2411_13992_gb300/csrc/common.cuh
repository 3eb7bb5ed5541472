// common.cuh -- device helpers shared by the libsphtv kernels: the Wendland
// C2 kernel (Sec. 4, h = 1.3 dp, support 2h), the cell grid of the
// cell-linked list, compensated FP32 summation, and the context's buffer
// layout.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sphtv.h"

namespace sphtv {

constexpr double kPi = 3.14159265358979323846;

// Device error word bits (sticky; read back by sph_sync).
enum : uint32_t { ERRB_OVERFLOW = 1u, ERRB_NAN = 2u, ERRB_DOMAIN = 4u, ERRB_INPUT = 8u };

// Device state of the dual-criteria integrator (doubles).
enum {
    DU_DT_AD = 0,     // advection step size of the current step (Eq. 9-10)
    DU_VAD = 1,       // advection speed |v|_ad (Eq. 10)
    DU_T = 2,         // time advanced by the substeps so far
    DU_DT = 3,        // size of the next (or current) acoustic substep (Eq. 11)
    DU_HDT_PREV = 4,  // half the previous substep (its density update is completed late)
    DU_LAST = 5,      // 1: the current substep ends the advection step
    DU_DONE = 6,      // 1: the advection step is complete (later substep launches are no-ops)
    DU_K = 7,         // substeps taken in the current advection step
    DU_FIRST = 8,     // 1: the next substep is the first of its advection step
    DU_COUNT = 16
};

// Number of FP64 per-block partial values the fused force kernel writes
// (layout in block_partials).
constexpr int kNPart = 12;
// Indices into the device diagnostics block (doubles).
enum {
    DG_MASS = 0, DG_MOM = 1, DG_KE = 4, DG_VMAX = 5, DG_VTMAX = 6, DG_DRMAX = 7, DG_NCHI = 8,
    DG_DT = 9, DG_DTNEXT = 10, DG_STEPS = 11, DG_SUBSTEPS = 12, DG_FBODY = 13, DG_IMPULSE = 16, DG_TIME = 19,
    DG_COUNT = 20
};

// Cell grid of the cell-linked list: edge >= 2 h_max / R along every axis,
// so every neighbour of a particle lies in the (2R+1)^D block of cells around
// its own (R = stencil radius in cells).
constexpr int kStencilR = 2;
struct Grid {
    int R;              // stencil radius in cells
    int nc[3];
    int periodic[3];
    double lo[3];
    double hi[3];       // lo + L, computed once on the host
    double L[3];
    double half_L[3];
    double edge[3];
    double inv_edge[3];
    float edgef[3];
    int ncell;
    int sms;            // streaming multiprocessors of the device (grid sizing of the pair passes)
    // The counting sort may refine each cell along axis 0 into 2^sub_shift
    // sub-cells (sorted by sub-cell, then by id, inside the cell): sub_start
    // [(ncell << sub_shift) + 1] holds the first particle of each sub-cell
    // in the sort order, so that a row walk can cut its runs at sub-cell
    // rather than cell granularity.  inv_edge_sub0 = inv_edge[0] 2^sub_shift.
    int sub_shift;
    double inv_edge_sub0;
    const int32_t* sub_start;
};

// Constants of the method for one precision.
template <typename Real>
struct Consts {
    Real rho0, c, c2, eta, two_eta, beta_slope, inv_c;
    Real g[3];
    Real h_min, tv_xi, tv_C, tv_thresh;
    int tv_mode, tv_h_particle, h_pair_max, kahan;
    // uniform resolution (h_min == h_max): every pair has h_ij = h
    int uniform_h;
    // sum the fluid's pair-force momentum rate (the body force of Eq. 18)
    int body_force;
    // fringe-region free-stream forcing lambda(x) (U_inf - v) along axis 0:
    // fr_lambda (0: off), U_inf, and x0, x1, rise, fall
    int fr_on;
    Real fr_lambda;
    Real fr_u[3];
    Real fr_x[4];
    // h_u = h_max (the h of every pair at uniform resolution)
    Real h_u, inv_h_u, four_h2_u, dwr_coef_u;   // dwr_coef_u: W'(r)/r = dwr_coef_u t^3
};

// Velocity + density deviation packed per particle for the pair pass:
// w = rho - rho0 (fluid), +inf marks a wall particle.
template <typename Real> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
template <> struct Vec4<double> { using T = double4_32a; };

// ------------------------------------------------------------ kernel W

template <int DIM, typename Real>
__device__ __forceinline__ Real kernel_norm()
{
    // a_D h^D: 7/(4 pi) in 2-D, 21/(16 pi) in 3-D
    return DIM == 2 ? Real(7.0 / (4.0 * kPi)) : Real(21.0 / (16.0 * kPi));
}

template <int DIM, typename Real>
__device__ __forceinline__ Real pow_dim(Real x)
{
    return DIM == 2 ? x * x : x * x * x;
}

// W(r, h) for r < 2h (callers test the support first).
template <int DIM, typename Real>
__device__ __forceinline__ Real wendland_W(Real r, Real inv_h)
{
    Real q = r * inv_h;
    Real t = Real(1) - Real(0.5) * q;
    Real t2 = t * t;
    return kernel_norm<DIM, Real>() * pow_dim<DIM, Real>(inv_h) * (t2 * t2) * (Real(2) * q + Real(1));
}

// dW/dr (r, h) for r < 2h.
template <int DIM, typename Real>
__device__ __forceinline__ Real wendland_dW(Real r, Real inv_h)
{
    Real q = r * inv_h;
    Real t = Real(1) - Real(0.5) * q;
    return kernel_norm<DIM, Real>() * pow_dim<DIM, Real>(inv_h) * inv_h * (Real(-5) * q) * (t * t * t);
}

// d^2W/dr^2 (r, h) for r < 2h.
template <int DIM, typename Real>
__device__ __forceinline__ Real wendland_d2W(Real r, Real inv_h)
{
    Real q = r * inv_h;
    Real t = Real(1) - Real(0.5) * q;
    return kernel_norm<DIM, Real>() * pow_dim<DIM, Real>(inv_h) * inv_h * inv_h * Real(-5) * (t * t) *
           (Real(1) - Real(2) * q);
}

// ------------------------------------------------------- compensated sum

struct KSum {
    float s, c;
    __device__ __forceinline__ KSum() : s(0.f), c(0.f) {}
    __device__ __forceinline__ void add(float x)
    {
        // Kahan: explicit round-to-nearest intrinsics so that neither
        // contraction nor reassociation removes the compensation.
        float y = __fsub_rn(x, c);
        float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    // add(x) when p holds, else nothing (selected, no branch)
    __device__ __forceinline__ void add_if(float x, bool p)
    {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        const float cn = __fsub_rn(__fsub_rn(t, s), y);
        s = p ? t : s;
        c = p ? cn : c;
    }
    __device__ __forceinline__ float value() const { return s; }
};

struct PlainF {
    float s;
    __device__ __forceinline__ PlainF() : s(0.f) {}
    __device__ __forceinline__ void add(float x) { s += x; }
    __device__ __forceinline__ void add_if(float x, bool p) { s = p ? s + x : s; }
    __device__ __forceinline__ float value() const { return s; }
};

struct PlainD {
    double s;
    __device__ __forceinline__ PlainD() : s(0.0) {}
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

// ------------------------------------------------------------ cell grid

// Cell coordinate along axis d, clamped to the grid.  Truncation equals
// floor for t >= 0, and negative t clamps to 0 either way; the conversion
// saturates large values and maps NaN to 0 (the kick-drift kernel flags
// non-finite positions separately).  Two FP64 operations and a conversion:
// GB300's FP64 pipe is narrow.
// Order key of a double on the integer ALU: for non-NaN a and b, a < b
// exactly when dkey(a) < dkey(b) (the magnitude bits of negative values
// inverted, -0.0 folded onto +0.0), which keeps comparisons off the FP64 pipe.
__device__ __forceinline__ long long dkey(double a)
{
    long long k = __double_as_longlong(a);
    if (k == (long long)0x8000000000000000ULL) k = 0;
    return k ^ ((k >> 63) & 0x7fffffffffffffffLL);
}

// The value of a float as a double, exactly, on the integer ALU (IEEE 754
// binary32 -> binary64: same sign, exponent rebased by 1023 - 127, fraction
// shifted by 52 - 23; zero keeps its sign); subnormal, infinite and NaN
// floats take the hardware conversion.  Keeps the conversion off the FP64
// pipe, which the position update saturates.
__device__ __forceinline__ double f2d_exact(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    if (e == 0u) {
        if ((u & 0x7fffffu) == 0u) return __longlong_as_double((long long)sign);
        return (double)f;
    }
    if (e == 0xffu) return (double)f;
    return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 896u) << 52) |
                                            ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// max(trunc(t), 0) on the integer ALU for the cell index (the callers clamp
// it to [0, nc - 1]), as the hardware conversion toward zero then the clamp
// would give it: 0 for t < 1 (and -0.0, negative t, NaN), the integer part
// read from the binary64 fraction for 1 <= t < 2^31, INT_MAX beyond.
__device__ __forceinline__ int trunc_nonneg(double t)
{
    const long long b = __double_as_longlong(t);
    if (b < 0) return 0;
    const int E = (int)((b >> 52) & 0x7ff) - 1023;
    if (E < 0) return 0;
    if (E == 1024 && (b & 0xfffffffffffffLL) != 0) return 0;     // NaN
    if (E > 30) return 0x7fffffff;
    const long long m = (b & 0xfffffffffffffLL) | (1LL << 52);
    return (int)(m >> (52 - E));
}

__device__ __forceinline__ int cell_coord(const Grid& G, double x, int d)
{
    // x - lo is x itself when lo = 0 (bit for bit), one FP64 operation fewer
    // (lo = +-0 read from its bit pattern); the truncation (toward zero, then
    // clamped) on the integer ALU
    const double t = (__double_as_longlong(G.lo[d]) << 1) == 0 ? x : __dsub_rn(x, G.lo[d]);
    const int c = trunc_nonneg(t * G.inv_edge[d]);
    return min(max(c, 0), G.nc[d] - 1);
}

// x is finite (not inf or NaN), tested on the exponent bits.
__device__ __forceinline__ bool finite_bits(double x)
{
    return (__double_as_longlong(x) & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}

template <int DIM>
__device__ __forceinline__ int cell_index(const Grid& G, const double* xs)
{
    int c0 = cell_coord(G, xs[0], 0);
    int c1 = cell_coord(G, xs[1], 1);
    int c2 = DIM == 3 ? cell_coord(G, xs[2], 2) : 0;
    return c0 + G.nc[0] * (c1 + G.nc[1] * c2);
}

// The sort key of a position: the cell index when sub_shift = 0; else the
// sub-cell index ((cell << sub_shift) | sub-cell along axis 0), whose high
// bits are cell_index's: the sub-cell coordinate is the truncation of
// (x - lo) inv_edge 2^s, and the scaling by 2^s is exact, so shifting the
// coordinate right by s gives the truncation of (x - lo) inv_edge (the
// clamps to the last cell and sub-cell commute with the shift as well).
template <int DIM>
__device__ __forceinline__ int sort_key(const Grid& G, const double* xs)
{
    if (G.sub_shift == 0) return cell_index<DIM>(G, xs);
    const int nsx = G.nc[0] << G.sub_shift;
    const double t = (__double_as_longlong(G.lo[0]) << 1) == 0 ? xs[0] : __dsub_rn(xs[0], G.lo[0]);
    const int s0 = min(max(trunc_nonneg(t * G.inv_edge_sub0), 0), nsx - 1);
    const int c1 = cell_coord(G, xs[1], 1);
    const int c2 = DIM == 3 ? cell_coord(G, xs[2], 2) : 0;
    return s0 + nsx * (c1 + G.nc[1] * c2);
}

__device__ __forceinline__ void cell_decode(const Grid& G, int key, int* c)
{
    c[0] = key % G.nc[0];
    int r = key / G.nc[0];
    c[1] = r % G.nc[1];
    c[2] = r / G.nc[1];
}

// Neighbour cell coordinate along axis d, or -1 when it falls outside a
// non-periodic axis.
__device__ __forceinline__ int cell_step(const Grid& G, int c, int dc, int d)
{
    int n = c + dc;
    if (n < 0 || n >= G.nc[d]) {
        if (!G.periodic[d]) return -1;
        n = n < 0 ? n + G.nc[d] : n - G.nc[d];
    }
    return n;
}

// x_i - x_j along axis d with the minimum image on periodic axes (FP64).
__device__ __forceinline__ double min_image(const Grid& G, double xi, double xj, int d)
{
    double dx = __dsub_rn(xi, xj);
    if (G.periodic[d]) {
        if (dx > G.half_L[d]) dx = __dsub_rn(dx, G.L[d]);
        else if (dx < -G.half_L[d]) dx = __dadd_rn(dx, G.L[d]);
    }
    return dx;
}

// 1/x and sqrt(x) to ~1 ulp on the special-function unit (x > 0, normal):
// the FP32 form needs neither the IEEE-rounded division nor square root.
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Neighbour-list entries: (j << kCodeBits) | stencil code of j's cell, the
// code being (dx + R) + S (dy + R) + S^2 (dz + R) with S = 2R + 1.
constexpr int kSide = 2 * kStencilR + 1;                 // stencil cells per axis
constexpr int kCodes = kSide * kSide * kSide;            // 125 for R = 2
constexpr int kCodeBits = 7;
static_assert(kCodes <= (1 << kCodeBits), "stencil code does not fit");

// Entries per particle of the force-neighbour list (a particle with more
// neighbours is walked over its cells instead).
__host__ __device__ constexpr int list_capacity(int dim) { return dim == 3 ? 128 : 96; }

// FP32 shift of a neighbour cell from its stencil code: the pair vector is
// (o_i - o_j) + shift for cell-relative offsets o.
__device__ __forceinline__ void code_shift(const Grid& G, uint32_t code, float* sh)
{
    const int dx = (int)(code % kSide) - kStencilR, dy = (int)((code / kSide) % kSide) - kStencilR,
              dz = (int)(code / (kSide * kSide)) - kStencilR;
    sh[0] = -(float)dx * G.edgef[0];
    sh[1] = -(float)dy * G.edgef[1];
    sh[2] = -(float)dz * G.edgef[2];
}

// ------------------------------------------------------------ buffers

// Particle arrays of one cell-sorted copy of the state.
template <typename Real>
struct StateSet {
    double* x;      // [DIM][n] positions (FP64 master in both precisions)
    Real* v;        // [DIM][n] velocities (walls: prescribed velocity)
    Real* a;        // [DIM][n] accelerations (only carried by the first sort)
    Real* dr;       // [DIM][n] transport displacements (only carried by the first sort)
    Real* drho;     // [n] density rate of the dual-criteria integrator (carried by every sort), or null
    double* h;      // [n] smoothing lengths
    double* m;      // [n] masses
    double* s0;     // [n] reference sums sigma0 (Eq. 8)
    int32_t* id;    // [n] caller's particle index
    int8_t* kind;   // [n] 0 fluid, 1 wall
};

}  // namespace sphtv
