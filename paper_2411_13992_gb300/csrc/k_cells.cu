// k_cells.cu -- the kick-drift stage and the cell-linked list of libsphtv.
//
// Per step:  kick + drift + cell key + histogram  ->  exclusive scan of the
// cell counts  ->  atomic scatter into cell ranges  ->  per-cell ordering by
// particle id (so the sorted order never depends on atomic timing)  ->
// permute the particle arrays into the new order (and, in both forms,
// emit FP32 positions relative to each particle's cell origin).
//
// The kick-drift follows the kick-drift-kick scheme the paper names (Sec. 1,
// Sec. 3): v += dt/2 a; x += dt v + dr, where dr is the transport-velocity
// displacement of the previous step (Eq. 16), applied once per step.  With the
// dual-criteria integrator (Sec. 2.4) the substeps have moved the particles
// already and this stage only wraps the periodic axes.
#include "common.cuh"
#include "launch.h"

namespace sphtv {

// A non-negative int as a double, exactly, on the integer ALU: the leading
// one sets the binary64 exponent, the bits below it the fraction.
__device__ __forceinline__ double i2d_exact(int c)
{
    if (c <= 0) return 0.0;                   // callers pass cell coordinates >= 0
    const int e = 31 - __clz(c);
    const unsigned long long frac = ((unsigned long long)c << (52 - e)) & 0xfffffffffffffULL;
    return __longlong_as_double((long long)(((unsigned long long)(e + 1023) << 52) | frac));
}

// A double rounded to the nearest float (ties to even), as the hardware
// conversion rounds it, on the integer ALU for results that are normal
// floats: the 52-bit fraction is cut to 23 bits and rounded up when the cut
// part is above half an ulp, or exactly half with an odd last kept bit (a
// carry out of the fraction raises the exponent, and past the largest float
// gives infinity, as rounding does).  Zeros, subnormal results, infinities
// and NaN take the hardware conversion.
__device__ __forceinline__ float d2f_rn(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7ff) - 1023;
    if (E < -126 || E > 127) return (float)x;
    const unsigned long long frac = b & 0xfffffffffffffULL;
    const unsigned keep = (unsigned)(frac >> 29);
    const unsigned long long cut = frac & 0x1fffffffULL;               // the 29 bits cut off
    const unsigned up = (cut > 0x10000000ULL || (cut == 0x10000000ULL && (keep & 1u))) ? 1u : 0u;
    const unsigned f = (((unsigned)(E + 127) << 23) + keep + up) | ((unsigned)(b >> 32) & 0x80000000u);
    return __uint_as_float(f);
}

template <typename Real>
__device__ __forceinline__ Real kick(Real v, double hdt, Real a);

template <>
__device__ __forceinline__ double kick<double>(double v, double hdt, double a)
{
    return __dadd_rn(v, __dmul_rn(hdt, a));
}

template <>
__device__ __forceinline__ float kick<float>(float v, double hdt, float a)
{
    return __fadd_rn(v, __fmul_rn(d2f_rn(hdt), a));
}

// FP64 value of a velocity or displacement component (exact either way).
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(float x) { return f2d_exact(x); }

// -1 for x < lo, +1 for x >= hi, else 0: the periodic wrap of axis d, as
// integer comparisons of order keys (dkey).
__device__ __forceinline__ int wrap_side(const Grid& G, double x, int d)
{
    const long long kx = dkey(x);
    return kx < dkey(G.lo[d]) ? -1 : (kx >= dkey(G.hi[d]) ? 1 : 0);
}

template <typename Real, int DIM>
__global__ void k_kick_drift_key(int n, StateSet<Real> S, const double* __restrict__ dt_ptr, int drift, Grid G,
                                 int32_t* __restrict__ key, int32_t* __restrict__ count, uint32_t* err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double xs[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) xs[d] = S.x[(size_t)d * n + i];
    uint32_t e = 0;
    if (drift == 2 && S.kind[i] == 0) {
        // dual-criteria integrator: the substeps moved the particles; only
        // the periodic wrap is left to do here
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            if (!G.periodic[d]) continue;
            const int w = wrap_side(G, xs[d], d);
            if (__any_sync(__activemask(), w != 0) && w != 0) {
                xs[d] = w < 0 ? __dadd_rn(xs[d], G.L[d]) : __dsub_rn(xs[d], G.L[d]);
                S.x[(size_t)d * n + i] = xs[d];
            }
        }
    } else if (drift == 1) {
        // every load issued before the kind test and the arithmetic
        Real vv[3] = {0, 0, 0}, aa[3] = {0, 0, 0}, rr[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const size_t o = (size_t)d * n + i;
            vv[d] = S.v[o];
            aa[d] = S.a[o];
            rr[d] = S.dr[o];
        }
        const double dt = *dt_ptr;
        if (S.kind[i] == 0) {
            const double hdt = 0.5 * dt;
            // FP32 form: the displacement dt v + dr in FP32 (one rounding, from
            // FP32 inputs), accumulated into the FP64 position
            const float dt_f = d2f_rn(dt);
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                size_t o = (size_t)d * n + i;
                Real vh = kick<Real>(vv[d], hdt, aa[d]);
                S.v[o] = vh;
                double xn;
                if (sizeof(Real) == 4)
                    xn = __dadd_rn(xs[d], to_double(__fmaf_rn(dt_f, (float)vh, (float)rr[d])));
                else
                    xn = __dadd_rn(__dadd_rn(xs[d], __dmul_rn(dt, to_double(vh))), to_double(rr[d]));
                if (G.periodic[d]) {
                    // the wrap only in warps where a particle left the box (the
                    // FP64 operation would otherwise be issued for every warp)
                    const int w = wrap_side(G, xn, d);
                    if (__any_sync(__activemask(), w != 0) && w != 0)
                        xn = w < 0 ? __dadd_rn(xn, G.L[d]) : __dsub_rn(xn, G.L[d]);
                }
                xs[d] = xn;
                S.x[o] = xn;
            }
        }
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        if (!finite_bits(xs[d])) e |= ERRB_NAN;
        else if (!G.periodic[d] && (dkey(xs[d]) < dkey(G.lo[d]) || dkey(xs[d]) > dkey(G.hi[d]))) e |= ERRB_DOMAIN;
    }
    if (e) atomicOr(err, e);
    int k = sort_key<DIM>(G, xs);
    key[i] = k;
    // one atomic per particle: with the sub-cell bins a warp's lanes seldom
    // share a bin, and aggregating them by __match_any_sync cost more than
    // it saved (3 % of this kernel at 128^3)
    atomicAdd(&count[k], 1);
}

// ------------------------------------------------------- exclusive scan

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan of in[0, n) into out (in place allowed); each block scans
// one tile and writes its total to bsum[blockIdx.x].
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const int32_t* in, int32_t* out, int32_t* bsum, int n)
{
    __shared__ int32_t warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int32_t vals[kScanItems];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int idx = base + k;
        vals[k] = idx < n ? in[idx] : 0;
        s += vals[k];
    }
    int32_t incl = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        constexpr int nw = kScanThreads / 32;
        int32_t t = lane < nw ? warp_tot[lane] : 0;
        int32_t ti = t;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int32_t u = __shfl_up_sync(0xffffffffu, ti, off);
            if (lane >= off) ti += u;
        }
        if (lane < nw) warp_tot[lane] = ti - t;
        if (lane == nw - 1) bsum[blockIdx.x] = ti;
    }
    __syncthreads();
    int32_t pre = warp_tot[w] + incl - s;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int idx = base + k;
        if (idx < n) out[idx] = pre;
        pre += vals[k];
    }
}

__global__ void k_scan_add(int32_t* out, const int32_t* boff, int n)
{
    int idx = blockIdx.x * kScanTile + threadIdx.x;
    int32_t add = boff[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k, idx += kScanThreads)
        if (idx < n) out[idx] += add;
}

size_t scan_temp_elems(int n)
{
    size_t tot = 0;
    while (n > 1) {
        n = (n + kScanTile - 1) / kScanTile;
        tot += (size_t)n + 1;
    }
    return tot + 1;
}

cudaError_t launch_exclusive_scan(const int32_t* in, int32_t* out, int n, int32_t* tmp, cudaStream_t st,
                                  int64_t* launches)
{
    int nb = (n + kScanTile - 1) / kScanTile;
    k_scan_tile<<<nb, kScanThreads, 0, st>>>(in, out, tmp, n);
    ++*launches;
    if (nb > 1) {
        cudaError_t e = launch_exclusive_scan(tmp, tmp, nb, tmp + nb + 1, st, launches);
        if (e != cudaSuccess) return e;
        k_scan_add<<<nb, kScanThreads, 0, st>>>(out, tmp, n);
        ++*launches;
    }
    return cudaGetLastError();
}

// The sort's scan without its last pass: prefix[k] = the exclusive sum of
// count[0, k) within k's tile of kScanTile bins, tile_off[b] (tmp) the sum of
// the tiles before tile b.  The start of bin k is prefix[k] +
// tile_off[k / kScanTile]; the scatter and the per-bin ordering add the tile
// offset as they read a start (one pass over the bins fewer).  Returns
// tile_off, or null for a single tile.
cudaError_t launch_scan_tiles(const int32_t* count, int32_t* prefix, int n, int32_t* tmp, cudaStream_t st,
                              int64_t* launches, const int32_t** tile_off)
{
    int nb = (n + kScanTile - 1) / kScanTile;
    k_scan_tile<<<nb, kScanThreads, 0, st>>>(count, prefix, tmp, n);
    ++*launches;
    *tile_off = nullptr;
    if (nb > 1) {
        cudaError_t e = launch_exclusive_scan(tmp, tmp, nb, tmp + nb + 1, st, launches);
        if (e != cudaSuccess) return e;
        *tile_off = tmp;
    }
    return cudaGetLastError();
}

__device__ __forceinline__ int bin_start_of(const int32_t* __restrict__ prefix, const int32_t* __restrict__ tile_off,
                                            int k)
{
    return prefix[k] + (tile_off ? tile_off[k / kScanTile] : 0);
}

// ------------------------------------------------ scatter and cell order

// Slots by atomics on the bins' counts, counting down: a bin of c particles
// hands out c - 1 .. 0, so every count is back at zero after the scatter
// (the next sort needs no clearing).  The order inside a bin is fixed
// afterwards by k_order_cells.  One atomic per particle: the sub-cell bins
// are seldom shared within a warp, and aggregating the lanes by
// __match_any_sync cost more than it saved.
__global__ void k_scatter(int n, const int32_t* __restrict__ key, const int32_t* __restrict__ prefix,
                          const int32_t* __restrict__ tile_off, int32_t* __restrict__ count,
                          int32_t* __restrict__ perm)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = key[i];
    const int pos = bin_start_of(prefix, tile_off, k) + atomicSub(&count[k], 1) - 1;
    perm[pos] = i;
}

// One thread per sort bin (cell, or sub-cell when the sort refines the
// cells): write the bin's start, and place the bin's particles in
// increasing caller id (ids are unique, so the rank of each is its slot).
// Cells hold about two particles (edge >= h_max), so the quadratic rank
// count is short.  With sub-cells (shift > 0) the thread of each cell's
// first sub-cell also writes the cell's start (the thread nbin, past the
// last bin, the end n).
__global__ void k_order_cells(int nbin, const int32_t* __restrict__ prefix, const int32_t* __restrict__ tile_off,
                              const int32_t* __restrict__ perm_in, const int32_t* __restrict__ id,
                              int32_t* __restrict__ perm_out, int32_t* __restrict__ start, int shift,
                              int32_t* __restrict__ cell_start)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > nbin) return;
    const int s = bin_start_of(prefix, tile_off, c);
    start[c] = s;
    if (shift && (c & ((1 << shift) - 1)) == 0) cell_start[c >> shift] = s;
    if (c == nbin) return;
    const int e = bin_start_of(prefix, tile_off, c + 1);
    for (int k = s; k < e; ++k) {
        const int p = perm_in[k];
        const int myid = id[p];
        int rank = 0;
        for (int t = s; t < e; ++t) rank += id[perm_in[t]] < myid;
        perm_out[s + rank] = p;
    }
}

// --------------------------------------------------------------- permute

// pos4 = {offset from the cell origin, h} (uniform resolution:
// {offset, m}, since h is then a constant), mf = m in FP32, cell_out = key;
// pos4c (when given: the FP32 form at uniform resolution) = {offset, bits of
// the cell index}, which the FP32 density walk reads instead of pos4 and
// cell_out.  When *varies is 0 every particle has particle 0's h, m and
// sigma0 and is a fluid particle, and both state sets hold these arrays
// (set by sph_set_state): they are left where they are.
template <typename Real, int DIM, bool CARRY_AD, bool F32POS>
__global__ void k_permute(int n, const int32_t* __restrict__ perm, StateSet<Real> src, StateSet<Real> dst,
                          const int32_t* __restrict__ key, Grid G, float4* __restrict__ pos4,
                          int32_t* __restrict__ cell_out, float* __restrict__ mf, int uniform_h,
                          float4* __restrict__ pos4c, const uint32_t* __restrict__ varies)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const bool moves = *varies != 0;
    int i = perm[k];
    double xs[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        size_t so = (size_t)d * n + i, dof = (size_t)d * n + k;
        xs[d] = src.x[so];
        dst.x[dof] = xs[d];
        dst.v[dof] = src.v[so];
        if (CARRY_AD) {
            dst.a[dof] = src.a[so];
            dst.dr[dof] = src.dr[so];
        }
    }
    if (src.drho) dst.drho[k] = src.drho[i];
    const double h = moves ? src.h[i] : src.h[0];
    const double m = moves ? src.m[i] : src.m[0];
    if (moves) {
        dst.h[k] = h;
        dst.m[k] = m;
        dst.s0[k] = src.s0[i];
        dst.kind[k] = src.kind[i];
    }
    dst.id[k] = src.id[i];
    if (F32POS) {
        int kk = key[i] >> G.sub_shift;   // the cell of the sort key
        int c[3];
        cell_decode(G, kk, c);
        float o[3] = {0.f, 0.f, 0.f};
        // the conversions on the integer ALU (the same values as the hardware
        // conversions, which run on the FP64 pipe)
#pragma unroll
        for (int d = 0; d < DIM; ++d) o[d] = d2f_rn(xs[d] - (G.lo[d] + i2d_exact(c[d]) * G.edge[d]));
        const float m_f = d2f_rn(m);
        pos4[k] = make_float4(o[0], o[1], o[2], uniform_h ? m_f : d2f_rn(h));
        if (pos4c) pos4c[k] = make_float4(o[0], o[1], o[2], __int_as_float(kk));
        cell_out[k] = kk;
        mf[k] = m_f;
    }
}

// ------------------------------------------------------------- launchers

static inline int nblk(int n, int t) { return (n + t - 1) / t; }

cudaError_t launch_kick_drift_key(int prec, int dim, int n, void* S, const double* dt, int drift, const Grid& G,
                                  int32_t* key, int32_t* count, uint32_t* err, cudaStream_t st)
{
    const int T = 256;
    if (prec == 64) {
        auto s = *(StateSet<double>*)S;
        if (dim == 2) k_kick_drift_key<double, 2><<<nblk(n, T), T, 0, st>>>(n, s, dt, drift, G, key, count, err);
        else k_kick_drift_key<double, 3><<<nblk(n, T), T, 0, st>>>(n, s, dt, drift, G, key, count, err);
    } else {
        auto s = *(StateSet<float>*)S;
        if (dim == 2) k_kick_drift_key<float, 2><<<nblk(n, T), T, 0, st>>>(n, s, dt, drift, G, key, count, err);
        else k_kick_drift_key<float, 3><<<nblk(n, T), T, 0, st>>>(n, s, dt, drift, G, key, count, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_scatter_order(int n, int nbin, const int32_t* key, const int32_t* prefix, const int32_t* tile_off,
                                 int32_t* count, int32_t* perm_tmp, const int32_t* id, int32_t* perm, int32_t* start,
                                 int shift, int32_t* cell_start, cudaStream_t st, int64_t* launches)
{
    const int T = 256;
    k_scatter<<<nblk(n, T), T, 0, st>>>(n, key, prefix, tile_off, count, perm_tmp);
    k_order_cells<<<nblk(nbin + 1, T), T, 0, st>>>(nbin, prefix, tile_off, perm_tmp, id, perm, start, shift,
                                                   cell_start);
    *launches += 2;
    return cudaGetLastError();
}

template <typename Real>
static void permute_t(int dim, int n, const int32_t* perm, void* src, void* dst, const int32_t* key,
                      const Grid& G, float4* pos4, int32_t* cell, float* mf, int uh, int carry_ad, cudaStream_t st,
                      float4* pos4c, const uint32_t* varies)
{
    const int T = 256;
    auto s = *(StateSet<Real>*)src;
    auto d = *(StateSet<Real>*)dst;
    constexpr bool F32 = true;   // both forms: the density passes walk the FP32 cell-relative positions
    if (dim == 2) {
        if (carry_ad)
            k_permute<Real, 2, true, F32><<<nblk(n, T), T, 0, st>>>(n, perm, s, d, key, G, pos4, cell, mf, uh, pos4c, varies);
        else
            k_permute<Real, 2, false, F32><<<nblk(n, T), T, 0, st>>>(n, perm, s, d, key, G, pos4, cell, mf, uh, pos4c, varies);
    } else {
        if (carry_ad)
            k_permute<Real, 3, true, F32><<<nblk(n, T), T, 0, st>>>(n, perm, s, d, key, G, pos4, cell, mf, uh, pos4c, varies);
        else
            k_permute<Real, 3, false, F32><<<nblk(n, T), T, 0, st>>>(n, perm, s, d, key, G, pos4, cell, mf, uh, pos4c, varies);
    }
}

cudaError_t launch_permute(int prec, int dim, int n, const int32_t* perm, void* src, void* dst, const int32_t* key,
                           const Grid& G, float4* pos4, int32_t* cell, float* mf, int uniform_h, int carry_ad,
                           cudaStream_t st, const uint32_t* varies, float4* pos4c)
{
    if (prec == 64)
        permute_t<double>(dim, n, perm, src, dst, key, G, pos4, cell, mf, uniform_h, carry_ad, st, pos4c, varies);
    else
        permute_t<float>(dim, n, perm, src, dst, key, G, pos4, cell, mf, uniform_h, carry_ad, st, pos4c, varies);
    return cudaGetLastError();
}

}  // namespace sphtv
