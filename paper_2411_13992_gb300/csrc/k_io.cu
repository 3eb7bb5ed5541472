// k_io.cu -- state transfer kernels of libsphtv: caller [n][3] rows <->
// per-component arrays, un-permuting from the cell order back to the
// caller's order, wall velocities, and the per-particle reference sums
// sigma0 of Eq. 8 (the perfect-lattice sum at the particle's own spacing
// dp = (m/rho0)^(1/D) and smoothing length h).
#include "common.cuh"
#include "launch.h"

namespace sphtv {

template <typename Real, int DIM>
__global__ void k_vec_in(int n, const double* __restrict__ src3, Real* __restrict__ dst)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int d = 0; d < DIM; ++d) dst[(size_t)d * n + i] = (Real)src3[3 * (size_t)i + d];
}

template <typename Real, int DIM>
__global__ void k_vec_out(int n, const Real* __restrict__ src, const int32_t* __restrict__ id,
                          double* __restrict__ dst3)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    size_t o = 3 * (size_t)id[k];
#pragma unroll
    for (int d = 0; d < 3; ++d) dst3[o + d] = d < DIM ? (double)src[(size_t)d * n + k] : 0.0;
}

// pos[id[k]] = k: where the particle the caller gave as number i sits in
// the cell order.
__global__ void k_inverse_perm(int n, const int32_t* __restrict__ id, int32_t* __restrict__ pos)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) pos[id[k]] = k;
}

// k_vec_out by gathering: dst3 row i (the caller's order) from the sorted
// position pos[i], so the writes of a warp are contiguous (the destination
// may be page-locked host memory written across the host link).
template <typename Real, int DIM>
__global__ void k_vec_out_gather(int n, const Real* __restrict__ src, const int32_t* __restrict__ pos,
                                 double* __restrict__ dst3)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t k = (size_t)pos[i];
#pragma unroll
    for (int d = 0; d < 3; ++d) dst3[3 * (size_t)i + d] = d < DIM ? (double)src[(size_t)d * n + k] : 0.0;
}

template <typename V4>
__global__ void k_rho_out_gather(int n, const V4* __restrict__ vr, const int8_t* __restrict__ kind,
                                 const int32_t* __restrict__ pos, double rho0, double* __restrict__ dst)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = pos[i];
    dst[i] = kind[k] ? rho0 : rho0 + (double)vr[k].w;
}

template <typename Real, int DIM>
__global__ void k_walls_velocity(int n, const int8_t* __restrict__ kind, const double* __restrict__ vw3,
                                 Real* __restrict__ v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !kind[i]) return;
#pragma unroll
    for (int d = 0; d < DIM; ++d) v[(size_t)d * n + i] = vw3 ? (Real)vw3[3 * (size_t)i + d] : Real(0);
}

__global__ void k_init_ids(int n, int32_t* id)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) id[i] = i;
}

template <int DIM>
__device__ double sigma0_of(double h, double m, double rho0)
{
    const double vol = m / rho0;
    const double dp = DIM == 2 ? sqrt(vol) : cbrt(vol);
    const double ratio = h / dp;               // smoothing length in units of dp
    const double reach2 = 4.0 * ratio * ratio;
    const int K = (int)ceil(2.0 * ratio);
    const double inv = 1.0 / ratio;
    // One octant of the integer lattice; each point stands for its 2^(number
    // of non-zero coordinates) mirror images.
    double s = 0.0;
    const int kz1 = DIM == 3 ? K : 0;
    for (int kz = 0; kz <= kz1; ++kz)
        for (int ky = 0; ky <= K; ++ky)
            for (int kx = 0; kx <= K; ++kx) {
                double r2 = (double)(kx * kx + ky * ky + kz * kz);
                if (r2 >= reach2) continue;
                double mult = (kx ? 2.0 : 1.0) * (ky ? 2.0 : 1.0) * (kz ? 2.0 : 1.0);
                s += mult * wendland_W<DIM, double>(sqrt(r2), inv);
            }
    return s / (DIM == 2 ? dp * dp : dp * dp * dp);
}

// The reference sum depends on (h, m) only: particle 0's value is computed
// once (k_sigma0_first) and copied to every particle with the same h and m;
// the others compute their own (the lattice sum is FP64 work, and FP64 runs
// at 1/74 of the FP32 rate).
template <int DIM>
__global__ void k_sigma0_first(const double* __restrict__ h, const double* __restrict__ m, double rho0,
                               double* __restrict__ s0)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) s0[0] = sigma0_of<DIM>(h[0], m[0], rho0);
}

template <int DIM>
__global__ void k_sigma0(int n, const double* __restrict__ h, const double* __restrict__ m, double rho0,
                         double* __restrict__ s0)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 1 || i >= n) return;
    s0[i] = (h[i] == h[0] && m[i] == m[0]) ? s0[0] : sigma0_of<DIM>(h[i], m[i], rho0);
}

template <typename V4>
__global__ void k_rho_out(int n, const V4* __restrict__ vr, const int8_t* __restrict__ kind,
                          const int32_t* __restrict__ id, double rho0, double* __restrict__ dst)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    dst[id[k]] = kind[k] ? rho0 : rho0 + (double)vr[k].w;
}

// Every h must lie in [h_min, h_max] (the cell edge is sized by h_max) and
// every mass must be positive and finite.
__global__ void k_check_input(int n, const double* __restrict__ h, const double* __restrict__ m, double h_min,
                              double h_max, uint32_t* err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool ok = h[i] >= h_min && h[i] <= h_max && m[i] > 0.0 && isfinite(m[i]);
    if (!ok) atomicOr(err, ERRB_INPUT);
}

// Sets *varies (cleared by the caller) when a particle's h, m or sigma0
// differs from particle 0's or a particle is a wall particle.
__global__ void k_check_constants(int n, const double* __restrict__ h, const double* __restrict__ m,
                                  const double* __restrict__ s0, const int8_t* __restrict__ kind, uint32_t* varies)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool v = kind[i] != 0 || h[i] != h[0] || m[i] != m[0] || s0[i] != s0[0];
    const unsigned b = __ballot_sync(__activemask(), v);
    if (b && (threadIdx.x & 31) == __ffs(b) - 1) atomicOr(varies, 1u);
}

template <typename Real>
__global__ void k_scalar_out(int n, const Real* __restrict__ src, const int32_t* __restrict__ id,
                             double* __restrict__ dst)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dst[id[k]] = (double)src[k];
}

// Caller-order scalar in (walls get 0); used before the first sort, when the
// internal order is the caller's.
template <typename Real>
__global__ void k_scalar_in(int n, const double* __restrict__ src, const int8_t* __restrict__ kind,
                            Real* __restrict__ dst)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = kind[i] ? Real(0) : (Real)src[i];
}

static inline int nblk(int n, int t) { return (n + t - 1) / t; }

cudaError_t launch_vec_in(int prec, int dim, int n, const double* src3, void* dst, cudaStream_t st)
{
    const int T = 256;
    if (prec == 64) {
        if (dim == 2) k_vec_in<double, 2><<<nblk(n, T), T, 0, st>>>(n, src3, (double*)dst);
        else k_vec_in<double, 3><<<nblk(n, T), T, 0, st>>>(n, src3, (double*)dst);
    } else {
        if (dim == 2) k_vec_in<float, 2><<<nblk(n, T), T, 0, st>>>(n, src3, (float*)dst);
        else k_vec_in<float, 3><<<nblk(n, T), T, 0, st>>>(n, src3, (float*)dst);
    }
    return cudaGetLastError();
}

cudaError_t launch_vec_out(int prec, int dim, int n, const void* src, const int32_t* id, double* dst3,
                           cudaStream_t st)
{
    const int T = 256;
    if (prec == 64) {
        if (dim == 2) k_vec_out<double, 2><<<nblk(n, T), T, 0, st>>>(n, (const double*)src, id, dst3);
        else k_vec_out<double, 3><<<nblk(n, T), T, 0, st>>>(n, (const double*)src, id, dst3);
    } else {
        if (dim == 2) k_vec_out<float, 2><<<nblk(n, T), T, 0, st>>>(n, (const float*)src, id, dst3);
        else k_vec_out<float, 3><<<nblk(n, T), T, 0, st>>>(n, (const float*)src, id, dst3);
    }
    return cudaGetLastError();
}

cudaError_t launch_walls_velocity(int prec, int dim, int n, const int8_t* kind, const double* vw3, void* v,
                                  cudaStream_t st)
{
    const int T = 256;
    if (prec == 64) {
        if (dim == 2) k_walls_velocity<double, 2><<<nblk(n, T), T, 0, st>>>(n, kind, vw3, (double*)v);
        else k_walls_velocity<double, 3><<<nblk(n, T), T, 0, st>>>(n, kind, vw3, (double*)v);
    } else {
        if (dim == 2) k_walls_velocity<float, 2><<<nblk(n, T), T, 0, st>>>(n, kind, vw3, (float*)v);
        else k_walls_velocity<float, 3><<<nblk(n, T), T, 0, st>>>(n, kind, vw3, (float*)v);
    }
    return cudaGetLastError();
}

cudaError_t launch_init_ids(int n, int32_t* id, cudaStream_t st)
{
    k_init_ids<<<nblk(n, 256), 256, 0, st>>>(n, id);
    return cudaGetLastError();
}

cudaError_t launch_sigma0(int dim, int n, const double* h, const double* m, double rho0, double* s0,
                          cudaStream_t st)
{
    if (dim == 2) {
        k_sigma0_first<2><<<1, 32, 0, st>>>(h, m, rho0, s0);
        k_sigma0<2><<<nblk(n, 128), 128, 0, st>>>(n, h, m, rho0, s0);
    } else {
        k_sigma0_first<3><<<1, 32, 0, st>>>(h, m, rho0, s0);
        k_sigma0<3><<<nblk(n, 128), 128, 0, st>>>(n, h, m, rho0, s0);
    }
    return cudaGetLastError();
}

cudaError_t launch_rho_out(int prec, int n, const void* vr, const int8_t* kind, const int32_t* id, double rho0,
                           double* dst, cudaStream_t st)
{
    if (prec == 64) k_rho_out<double4_32a><<<nblk(n, 256), 256, 0, st>>>(n, (const double4_32a*)vr, kind, id, rho0, dst);
    else k_rho_out<float4><<<nblk(n, 256), 256, 0, st>>>(n, (const float4*)vr, kind, id, rho0, dst);
    return cudaGetLastError();
}

cudaError_t launch_inverse_perm(int n, const int32_t* id, int32_t* pos, cudaStream_t st)
{
    k_inverse_perm<<<nblk(n, 256), 256, 0, st>>>(n, id, pos);
    return cudaGetLastError();
}

cudaError_t launch_vec_out_gather(int prec, int dim, int n, const void* src, const int32_t* pos, double* dst3,
                                  cudaStream_t st)
{
    const int T = 256;
    if (prec == 64) {
        if (dim == 2) k_vec_out_gather<double, 2><<<nblk(n, T), T, 0, st>>>(n, (const double*)src, pos, dst3);
        else k_vec_out_gather<double, 3><<<nblk(n, T), T, 0, st>>>(n, (const double*)src, pos, dst3);
    } else {
        if (dim == 2) k_vec_out_gather<float, 2><<<nblk(n, T), T, 0, st>>>(n, (const float*)src, pos, dst3);
        else k_vec_out_gather<float, 3><<<nblk(n, T), T, 0, st>>>(n, (const float*)src, pos, dst3);
    }
    return cudaGetLastError();
}

cudaError_t launch_rho_out_gather(int prec, int n, const void* vr, const int8_t* kind, const int32_t* pos,
                                  double rho0, double* dst, cudaStream_t st)
{
    if (prec == 64)
        k_rho_out_gather<double4_32a><<<nblk(n, 256), 256, 0, st>>>(n, (const double4_32a*)vr, kind, pos, rho0, dst);
    else k_rho_out_gather<float4><<<nblk(n, 256), 256, 0, st>>>(n, (const float4*)vr, kind, pos, rho0, dst);
    return cudaGetLastError();
}

cudaError_t launch_check_input(int n, const double* h, const double* m, double h_min, double h_max, uint32_t* err,
                               cudaStream_t st)
{
    k_check_input<<<nblk(n, 256), 256, 0, st>>>(n, h, m, h_min, h_max, err);
    return cudaGetLastError();
}

cudaError_t launch_check_constants(int n, const double* h, const double* m, const double* s0, const int8_t* kind,
                                   uint32_t* varies, cudaStream_t st)
{
    k_check_constants<<<nblk(n, 256), 256, 0, st>>>(n, h, m, s0, kind, varies);
    return cudaGetLastError();
}

cudaError_t launch_scalar_in(int prec, int n, const double* src, const int8_t* kind, void* dst, cudaStream_t st)
{
    if (prec == 64) k_scalar_in<double><<<nblk(n, 256), 256, 0, st>>>(n, src, kind, (double*)dst);
    else k_scalar_in<float><<<nblk(n, 256), 256, 0, st>>>(n, src, kind, (float*)dst);
    return cudaGetLastError();
}

cudaError_t launch_scalar_out(int prec, int n, const void* src, const int32_t* id, double* dst, cudaStream_t st)
{
    if (prec == 64) k_scalar_out<double><<<nblk(n, 256), 256, 0, st>>>(n, (const double*)src, id, dst);
    else k_scalar_out<float><<<nblk(n, 256), 256, 0, st>>>(n, (const float*)src, id, dst);
    return cudaGetLastError();
}

}  // namespace sphtv
