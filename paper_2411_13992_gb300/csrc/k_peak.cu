// k_peak.cu -- fused multiply-add throughput of the GPU (sph_fma_peak), the
// measured denominator of the pair kernels' ALU roofline.
//
// Each thread runs 8 independent chains a <- a * b + c (b, c kernel
// arguments, so nothing folds at compile time); 8 chains per thread and a
// full SM of warps cover the FMA latency, so the launch is bound by the FMA
// issue rate alone.  With 0 < b < 1 every chain converges to c / (1 - b):
// no overflow, no subnormals.
#include <cuda_runtime.h>

#include "sphtv.h"

namespace sphtv {

constexpr int kPeakTPB = 256;
constexpr int kPeakChains = 8;

template <typename T>
__global__ void __launch_bounds__(kPeakTPB) k_fma_peak(int iters, T b, T c, T* __restrict__ sink)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    T a[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) a[k] = (T)(t & 15) * (T)0.0625 + (T)k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s += a[k];
    sink[t] = s;
}

}  // namespace sphtv

extern "C" SPH_API sph_status sph_fma_peak(int32_t precision, int32_t blocks, int32_t iters, void* sink,
                                           void* stream, double* flops)
{
    if ((precision != 32 && precision != 64) || blocks < 1 || iters < 1 || !sink || !flops) return SPH_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == 32)
        sphtv::k_fma_peak<float><<<blocks, sphtv::kPeakTPB, 0, s>>>(iters, 0.999f, 1e-3f, (float*)sink);
    else
        sphtv::k_fma_peak<double><<<blocks, sphtv::kPeakTPB, 0, s>>>(iters, 0.999, 1e-3, (double*)sink);
    if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
    *flops = 2.0 * sphtv::kPeakChains * (double)blocks * sphtv::kPeakTPB * (double)iters;
    return SPH_OK;
}
