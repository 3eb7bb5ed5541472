// launch.h -- internal (C++) launchers of the libsphtv kernels.  Each takes
// the precision (32 or 64) and dimension (2 or 3) at run time and picks the
// template instantiation.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace sphtv {

// Forward values of one step kept for the adjoint (device pointers).
struct TapeView {
    const int32_t* id;
    const int8_t* kind;
    const double* x;
    const double* h;
    const double* m;
    const double* s0;
    const void* vr;
    const void* R;
    const int32_t* start;
    const float4* pos4;
    const int32_t* cell;
    const double* dt;
    const uint32_t* nbl;   // FP32 form: the step's force-neighbour list (transposed, nbl_capacity rows)
    const int32_t* nbc;    // and its counts
};

// Adjoint buffers: cotangents in the caller's order ([3][n] FP64) and
// per-step scratch in the sorted order.
struct AdjView {
    double *xc, *vc, *ac, *drc;
    void *AR, *xbp, *vbp, *sigb;   // AR: per particle {Abar, Rbar} (k_adjoint.cu's record layout)
    double* partials;
    double* eta;
};

// k_cells.cu
cudaError_t launch_kick_drift_key(int prec, int dim, int n, void* S, const double* dt, int drift, const Grid& G,
                                  int32_t* key, int32_t* count, uint32_t* err, cudaStream_t st);
size_t scan_temp_elems(int n);
cudaError_t launch_exclusive_scan(const int32_t* in, int32_t* out, int n, int32_t* tmp, cudaStream_t st,
                                  int64_t* launches);
// The sort's scan without its last pass (see k_cells.cu): prefix within
// tiles, *tile_off the tiles' offsets (null for one tile).
cudaError_t launch_scan_tiles(const int32_t* count, int32_t* prefix, int n, int32_t* tmp, cudaStream_t st,
                              int64_t* launches, const int32_t** tile_off);
// nbin sort bins (cells, or sub-cells when shift > 0) whose starts are
// prefix + tile_off: scatter by the counts (left at zero), order each bin by
// id, write the bins' starts into start[nbin + 1] and, with shift > 0, the
// cells' starts into cell_start.
cudaError_t launch_scatter_order(int n, int nbin, const int32_t* key, const int32_t* prefix, const int32_t* tile_off,
                                 int32_t* count, int32_t* perm_tmp, const int32_t* id, int32_t* perm, int32_t* start,
                                 int shift, int32_t* cell_start, cudaStream_t st, int64_t* launches);
cudaError_t launch_permute(int prec, int dim, int n, const int32_t* perm, void* src, void* dst, const int32_t* key,
                           const Grid& G, float4* pos4, int32_t* cell, float* mf, int uniform_h, int carry_ad,
                           cudaStream_t st, const uint32_t* varies, float4* pos4c = nullptr);

// k_pair.cu (FP64 form; FP32 calls are forwarded to k_pair32.cu)
int pair_threads(int prec, int n, int sms);
int pair_blocks(int prec, int n, int sms);
// FP64 form: nbl / nbc may be null (no list); with them the density pass
// writes the neighbour list the dual-criteria integrator uses.
cudaError_t launch_density(int prec, int dim, int n, void* S, const int32_t* start, const Grid& G, const void* K,
                           void* vr, const float4* pos4, const int32_t* cell_of, uint32_t* nbl, int32_t* nbc,
                           cudaStream_t st, double* vol = nullptr, const float4* pos4c = nullptr, int tiles = 0);
cudaError_t launch_forces(int prec, int dim, int n, void* S, const int32_t* start, const Grid& G, const void* K,
                          const float* mf, const void* vr, const float4* pos4, const int32_t* cell_of,
                          const uint32_t* nbl, const int32_t* nbc, const double* dt, int kick_on, int write_ad,
                          void* Rout, void* chi, double* partials, cudaStream_t st, const double* vol = nullptr);

// k_pair32.cu
int nbl_capacity(int dim);
// tiles: at uniform resolution, the pass on cell-blocked shared-memory tiles
// (same results bit for bit as the row walk over global memory, tiles = 0)
cudaError_t launch_density32(int dim, int n, void* S, const int32_t* start, const Grid& G, const void* K, void* vr,
                             const float4* pos4, const int32_t* cell_of, uint32_t* nbl, int32_t* nbc,
                             cudaStream_t st, const float4* pos4c, int tiles = 0);
cudaError_t launch_forces32(int dim, int n, void* S, const int32_t* start, const Grid& G, const void* K,
                            const float* mf, const void* vr, const float4* pos4, const int32_t* cell_of,
                            const uint32_t* nbl, const int32_t* nbc, const double* dt, int kick_on, int write_ad,
                            void* Rout, void* chi, double* partials, cudaStream_t st);
cudaError_t launch_diag_only(int prec, int dim, int n, void* S, double* partials, int sms, cudaStream_t st);
int reduce_rows_blocks();
// First level of the fixed-order reduction of per-block partials: returns the
// number of rows written (0: too few partials, reduce them directly).
int launch_reduce_rows(int nblocks, const double* partials, double* rows, cudaStream_t st);
cudaError_t launch_finalize(int nblocks, const double* partials, double* rows, const sph_params& P, double* diag,
                            double* dt, int count_step, cudaStream_t st);

// k_io.cu
cudaError_t launch_vec_in(int prec, int dim, int n, const double* src3, void* dst, cudaStream_t st);
cudaError_t launch_vec_out(int prec, int dim, int n, const void* src, const int32_t* id, double* dst3,
                           cudaStream_t st);
cudaError_t launch_walls_velocity(int prec, int dim, int n, const int8_t* kind, const double* vw3, void* v,
                                  cudaStream_t st);
cudaError_t launch_init_ids(int n, int32_t* id, cudaStream_t st);
cudaError_t launch_sigma0(int dim, int n, const double* h, const double* m, double rho0, double* s0,
                          cudaStream_t st);
// Output by gathering (coalesced writes in the caller's order): pos from
// launch_inverse_perm of the sorted ids.
cudaError_t launch_inverse_perm(int n, const int32_t* id, int32_t* pos, cudaStream_t st);
cudaError_t launch_vec_out_gather(int prec, int dim, int n, const void* src, const int32_t* pos, double* dst3,
                                  cudaStream_t st);
cudaError_t launch_rho_out_gather(int prec, int n, const void* vr, const int8_t* kind, const int32_t* pos,
                                  double rho0, double* dst, cudaStream_t st);
cudaError_t launch_rho_out(int prec, int n, const void* vr, const int8_t* kind, const int32_t* id, double rho0,
                           double* dst, cudaStream_t st);
cudaError_t launch_check_input(int n, const double* h, const double* m, double h_min, double h_max, uint32_t* err,
                               cudaStream_t st);
cudaError_t launch_scalar_out(int prec, int n, const void* src, const int32_t* id, double* dst, cudaStream_t st);
cudaError_t launch_check_constants(int n, const double* h, const double* m, const double* s0, const int8_t* kind,
                                   uint32_t* varies, cudaStream_t st);
cudaError_t launch_scalar_in(int prec, int n, const double* src, const int8_t* kind, void* dst, cudaStream_t st);

// k_dual.cu (dual-criteria time stepping).  Device pointers of one context;
// S points at the StateSet<Real> of the current (sorted) copy.
struct DualArgs {
    int n, cap;
    const void* S;
    void* vr;
    float4* pos4;
    const int32_t* cell_of;
    const float* mf;
    const uint32_t* nbl;
    const int32_t* nbc;
    void* anu;
    void* R;
    void* chi;
    double* du;
    double* partials;
    double* rows;
    uint32_t* err;
};
int dual_pair_blocks(int prec, int n, int sms);
cudaError_t launch_dual_begin(const sph_params& P, const double* diag, double* du, cudaStream_t st);
cudaError_t launch_dual_advect(int prec, int dim, const DualArgs& a, const Grid& G, const void* K, cudaStream_t st);
cudaError_t launch_dual_substep(int prec, int dim, const DualArgs& a, const Grid& G, const void* K,
                                const sph_params& P, double* diag, double* dt_ptr, cudaStream_t st,
                                int64_t* launches);
cudaError_t launch_dual_complete(int prec, const DualArgs& a, cudaStream_t st);

// k_adjoint.cu
int adj_pair_blocks(int n);
cudaError_t launch_adjoint_step(int prec, int dim, int n, const TapeView& V, const Grid& G, const void* K,
                                const AdjView& A, int step_mode, cudaStream_t st);
cudaError_t launch_aos_to_soa(int n, const double* src3, double* dst, cudaStream_t st);
cudaError_t launch_soa_to_aos(int n, const double* src, double* dst3, cudaStream_t st);

}  // namespace sphtv
