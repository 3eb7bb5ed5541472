// pair_walk.cuh -- candidate walks over the 5^D cells around a particle's
// cell, on cell-relative FP32 positions (pos4 = {offset from the cell
// origin, m or h}; at uniform resolution the FP32 density pass walks a copy
// with the bits of the cell index in w).  Both visit the candidates in the
// same order: cells by (dz, dy, dx) ascending (periodic images in the order
// of the stencil step), particles by index within a cell.  Used by the FP32
// pair passes and, as a prefilter in front of the exact FP64 test, by the
// FP64 density pass.
#pragma once

#include "common.cuh"

namespace sphtv {

// Visit every candidate of the (2R+1)^D cells around cell_i (cell-relative
// FP32 positions plus the exact shift of the neighbour cell): f(j, code, pj,
// r2, rx, ry, rz) with code = stencil index of the neighbour cell.  Lanes of
// a warp whose particles share a cell read the same j at the same time, so
// the loads of pos4 are warp broadcasts.
template <int DIM, typename F>
__device__ __forceinline__ void for_candidates(const float* oi, int cell_i, const Grid& G,
                                               const int32_t* __restrict__ start,
                                               const float4* __restrict__ pos4, F& f)
{
    int c[3];
    cell_decode(G, cell_i, c);
    constexpr int R = kStencilR, zr = DIM == 3 ? R : 0;
    for (int dz = -zr; dz <= zr; ++dz) {
        int cz = DIM == 3 ? cell_step(G, c[2], dz, 2) : 0;
        if (cz < 0) continue;
        const float shz = -(float)dz * G.edgef[2];
        for (int dy = -R; dy <= R; ++dy) {
            int cy = cell_step(G, c[1], dy, 1);
            if (cy < 0) continue;
            const float shy = -(float)dy * G.edgef[1];
            const int row = G.nc[0] * (cy + G.nc[1] * cz);
            for (int dx = -R; dx <= R; ++dx) {
                int cx = cell_step(G, c[0], dx, 0);
                if (cx < 0) continue;
                const float shx = -(float)dx * G.edgef[0];
                const uint32_t code = (uint32_t)((dx + R) + kSide * (dy + R) + kSide * kSide * (dz + R));
                const int cell = cx + row;
                const int j1 = start[cell + 1];
                for (int j = start[cell]; j < j1; ++j) {
                    const float4 pj = pos4[j];
                    const float rx = (oi[0] - pj.x) + shx;
                    const float ry = (oi[1] - pj.y) + shy;
                    float r2 = rx * rx + ry * ry;
                    float rz = 0.f;
                    if (DIM == 3) {
                        rz = (oi[2] - pj.z) + shz;
                        r2 += rz * rz;
                    }
                    f(j, code, pj, r2, rx, ry, rz);
                }
            }
        }
    }
}

// The same visit as for_candidates, walked row by row and clipped to the
// particle's reach.  For each (dy, dz) row the cells are contiguous in the
// cell order, so the row is one run of particles (two runs across a periodic
// x boundary).  The x shift and stencil code of a candidate come from its own
// cell index (cell_of[j] - k_r = dx for every j of run r), so the walk has no
// inner loop over the cell boundaries of a run.  TWO: two candidates per
// iteration, their loads issued together (the FP32 density pass; the FP64
// pass, whose visit is larger, runs one at a time to stay within its
// registers).
// A row whose nearest y-z distance to particle i exceeds the reach (the
// largest support radius of any pair of i) is skipped, and the x extent of a
// row is cut to the cells within the remaining half-chord; every margin is
// 1e-3 of a cell edge, far above FP32 rounding, so every candidate that the
// full stencil would accept is still visited, in the same order.  About 2/3
// of the 5^3 cells remain in 3-D.  When the sort refines the cells along x
// into 2^s sub-cells (G.sub_shift = s), the x extent is cut at sub-cell
// granularity (the runs' bounds from G.sub_start; the same floor at 2^s
// times the resolution, whose coarsening is the cell cut): a row run then
// starts and ends within a sub-cell of the half-chord's ends.  The runs are
// still contiguous in the sort order, and the accepted candidates and their
// order are those of the cell cut.  CELL_IN_W: the cell index of each
// candidate is read from the bits of pos4.w (the copy with the cell index
// that the permute writes at uniform resolution) instead of a separate load
// from cell_of.
template <int DIM, bool TWO = true, bool CELL_IN_W = false, typename F>
__device__ __forceinline__ void for_candidates_rows(const float* oi, float reach, int cell_i, const Grid& G,
                                                    const int32_t* __restrict__ start,
                                                    const int32_t* __restrict__ cell_of,
                                                    const float4* __restrict__ pos4, F& f)
{
    int c[3];
    cell_decode(G, cell_i, c);
    constexpr int R = kStencilR, zr = DIM == 3 ? R : 0;
    const int ncx = G.nc[0];
    const float ex = G.edgef[0], ey = G.edgef[1], ez = G.edgef[2];
    const float inv_ex = 1.f / ex;
    const float reach2 = reach * reach;
    // the x cut in sub-cells (s = 0: cells): nsx along a row, the stencil's
    // sub-cells -R 2^s .. (R + 1) 2^s - 1 around the first of cell c[0]
    const int sh = G.sub_shift;
    const int32_t* __restrict__ rstart = sh ? G.sub_start : start;
    const int nsx = ncx << sh;
    const float inv_exs = inv_ex * (float)(1 << sh);   // exact: a power of two
    for (int dz = -zr; dz <= zr; ++dz) {
        int cz = DIM == 3 ? cell_step(G, c[2], dz, 2) : 0;
        if (cz < 0) continue;
        float rz = 0.f;
        if (DIM == 3) {
            rz = dz > 0 ? dz * ez - oi[2] : (dz < 0 ? oi[2] + (-dz - 1) * ez : 0.f);
            rz = fmaxf(rz - 1e-3f * ez, 0.f);
        }
        const float wz2 = reach2 - rz * rz;
        if (wz2 <= 0.f) continue;
        const float shz = -(float)dz * ez;
        for (int dy = -R; dy <= R; ++dy) {
            int cy = cell_step(G, c[1], dy, 1);
            if (cy < 0) continue;
            float ry = dy > 0 ? dy * ey - oi[1] : (dy < 0 ? oi[1] + (-dy - 1) * ey : 0.f);
            ry = fmaxf(ry - 1e-3f * ey, 0.f);
            const float w2 = wz2 - ry * ry;
            if (w2 <= 0.f) continue;
            const float w = sqrt_approx(w2) + 1e-3f * ex;
            const int slo = max(__float2int_rd((oi[0] - w) * inv_exs), -(R << sh));
            const int shi = min(__float2int_rd((oi[0] + w) * inv_exs), ((R + 1) << sh) - 1);
            if (slo > shi) continue;
            // runs along x: first sub-cell (x index along the row), number of
            // sub-cells, x step of the cell of the first sub-cell (>> is a floor
            // division); a periodic window (at most 5 <= ncx cells) wraps once at most
            int rc0[2], rn[2], rdx[2], nrun;
            const int a = (c[0] << sh) + slo, b = (c[0] << sh) + shi;
            if (!G.periodic[0]) {
                const int a0 = max(a, 0), b0 = min(b, nsx - 1);
                rc0[0] = a0; rn[0] = b0 - a0 + 1; rdx[0] = (a0 >> sh) - c[0]; nrun = rn[0] > 0 ? 1 : 0;
            } else if (a >= 0 && b < nsx) {
                rc0[0] = a; rn[0] = b - a + 1; rdx[0] = slo >> sh; nrun = 1;
            } else if (a < 0) {
                rc0[0] = nsx + a; rn[0] = min(-a, b - a + 1); rdx[0] = slo >> sh;
                rc0[1] = 0; rn[1] = b + 1; rdx[1] = -c[0]; nrun = b >= 0 ? 2 : 1;
            } else if (a >= nsx) {
                rc0[0] = a - nsx; rn[0] = b - a + 1; rdx[0] = slo >> sh; nrun = 1;
            } else {
                rc0[0] = a; rn[0] = nsx - a; rdx[0] = slo >> sh;
                rc0[1] = 0; rn[1] = b - nsx + 1; rdx[1] = ncx - c[0]; nrun = 2;
            }
            const float shy = -(float)dy * ey;
            const int row = ncx * (cy + G.nc[1] * cz);
            const uint32_t code_row = (uint32_t)(R + kSide * (dy + R) + kSide * kSide * (dz + R));
            for (int r = 0; r < nrun; ++r) {
                const int bin = (row << sh) + rc0[r];
                const int kr = row + (rc0[r] >> sh) - rdx[r];   // dx of candidate j = cell_of[j] - kr
                const int jend = rstart[bin + rn[r]];
                auto one = [&](int j, const float4& pj, int dx) {
                    const float shx = -(float)dx * ex;
                    // x and y in packed FP32x2 arithmetic (o_i - o_j as fma(o_j, -1, o_i): one rounding)
                    const float2 rxy = __fadd2_rn(__ffma2_rn(make_float2(pj.x, pj.y), make_float2(-1.f, -1.f),
                                                             make_float2(oi[0], oi[1])),
                                                  make_float2(shx, shy));
                    const float2 q = __fmul2_rn(rxy, rxy);
                    float r2 = q.x + q.y;
                    float rz_ = 0.f;
                    if (DIM == 3) {
                        rz_ = (oi[2] - pj.z) + shz;
                        r2 = fmaf(rz_, rz_, r2);
                    }
                    f(j, code_row + (uint32_t)dx, pj, r2, rxy.x, rxy.y, rz_);
                };
                auto cell_at = [&](int j, const float4& pj) {
                    return CELL_IN_W ? __float_as_int(pj.w) : cell_of[j];
                };
                int j = rstart[bin];
                for (; TWO && j + 1 < jend; j += 2) {
                    const float4 p0 = pos4[j], p1 = pos4[j + 1];
                    const int d0 = cell_at(j, p0) - kr, d1 = cell_at(j + 1, p1) - kr;
                    one(j, p0, d0);
                    one(j + 1, p1, d1);
                }
                for (; j < jend; ++j) {
                    const float4 pj = pos4[j];
                    one(j, pj, cell_at(j, pj) - kr);
                }
            }
        }
    }
}

}  // namespace sphtv
