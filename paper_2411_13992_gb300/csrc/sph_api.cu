// sph_api.cu -- host implementation of the libsphtv C ABI (include/sphtv.h).
//
// The context is a small host object.  Every device buffer is carved out of
// the caller's workspace; nothing here allocates device memory (the CUDA
// graph replay of sph_step adds a library-owned stream, two events and the
// graphs, which are driver objects).  Work is enqueued on the context's
// stream (graph replays on the library stream, ordered by events); the host
// waits in sph_sync, sph_get_diag, sph_get_state / sph_get_density_rate with
// host destinations, sph_set_dt, and once per advection step of the
// dual-criteria integrator.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "sphtv.h"

using namespace sphtv;

struct SetPtrs {
    StateSet<double> d;
    StateSet<float> f;
};

// One step's forward values kept for the adjoint.
struct TapeSlot {
    int32_t* id;
    int8_t* kind;
    double* x;
    double *h, *m, *s0;
    void* vr;
    void* R;
    int32_t* start;
    float4* pos4;
    int32_t* cell;
    double* dt;
    uint32_t* nbl;      // FP32 form: the step's force-neighbour list (the density pass's, transposed)
    int32_t* nbc;       // and its counts
};

struct sph_ctx {
    sph_params P;
    int64_t n;
    int dim, prec;
    cudaStream_t st;
    Grid G;
    Consts<double> K64;
    Consts<float> K32;
    SetPtrs set[2];
    int cur;
    // the sort: keys, permutations, bin counts (zero between sorts), the
    // scan's within-tile prefixes, the cells' starts and its scratch
    int32_t *key, *perm_tmp, *perm, *count, *prefix, *start, *scan_tmp;
    int32_t* sub_start;  // the sort's sub-cell starts (x_subcells > 1), else null
    int count_zero;      // count[] is known to be all zero (a complete sort ran since it was cleared)
    void* vr;
    float4* pos4;
    float4* pos4c;      // FP32 form, uniform h: pos4 with the cell index bits in w
    int32_t* cell;
    float* mf;
    uint32_t* nbl;      // neighbour lists of the density pass [cap][n], transposed
    int32_t* nbc;       // neighbour count per particle (with nbl)
    double* vol;        // FP64 form: V = m/rho per particle, written by the density pass for the force pass
    void* anu;          // dual integrator: viscous acceleration held for an advection step
    double* du;         // dual integrator: device state (DU_*)
    int dual_est;       // dual integrator: substeps to launch before the first check
    int density_only;   // sph_density_noalloc's view: no neighbour lists
    // CUDA graph replay of kick-drift-kick steps (params.graphs): two steps
    // per graph, one graph per parity of the ping-pong state sets
    cudaStream_t gst;           // library-owned stream of the replays
    cudaEvent_t gev[2];         // context stream -> gst, gst -> context stream
    cudaGraphExec_t gexec[2];
    int gstate[2];              // 0 not captured, 1 ready, -1 capture failed (launch directly)
    int64_t glaunches[2];       // kernels in one replay
    // the adjoint's segment (forward replay recording the tape, then the
    // reverse sweep) for one segment length, captured on first use
    cudaGraphExec_t aexec;
    int astate;                 // as gstate
    int asteps, acur0, acur1;   // segment length; state-set parity at its start and end
    int64_t alaunches;
    void* R;
    void* chi;
    double* partials;
    double* rows;        // first-level reduction of the partials
    double* diag;
    double* dt;
    uint32_t* err;          // [0] the sticky device error word; [1] nonzero when the particles' h, m,
                            // sigma0 or kind vary (else the sort leaves these arrays where they are)
    double* stage;
    int have_state, have_cells, ad_given;
    // kick-drift-kick, built with a and dr given: the state is still in the
    // caller's order, with no cell list and no densities; the next step
    // sorts it (its kick and drift need neither), sph_get_state(rho) sorts
    // it and runs the density pass first
    int cells_pending;
    int64_t launches;
    double host_dt;
    // adjoint (params.adjoint_steps > 0): tape slots, the per-particle
    // constants in the caller's order, cotangents and scratch
    TapeSlot* tape;
    double *orig_h, *orig_m, *orig_s0;
    double* orig_vw;      // [n][3] prescribed wall velocities
    int8_t* orig_kind;
    AdjView adj;
    // per-kernel timing (sph_profile_begin / sph_profile_end)
    std::vector<cudaEvent_t>* prof_ev;   // [step][class][begin, end]
    std::vector<int>* prof_used;         // [step][class] 0/1
    int prof_max, prof_step;
};

namespace {

constexpr size_t kAlign = 256;
// Largest cell grid (product over the axes) a context accepts: cell indices
// and the scan of the cell counts are int.
constexpr int64_t kMaxCells = (int64_t)1 << 30;

struct Carver {
    char* base;
    size_t off;
    template <typename T>
    T* take(size_t count)
    {
        off = (off + kAlign - 1) & ~(kAlign - 1);
        T* p = base ? (T*)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

sph_status check_params(const sph_params* p, int64_t n)
{
    if (!p || n < 1 || n > ((int64_t)1 << 25)) return SPH_ERR_ARG;   // list entries hold j in 25 bits
    if (p->dim != 2 && p->dim != 3) return SPH_ERR_ARG;
    if (p->precision != 32 && p->precision != 64) return SPH_ERR_ARG;
    if (!(p->rho0 > 0) || !(p->c0 > 0) || !(p->eta >= 0)) return SPH_ERR_ARG;
    if (!(p->h_min > 0) || !(p->h_max >= p->h_min)) return SPH_ERR_ARG;
    if (p->tv_mode < 0 || p->tv_mode > 3 || p->tv_h < 0 || p->tv_h > 1 || p->h_pair < 0 || p->h_pair > 1)
        return SPH_ERR_ARG;
    if (!(p->fixed_dt >= 0) || !(p->cfl_ad > 0) || !(p->cfl_ac > 0)) return SPH_ERR_ARG;
    if (p->adjoint_steps < 0 || p->adjoint_steps > 100000) return SPH_ERR_ARG;
    if (p->integrator != SPH_INT_KDK && p->integrator != SPH_INT_DUAL) return SPH_ERR_ARG;
    if (p->graphs != 0 && p->graphs != 1) return SPH_ERR_ARG;
    if (p->pair_tiles < 0 || p->pair_tiles > 3) return SPH_ERR_ARG;
    if (p->x_subcells != 0 && p->x_subcells != 1 && p->x_subcells != 2 && p->x_subcells != 4) return SPH_ERR_ARG;
    if (p->body_force != 0 && p->body_force != 1) return SPH_ERR_ARG;
    if (!(p->fringe_lambda >= 0.0) || !std::isfinite(p->fringe_lambda)) return SPH_ERR_ARG;
    if (p->fringe_lambda > 0.0) {
        if (p->integrator != SPH_INT_KDK) return SPH_ERR_ARG;     // the forcing acts in the kick-drift-kick force pass
        for (int k = 0; k < 4; ++k)
            if (!std::isfinite(p->fringe_x[k])) return SPH_ERR_ARG;
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(p->fringe_u[d])) return SPH_ERR_ARG;
        if (!(p->fringe_x[2] > 0.0) || !(p->fringe_x[3] > 0.0)) return SPH_ERR_ARG;
    }
    if (p->integrator == SPH_INT_DUAL && (p->fixed_dt != 0.0 || p->adjoint_steps != 0)) return SPH_ERR_ARG;
    // the cell grid: each axis and the product of all axes bounded, so that
    // cell indices, the count and start arrays and the workspace size stay
    // within int (the product is taken in int64 before anything is sized)
    int64_t ncell = 1;
    for (int d = 0; d < p->dim; ++d) {
        if (!(p->L[d] > 0) || !std::isfinite(p->lo[d]) || !std::isfinite(p->L[d])) return SPH_ERR_ARG;
        double nc = std::floor(p->L[d] * kStencilR / (2.0 * p->h_max));
        if (p->periodic[d] && nc < 2 * kStencilR + 1) return SPH_ERR_ARG;
        if (!(nc <= (double)(1 << 20))) return SPH_ERR_ARG;
        ncell *= nc < 1 ? 1 : (int64_t)nc;
        if (ncell > kMaxCells) return SPH_ERR_ARG;
    }
    return SPH_OK;
}

// Streaming multiprocessors of the current device (152 on GB300 if the
// query fails or there is no device, as in a workspace query on a host
// without one; the count only sizes grids).
int device_sms()
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        v <= 0) {
        cudaGetLastError();
        return 152;
    }
    return v;
}

// log2 of the sub-cells per cell of the sort: the requested count (1, 2 or
// 4), reduced while the cells times the sub-cells exceed the bin bound.
int sub_shift_for(int64_t ncell, int x_subcells)
{
    int s = x_subcells == 4 ? 2 : (x_subcells == 2 ? 1 : 0);
    while (s > 0 && (ncell << s) > kMaxCells) --s;
    return s;
}

Grid make_grid(const sph_params* p)
{
    Grid G;
    G.R = kStencilR;
    int64_t ncell = 1;
    for (int d = 0; d < 3; ++d) {
        if (d < p->dim) {
            int nc = (int)std::floor(p->L[d] * kStencilR / (2.0 * p->h_max));
            if (nc < 1) nc = 1;
            G.nc[d] = nc;
            G.periodic[d] = p->periodic[d] ? 1 : 0;
            G.lo[d] = p->lo[d];
            G.L[d] = p->L[d];
            G.hi[d] = p->lo[d] + p->L[d];
            G.half_L[d] = 0.5 * p->L[d];
            G.edge[d] = p->L[d] / nc;
            G.inv_edge[d] = (double)nc / p->L[d];
        } else {
            G.nc[d] = 1;
            G.periodic[d] = 0;
            G.lo[d] = 0.0;
            G.L[d] = 1.0;
            G.hi[d] = 1.0;
            G.half_L[d] = 0.5;
            G.edge[d] = 1.0;
            G.inv_edge[d] = 1.0;
        }
        G.edgef[d] = (float)G.edge[d];
        ncell *= G.nc[d];
    }
    G.ncell = (int)ncell;
    G.sms = device_sms();
    G.sub_shift = sub_shift_for(ncell, p->x_subcells);
    G.inv_edge_sub0 = G.inv_edge[0] * (double)(1 << G.sub_shift);
    G.sub_start = nullptr;   // set when the workspace is laid out
    return G;
}

// Sort bins: the cells, or their sub-cells along x.
static inline size_t sort_bins(const Grid& G) { return (size_t)G.ncell << G.sub_shift; }

// The grid without the sub-cell refinement (for walks over stored cell
// starts, such as the adjoint's tape).
static inline Grid cells_only(Grid G)
{
    G.sub_shift = 0;
    G.inv_edge_sub0 = G.inv_edge[0];
    G.sub_start = nullptr;
    return G;
}

template <typename Real>
Consts<Real> make_consts(const sph_params* p)
{
    Consts<Real> K;
    double c2 = p->c0 * p->c0;
    K.rho0 = (Real)p->rho0;
    K.c = (Real)p->c0;
    K.c2 = (Real)c2;
    K.eta = (Real)p->eta;
    K.two_eta = (Real)(2.0 * p->eta);
    K.beta_slope = (Real)p->riemann_eta;
    K.inv_c = (Real)(1.0 / p->c0);
    for (int d = 0; d < 3; ++d) K.g[d] = (Real)p->g[d];
    K.h_min = (Real)p->h_min;
    K.tv_xi = (Real)p->tv_xi;
    K.tv_C = (Real)p->tv_C;
    K.tv_thresh = (Real)p->tv_thresh;
    K.tv_mode = p->tv_mode;
    K.tv_h_particle = p->tv_h == SPH_TVH_PARTICLE;
    K.h_pair_max = p->h_pair == SPH_HPAIR_MAX;
    K.kahan = p->kahan;
    K.uniform_h = p->h_min == p->h_max;
    K.body_force = p->body_force;
    K.fr_on = p->fringe_lambda > 0.0;
    K.fr_lambda = (Real)p->fringe_lambda;
    for (int d = 0; d < 3; ++d) K.fr_u[d] = (Real)p->fringe_u[d];
    for (int k = 0; k < 4; ++k) K.fr_x[k] = (Real)p->fringe_x[k];
    K.h_u = (Real)p->h_max;
    K.inv_h_u = (Real)(1.0 / p->h_max);
    K.four_h2_u = (Real)(4.0 * p->h_max * p->h_max);
    {
        // W'(r)/r = -5 a_D h^-(D+2) t^3 with a_D = 7/(4 pi) (2-D), 21/(16 pi) (3-D)
        const double pi = 3.14159265358979323846;
        const double norm = p->dim == 2 ? 7.0 / (4.0 * pi) : 21.0 / (16.0 * pi);
        K.dwr_coef_u = (Real)(-5.0 * norm * std::pow(1.0 / p->h_max, p->dim + 2));
    }
    return K;
}

// Lay the buffers out in the workspace (base == nullptr: only measure).
size_t carve(sph_ctx* c, char* base)
{
    Carver W{base, 0};
    const size_t n = (size_t)c->n;
    const int D = c->dim;
    const size_t rs = c->prec == 64 ? 8 : 4;
    const size_t nc1 = (size_t)c->G.ncell + 1;
    const bool dual = c->P.integrator == SPH_INT_DUAL;
    for (int s = 0; s < 2; ++s) {
        double* x = W.take<double>(D * n);
        char* v = W.take<char>(D * n * rs);
        // (the density-only view of sph_density_noalloc needs no a, dr, R, chi)
        char* a = c->density_only ? nullptr : W.take<char>(D * n * rs);
        char* dr = c->density_only ? nullptr : W.take<char>(D * n * rs);
        char* drho = dual ? W.take<char>(n * rs) : nullptr;
        double* h = W.take<double>(n);
        double* m = W.take<double>(n);
        double* s0 = W.take<double>(n);
        int32_t* id = W.take<int32_t>(n);
        int8_t* kind = W.take<int8_t>(n);
        c->set[s].d = StateSet<double>{x, (double*)v, (double*)a, (double*)dr, (double*)drho, h, m, s0, id, kind};
        c->set[s].f = StateSet<float>{x, (float*)v, (float*)a, (float*)dr, (float*)drho, h, m, s0, id, kind};
    }
    c->key = W.take<int32_t>(n);
    c->perm_tmp = W.take<int32_t>(n);
    c->perm = W.take<int32_t>(n);
    const size_t nb1 = sort_bins(c->G) + 1;
    c->count = W.take<int32_t>(nb1);
    c->prefix = W.take<int32_t>(nb1);
    c->start = W.take<int32_t>(nc1);
    c->sub_start = c->G.sub_shift ? W.take<int32_t>(nb1) : nullptr;
    c->G.sub_start = c->sub_start;
    c->scan_tmp = W.take<int32_t>(scan_temp_elems((int)nb1));
    c->vr = W.take<char>(n * 4 * rs);
    c->pos4 = W.take<float4>(n);     // both forms: FP32 cell-relative positions for the candidate walks
    c->pos4c = c->prec == 32 && c->P.h_min == c->P.h_max ? W.take<float4>(n) : nullptr;
    c->cell = W.take<int32_t>(n);
    c->mf = W.take<float>(n);
    const bool lists = !c->density_only;   // both forms: the force pass walks the density pass's list
    c->nbl = lists ? W.take<uint32_t>((size_t)nbl_capacity(D) * n) : nullptr;
    c->nbc = lists ? W.take<int32_t>(n) : nullptr;
    c->vol = lists && c->prec == 64 ? W.take<double>(n) : nullptr;
    c->anu = dual ? W.take<char>(D * n * rs) : nullptr;
    c->du = dual ? W.take<double>(DU_COUNT) : nullptr;
    c->R = c->density_only ? nullptr : W.take<char>(D * n * rs);
    c->chi = c->density_only ? nullptr : W.take<char>(n * rs);
    // one partials row per block of a pair pass; blocks are never smaller than a warp
    c->partials = W.take<double>(((size_t)n + 31) / 32 * kNPart);
    c->rows = W.take<double>((size_t)reduce_rows_blocks() * kNPart);
    c->diag = W.take<double>(DG_COUNT);
    c->dt = W.take<double>(1);
    c->err = W.take<uint32_t>(4);
    c->stage = W.take<double>(3 * n);
    const int K = c->P.adjoint_steps;
    if (K > 0) {
        c->orig_h = W.take<double>(n);
        c->orig_m = W.take<double>(n);
        c->orig_s0 = W.take<double>(n);
        c->orig_vw = W.take<double>(3 * n);
        c->orig_kind = W.take<int8_t>(n);
        for (int t = 0; t < K; ++t) {
            TapeSlot sl;
            sl.id = W.take<int32_t>(n);
            sl.kind = W.take<int8_t>(n);
            sl.x = W.take<double>(D * n);
            sl.h = W.take<double>(n);
            sl.m = W.take<double>(n);
            sl.s0 = W.take<double>(n);
            sl.vr = W.take<char>(n * 4 * rs);
            sl.R = W.take<char>(D * n * rs);
            sl.start = W.take<int32_t>(nc1);
            sl.pos4 = c->prec == 32 ? W.take<float4>(n) : nullptr;
            sl.cell = c->prec == 32 ? W.take<int32_t>(n) : nullptr;
            sl.dt = W.take<double>(1);
            sl.nbl = c->prec == 32 ? W.take<uint32_t>((size_t)nbl_capacity(D) * n) : nullptr;
            sl.nbc = c->prec == 32 ? W.take<int32_t>(n) : nullptr;
            if (base && c->tape) c->tape[t] = sl;
        }
        AdjView& A = c->adj;
        A.xc = W.take<double>(3 * n);
        A.vc = W.take<double>(3 * n);
        A.ac = W.take<double>(3 * n);
        A.drc = W.take<double>(3 * n);
        A.AR = W.take<char>((size_t)(D == 3 ? 8 : 4) * n * rs);   // {Abar, Rbar} records (k_adjoint.cu)
        A.xbp = W.take<char>(D * n * rs);
        A.vbp = W.take<char>(D * n * rs);
        A.sigb = W.take<char>(n * rs);
        A.partials = W.take<double>((size_t)adj_pair_blocks((int)n) * kNPart);
        A.eta = W.take<double>(1);
    }
    return (W.off + kAlign - 1) & ~(kAlign - 1);
}

void* cur_set(sph_ctx* c) { return c->prec == 64 ? (void*)&c->set[c->cur].d : (void*)&c->set[c->cur].f; }
void* other_set(sph_ctx* c) { return c->prec == 64 ? (void*)&c->set[1 - c->cur].d : (void*)&c->set[1 - c->cur].f; }
const void* consts(sph_ctx* c) { return c->prec == 64 ? (const void*)&c->K64 : (const void*)&c->K32; }

#define SPH_CU(call)                                 \
    do {                                             \
        if ((call) != cudaSuccess) return SPH_ERR_CUDA; \
    } while (0)

// Event marks around a kernel class when a profile is open and the current
// step is within its range (the step index advances in sph_step).
inline cudaError_t prof_mark(sph_ctx* c, int cls, int end)
{
    if (!c->prof_ev || c->prof_step < 0 || c->prof_step >= c->prof_max) return cudaSuccess;
    size_t k = ((size_t)c->prof_step * SPH_K_NCLASS + cls);
    if (!end) (*c->prof_used)[k] = 1;
    return cudaEventRecord((*c->prof_ev)[2 * k + end], c->st);
}

#define SPH_MARK(cls, end) SPH_CU(prof_mark(c, cls, end))

#define SPH_TRY(call)                    \
    do {                                 \
        sph_status s_ = (call);          \
        if (s_ != SPH_OK) return s_;     \
    } while (0)

// Kick-drift (optional), cell keys, counting sort, permute.
sph_status run_sort(sph_ctx* c, int drift, int carry_ad)
{
    const int n = (int)c->n;
    const size_t nb1 = sort_bins(c->G) + 1;
    // the bins' starts: the sub-cells' (the cells' then follow from them) or the cells'
    int32_t* bin_start = c->G.sub_shift ? c->sub_start : c->start;
    SPH_MARK(SPH_K_KICKDRIFT, 0);
    // the scatter counts every bin back down to zero: clear only when a sort
    // did not complete since the counts were last known to be zero
    if (!c->count_zero) SPH_CU(cudaMemsetAsync(c->count, 0, nb1 * sizeof(int32_t), c->st));
    c->count_zero = 0;
    SPH_CU(launch_kick_drift_key(c->prec, c->dim, n, cur_set(c), c->dt, drift, c->G, c->key, c->count, c->err, c->st));
    ++c->launches;
    SPH_MARK(SPH_K_KICKDRIFT, 1);
    SPH_MARK(SPH_K_SCAN, 0);
    const int32_t* tile_off = nullptr;
    SPH_CU(launch_scan_tiles(c->count, c->prefix, (int)nb1, c->scan_tmp, c->st, &c->launches, &tile_off));
    SPH_MARK(SPH_K_SCAN, 1);
    const int32_t* id = c->prec == 64 ? c->set[c->cur].d.id : c->set[c->cur].f.id;
    SPH_MARK(SPH_K_ORDER, 0);
    SPH_CU(launch_scatter_order(n, (int)sort_bins(c->G), c->key, c->prefix, tile_off, c->count, c->perm_tmp, id,
                                c->perm, bin_start, c->G.sub_shift, c->start, c->st, &c->launches));
    c->count_zero = 1;
    SPH_MARK(SPH_K_ORDER, 1);
    SPH_MARK(SPH_K_PERMUTE, 0);
    SPH_CU(launch_permute(c->prec, c->dim, n, c->perm, cur_set(c), other_set(c), c->key, c->G, c->pos4, c->cell,
                          c->mf, c->K32.uniform_h, carry_ad, c->st, c->err + 1, c->pos4c));
    ++c->launches;
    SPH_MARK(SPH_K_PERMUTE, 1);
    c->cur = 1 - c->cur;
    return SPH_OK;
}

// Density, fused forces (+ closing kick), reductions and dt.  With
// pairs == 0 (a and dr supplied by the caller) only the density and the
// diagnostics run.
sph_status run_forces(sph_ctx* c, int kick_on, int pairs, int count_step)
{
    const int n = (int)c->n;
    if (!pairs) {
        SPH_CU(launch_density(c->prec, c->dim, n, cur_set(c), c->start, c->G, consts(c), c->vr, c->pos4, c->cell,
                              c->nbl, c->nbc, c->st, c->vol, c->pos4c, c->P.pair_tiles));
        SPH_CU(launch_diag_only(c->prec, c->dim, n, cur_set(c), c->partials, c->G.sms, c->st));
        SPH_CU(launch_finalize(pair_blocks(c->prec, n, c->G.sms), c->partials, c->rows, c->P, c->diag, c->dt,
                               count_step, c->st));
        c->launches += 3;
        return SPH_OK;
    }
    const int write_ad = 1;
    SPH_MARK(SPH_K_DENSITY, 0);
    SPH_CU(launch_density(c->prec, c->dim, n, cur_set(c), c->start, c->G, consts(c), c->vr, c->pos4, c->cell, c->nbl,
                          c->nbc, c->st, c->vol, c->pos4c, c->P.pair_tiles));
    SPH_MARK(SPH_K_DENSITY, 1);
    SPH_MARK(SPH_K_FORCES, 0);
    SPH_CU(launch_forces(c->prec, c->dim, n, cur_set(c), c->start, c->G, consts(c), c->mf, c->vr, c->pos4, c->cell,
                         c->nbl, c->nbc, c->dt, kick_on, write_ad, c->R, c->chi, c->partials, c->st,
                         c->vol));
    SPH_MARK(SPH_K_FORCES, 1);
    SPH_MARK(SPH_K_FINALIZE, 0);
    SPH_CU(launch_finalize(pair_blocks(c->prec, n, c->G.sms), c->partials, c->rows, c->P, c->diag, c->dt,
                           count_step, c->st));
    SPH_MARK(SPH_K_FINALIZE, 1);
    c->launches += 3;
    return SPH_OK;
}

DualArgs dual_args(sph_ctx* c)
{
    DualArgs a;
    a.n = (int)c->n;
    a.cap = nbl_capacity(c->dim);
    a.S = cur_set(c);
    a.vr = c->vr;
    a.pos4 = c->pos4;
    a.cell_of = c->cell;
    a.mf = c->mf;
    a.nbl = c->nbl;
    a.nbc = c->nbc;
    a.anu = c->anu;
    a.R = c->R;
    a.chi = c->chi;
    a.du = c->du;
    a.partials = c->partials;
    a.rows = c->rows;
    a.err = c->err;
    return a;
}

// One advection step of the dual-criteria integrator (Sec. 2.4): sort (wrap
// only), density pass with the frozen neighbour list, Dt_ad, the viscous
// force and the correction; then acoustic substeps until the device marks the
// advection step done.  Substeps are launched in batches; a batch may run
// past the end (the extra launches return at once) and the host reads the
// device state once per batch.
sph_status run_dual_step(sph_ctx* c)
{
    const int n = (int)c->n;
    SPH_TRY(run_sort(c, 2, 0));
    SPH_MARK(SPH_K_DENSITY, 0);
    SPH_CU(launch_density(c->prec, c->dim, n, cur_set(c), c->start, c->G, consts(c), c->vr, c->pos4, c->cell,
                          c->nbl, c->nbc, c->st, c->vol, c->pos4c, c->P.pair_tiles));
    SPH_MARK(SPH_K_DENSITY, 1);
    SPH_MARK(SPH_K_ADVECT, 0);
    SPH_CU(launch_dual_begin(c->P, c->diag, c->du, c->st));
    const DualArgs a = dual_args(c);
    SPH_CU(launch_dual_advect(c->prec, c->dim, a, c->G, consts(c), c->st));
    SPH_MARK(SPH_K_ADVECT, 1);
    c->launches += 3;
    double hb[DU_COUNT];
    if (c->dual_est <= 0) {
        SPH_CU(cudaMemcpyAsync(hb, c->du, sizeof(hb), cudaMemcpyDeviceToHost, c->st));
        SPH_CU(cudaStreamSynchronize(c->st));
        const double ratio = hb[DU_DT_AD] / hb[DU_DT];
        c->dual_est = std::isfinite(ratio) && ratio < 1.0e6 ? (int)std::ceil(ratio) + 1 : 2;
    }
    SPH_MARK(SPH_K_ACOUSTIC, 0);
    int batch = c->dual_est, taken = 0;
    constexpr int kMaxSubsteps = 1 << 20;
    for (;;) {
        for (int b = 0; b < batch; ++b)
            SPH_CU(launch_dual_substep(c->prec, c->dim, a, c->G, consts(c), c->P, c->diag, c->dt, c->st,
                                       &c->launches));
        taken += batch;
        SPH_CU(cudaMemcpyAsync(hb, c->du, sizeof(hb), cudaMemcpyDeviceToHost, c->st));
        SPH_CU(cudaStreamSynchronize(c->st));
        if (hb[DU_DONE] != 0.0) break;
        if (taken >= kMaxSubsteps) return SPH_ERR_NAN;   // the step sizes are not finite or vanish
        batch = 2;
    }
    SPH_CU(launch_dual_complete(c->prec, a, c->st));
    ++c->launches;
    SPH_MARK(SPH_K_ACOUSTIC, 1);
    c->dual_est = (int)hb[DU_K] + 1;
    return SPH_OK;
}

// Capture two kick-drift-kick steps starting from state-set parity par into
// a graph on the library stream.  Nothing runs during the capture (the sets
// and counters are left as they were); on any failure the context falls
// back to direct launches for that parity.
// The library stream of the replays and the two events that fence it
// against the context's stream; false if they cannot be created.
bool graph_stream(sph_ctx* c)
{
    if (c->gst) return true;
    if (cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking) != cudaSuccess) {
        c->gst = nullptr;
        cudaGetLastError();
        return false;
    }
    if (cudaEventCreateWithFlags(&c->gev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->gev[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamDestroy(c->gst);
        c->gst = nullptr;
        return false;
    }
    return true;
}

void graph_capture(sph_ctx* c, int par)
{
    c->gstate[par] = -1;
    if (!graph_stream(c)) return;
    cudaStream_t user = c->st;
    const int cur0 = c->cur;
    const int64_t l0 = c->launches;
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(c->gst, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        c->st = c->gst;
        for (int k = 0; k < 2 && ok; ++k) ok = run_sort(c, 1, 0) == SPH_OK && run_forces(c, 1, 1, 1) == SPH_OK;
        c->st = user;
        ok = cudaStreamEndCapture(c->gst, &g) == cudaSuccess && ok && g;
    }
    c->cur = cur0;
    c->glaunches[par] = c->launches - l0;
    c->launches = l0;
    if (ok && cudaGraphInstantiate(&c->gexec[par], g, 0) == cudaSuccess) c->gstate[par] = 1;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
}

void graph_release(sph_ctx* c)
{
    for (int par = 0; par < 2; ++par) {
        if (c->gstate[par] == 1) cudaGraphExecDestroy(c->gexec[par]);
        c->gstate[par] = 0;
    }
    if (c->astate == 1) cudaGraphExecDestroy(c->aexec);
    c->astate = 0;
    c->asteps = 0;
}

// Launch a captured graph on the library stream, fenced against the
// context's stream on both sides.
sph_status graph_launch(sph_ctx* c, cudaGraphExec_t g, int times)
{
    SPH_CU(cudaEventRecord(c->gev[0], c->st));
    SPH_CU(cudaStreamWaitEvent(c->gst, c->gev[0], 0));
    for (int k = 0; k < times; ++k) SPH_CU(cudaGraphLaunch(g, c->gst));
    SPH_CU(cudaEventRecord(c->gev[1], c->gst));
    SPH_CU(cudaStreamWaitEvent(c->st, c->gev[1], 0));
    return SPH_OK;
}

bool is_host_ptr(const void* p)
{
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged;
}


// ------------------------------------------------------------------ adjoint

// Load a state (caller order) with the per-particle constants of the last
// sph_set_state.  a and dr may be NULL (then computed by the force pass).
// Address through which this device's kernels can reach p directly: p for
// memory of the current device (or managed memory), the mapped alias of
// page-locked host memory; nullptr otherwise (pageable host memory, another
// device), which then goes through the staging buffer by a copy.
void* device_view(const void* p)
{
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (attr.type == cudaMemoryTypeManaged) return const_cast<void*>(p);
    if (attr.type == cudaMemoryTypeDevice) return attr.device == dev ? const_cast<void*>(p) : nullptr;
    if (attr.type == cudaMemoryTypeHost && attr.devicePointer) return attr.devicePointer;
    return nullptr;
}

// [n][3] rows of src (host or device) into the per-component array dst of
// precision prec: read in place when the device can reach src (page-locked
// host memory streams across the host link inside the conversion kernel),
// else copied to the staging buffer first.
sph_status vec_in(sph_ctx* c, int prec, const double* src, void* dst)
{
    const size_t n = (size_t)c->n;
    const double* dv = (const double*)device_view(src);
    if (!dv) {
        SPH_CU(cudaMemcpyAsync(c->stage, src, 3 * n * sizeof(double), cudaMemcpyDefault, c->st));
        dv = c->stage;
    }
    SPH_CU(launch_vec_in(prec, c->dim, (int)n, dv, dst, c->st));
    ++c->launches;
    return SPH_OK;
}

// h, m, sigma0 and kind of state set 0 into state set 1: the sort leaves these
// arrays where they are when they do not vary over the particles, so both
// sets must hold them.
sph_status copy_constants(sph_ctx* c)
{
    const size_t n = (size_t)c->n;
    const StateSet<double>& A = c->set[0].d;
    const StateSet<double>& B = c->set[1].d;
    SPH_CU(cudaMemcpyAsync(B.h, A.h, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    SPH_CU(cudaMemcpyAsync(B.m, A.m, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    SPH_CU(cudaMemcpyAsync(B.s0, A.s0, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    SPH_CU(cudaMemcpyAsync(B.kind, A.kind, n, cudaMemcpyDeviceToDevice, c->st));
    return SPH_OK;
}

sph_status reload_state(sph_ctx* c, const double* x, const double* v, const double* a, const double* dr)
{
    const size_t n = (size_t)c->n;
    const size_t rs = c->prec == 64 ? 8 : 4;
    c->cur = 0;
    StateSet<double>& Sd = c->set[0].d;
    void* sv = c->prec == 64 ? (void*)c->set[0].d.v : (void*)c->set[0].f.v;
    void* sa = c->prec == 64 ? (void*)c->set[0].d.a : (void*)c->set[0].f.a;
    void* sdr = c->prec == 64 ? (void*)c->set[0].d.dr : (void*)c->set[0].f.dr;
    SPH_TRY(vec_in(c, 64, x, Sd.x));
    SPH_TRY(vec_in(c, c->prec, v, sv));
    if (a) {
        SPH_TRY(vec_in(c, c->prec, a, sa));
        SPH_TRY(vec_in(c, c->prec, dr, sdr));
    } else {
        SPH_CU(cudaMemsetAsync(sa, 0, c->dim * n * rs, c->st));
        SPH_CU(cudaMemsetAsync(sdr, 0, c->dim * n * rs, c->st));
    }
    SPH_CU(cudaMemcpyAsync(Sd.h, c->orig_h, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    SPH_CU(cudaMemcpyAsync(Sd.m, c->orig_m, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    SPH_CU(cudaMemcpyAsync(Sd.s0, c->orig_s0, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    SPH_CU(cudaMemcpyAsync(Sd.kind, c->orig_kind, n, cudaMemcpyDeviceToDevice, c->st));
    SPH_TRY(copy_constants(c));
    SPH_CU(launch_walls_velocity(c->prec, c->dim, (int)n, Sd.kind, c->orig_vw, sv, c->st));
    SPH_CU(launch_init_ids((int)n, Sd.id, c->st));
    c->launches += 2;
    c->have_state = 1;
    c->have_cells = 0;
    c->ad_given = a != nullptr;
    return SPH_OK;
}

// Copy the current step's forward values into tape slot t (dt is copied by
// the caller before the step runs).  list_in_slot: the step's density pass
// wrote its neighbour list into the slot's own list buffers (the FP32
// form's adjoint walks that list); otherwise the list is copied from the
// context's buffers.
sph_status save_tape(sph_ctx* c, int t, bool list_in_slot = false)
{
    const size_t n = (size_t)c->n;
    const size_t rs = c->prec == 64 ? 8 : 4;
    const size_t nc1 = (size_t)c->G.ncell + 1;
    const StateSet<double>& S = c->set[c->cur].d;
    TapeSlot& T = c->tape[t];
    SPH_CU(cudaMemcpyAsync(T.id, S.id, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->st));
    SPH_CU(cudaMemcpyAsync(T.kind, S.kind, n, cudaMemcpyDeviceToDevice, c->st));
    SPH_CU(cudaMemcpyAsync(T.x, S.x, c->dim * n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    SPH_CU(cudaMemcpyAsync(T.h, S.h, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    SPH_CU(cudaMemcpyAsync(T.m, S.m, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    SPH_CU(cudaMemcpyAsync(T.s0, S.s0, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    SPH_CU(cudaMemcpyAsync(T.vr, c->vr, n * 4 * rs, cudaMemcpyDeviceToDevice, c->st));
    SPH_CU(cudaMemcpyAsync(T.R, c->R, c->dim * n * rs, cudaMemcpyDeviceToDevice, c->st));
    SPH_CU(cudaMemcpyAsync(T.start, c->start, nc1 * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->st));
    if (c->prec == 32) {
        SPH_CU(cudaMemcpyAsync(T.pos4, c->pos4, n * sizeof(float4), cudaMemcpyDeviceToDevice, c->st));
        SPH_CU(cudaMemcpyAsync(T.cell, c->cell, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->st));
        if (!list_in_slot) {
            SPH_CU(cudaMemcpyAsync(T.nbl, c->nbl, (size_t)nbl_capacity(c->dim) * n * sizeof(uint32_t),
                                   cudaMemcpyDeviceToDevice, c->st));
            SPH_CU(cudaMemcpyAsync(T.nbc, c->nbc, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->st));
        }
    }
    return SPH_OK;
}

TapeView tape_view(const TapeSlot& T)
{
    return TapeView{T.id, T.kind, T.x, T.h, T.m, T.s0, T.vr, T.R, T.start, T.pos4, T.cell, T.dt, T.nbl, T.nbc};
}

// Caller [n][3] cotangents -> [3][n] FP64 (z row zeroed in 2-D), and back.
sph_status cot_in(sph_ctx* c, const double* src, double* dst)
{
    const size_t n = (size_t)c->n;
    SPH_CU(cudaMemcpyAsync(c->stage, src, 3 * n * sizeof(double), cudaMemcpyDefault, c->st));
    SPH_CU(launch_aos_to_soa((int)n, c->stage, dst, c->st));
    if (c->dim == 2) SPH_CU(cudaMemsetAsync(dst + 2 * n, 0, n * sizeof(double), c->st));
    ++c->launches;
    return SPH_OK;
}

sph_status cot_out(sph_ctx* c, const double* src, double* dst)
{
    const size_t n = (size_t)c->n;
    SPH_CU(launch_soa_to_aos((int)n, src, c->stage, c->st));
    SPH_CU(cudaMemcpyAsync(dst, c->stage, 3 * n * sizeof(double), cudaMemcpyDefault, c->st));
    ++c->launches;
    return SPH_OK;
}

// One segment of the adjoint after the cotangents are in: nsteps forward
// steps from the reloaded state that record the tape (with the step sizes
// taken), then the reverse sweep over them.  No host work between the
// launches, so the whole segment can be captured in one graph.
sph_status adjoint_segment(sph_ctx* c, int nsteps)
{
    for (int t = 0; t < nsteps; ++t) {
        SPH_CU(cudaMemcpyAsync(c->tape[t].dt, c->dt, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        SPH_TRY(run_sort(c, 1, 0));
        // FP32 form: the step's density pass writes its neighbour list
        // straight into the tape slot (no copy), the force pass reads it there
        uint32_t* const nbl = c->nbl;
        int32_t* const nbc = c->nbc;
        const bool in_slot = c->prec == 32;
        if (in_slot) {
            c->nbl = c->tape[t].nbl;
            c->nbc = c->tape[t].nbc;
        }
        const sph_status s = run_forces(c, 1, 1, 1);
        c->nbl = nbl;
        c->nbc = nbc;
        SPH_TRY(s);
        SPH_TRY(save_tape(c, t, in_slot));
    }
    AdjView& A = c->adj;
    SPH_CU(cudaMemsetAsync(A.eta, 0, sizeof(double), c->st));
    for (int t = nsteps - 1; t >= 0; --t) {
        SPH_CU(launch_adjoint_step(c->prec, c->dim, (int)c->n, tape_view(c->tape[t]), cells_only(c->G), consts(c), A, 1,
                                      c->st));
        c->launches += 3;
    }
    return SPH_OK;
}

// Capture adjoint_segment(nsteps) from the current state-set parity into a
// graph on the library stream (same rules as graph_capture).
void adjoint_capture(sph_ctx* c, int nsteps)
{
    if (c->astate == 1) cudaGraphExecDestroy(c->aexec);
    c->astate = -1;
    c->asteps = nsteps;
    c->acur0 = c->cur;
    if (!graph_stream(c)) return;
    cudaStream_t user = c->st;
    const int64_t l0 = c->launches;
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(c->gst, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        c->st = c->gst;
        ok = adjoint_segment(c, nsteps) == SPH_OK;
        c->st = user;
        ok = cudaStreamEndCapture(c->gst, &g) == cudaSuccess && ok && g;
    }
    c->acur1 = c->cur;
    c->cur = c->acur0;
    c->alaunches = c->launches - l0;
    c->launches = l0;
    if (ok && cudaGraphInstantiate(&c->aexec, g, 0) == cudaSuccess) c->astate = 1;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
}

}  // namespace

extern "C" {

sph_status sph_default_params(sph_params* p)
{
    if (!p) return SPH_ERR_ARG;
    std::memset(p, 0, sizeof(*p));
    p->dim = 2;
    p->precision = 64;
    p->tv_mode = SPH_TV_LIMITED;
    for (int d = 0; d < 3; ++d) p->L[d] = 1.0;
    p->rho0 = 1.0;
    p->c0 = 10.0;
    p->riemann_eta = 3.0;
    p->tv_xi = -0.2;
    p->tv_C = 1.0e3;
    p->tv_thresh = 5.0e-4;
    p->cfl_ad = 0.25;
    p->cfl_ac = 0.6;
    p->tv_h = SPH_TVH_MIN;
    p->h_pair = SPH_HPAIR_MEAN;
    p->kahan = 1;
    p->graphs = 1;
    p->pair_tiles = 0;
    p->x_subcells = 4;
    return SPH_OK;
}

sph_status sph_query_workspace(const sph_params* p, int64_t n, size_t* bytes)
{
    sph_status s = check_params(p, n);
    if (s != SPH_OK) return s;
    if (!bytes) return SPH_ERR_ARG;
    sph_ctx c;
    std::memset(&c, 0, sizeof(c));
    c.P = *p;
    c.n = n;
    c.dim = p->dim;
    c.prec = p->precision;
    c.G = make_grid(p);
    *bytes = carve(&c, nullptr);
    return SPH_OK;
}

sph_status sph_create(const sph_params* p, int64_t n, void* workspace, size_t bytes, void* stream, sph_ctx** out)
{
    if (!out) return SPH_ERR_ARG;
    *out = nullptr;
    sph_status s = check_params(p, n);
    if (s != SPH_OK) return s;
    if (!workspace || ((uintptr_t)workspace & (kAlign - 1))) return SPH_ERR_WORKSPACE;
    sph_ctx* c = new (std::nothrow) sph_ctx;
    if (!c) return SPH_ERR_ARG;
    std::memset(c, 0, sizeof(*c));
    c->P = *p;
    c->n = n;
    c->dim = p->dim;
    c->prec = p->precision;
    c->st = (cudaStream_t)stream;
    c->G = make_grid(p);
    c->K64 = make_consts<double>(p);
    c->K32 = make_consts<float>(p);
    size_t need = carve(c, nullptr);
    if (bytes < need) {
        delete c;
        return SPH_ERR_WORKSPACE;
    }
    if (p->adjoint_steps > 0) {
        c->tape = new (std::nothrow) TapeSlot[p->adjoint_steps];
        if (!c->tape) {
            delete c;
            return SPH_ERR_ARG;
        }
    }
    carve(c, (char*)workspace);
    if (cudaMemsetAsync(c->err, 0, 4 * sizeof(uint32_t), c->st) != cudaSuccess ||
        cudaMemsetAsync(c->err + 1, 1, 1, c->st) != cudaSuccess ||
        cudaMemsetAsync(c->diag, 0, DG_COUNT * sizeof(double), c->st) != cudaSuccess) {
        delete c;
        return SPH_ERR_CUDA;
    }
    c->host_dt = p->fixed_dt;
    if (cudaMemcpyAsync(c->dt, &c->host_dt, sizeof(double), cudaMemcpyHostToDevice, c->st) != cudaSuccess) {
        delete c;
        return SPH_ERR_CUDA;
    }
    *out = c;
    return SPH_OK;
}

sph_status sph_set_state(sph_ctx* c, const double* x, const double* v, const double* a, const double* dr,
                         const double* h, const double* m, const int8_t* kind, const double* vw, const double* sigma0)
{
    if (!c || !x || !v || !h || !m) return SPH_ERR_ARG;
    if ((a == nullptr) != (dr == nullptr)) return SPH_ERR_ARG;
    const size_t n = (size_t)c->n;
    const size_t vb = 3 * n * sizeof(double);
    c->cur = 0;
    StateSet<double>& Sd = c->set[0].d;
    void* S = cur_set(c);
    void* sv = c->prec == 64 ? (void*)c->set[0].d.v : (void*)c->set[0].f.v;
    void* sa = c->prec == 64 ? (void*)c->set[0].d.a : (void*)c->set[0].f.a;
    void* sdr = c->prec == 64 ? (void*)c->set[0].d.dr : (void*)c->set[0].f.dr;
    (void)S;
    const size_t rs = c->prec == 64 ? 8 : 4;
    SPH_TRY(vec_in(c, 64, x, Sd.x));
    SPH_TRY(vec_in(c, c->prec, v, sv));
    if (a) {
        SPH_TRY(vec_in(c, c->prec, a, sa));
        SPH_TRY(vec_in(c, c->prec, dr, sdr));
    } else {
        SPH_CU(cudaMemsetAsync(sa, 0, c->dim * n * rs, c->st));
        SPH_CU(cudaMemsetAsync(sdr, 0, c->dim * n * rs, c->st));
    }
    SPH_CU(cudaMemcpyAsync(Sd.h, h, n * sizeof(double), cudaMemcpyDefault, c->st));
    SPH_CU(cudaMemcpyAsync(Sd.m, m, n * sizeof(double), cudaMemcpyDefault, c->st));
    if (kind) SPH_CU(cudaMemcpyAsync(Sd.kind, kind, n, cudaMemcpyDefault, c->st));
    else SPH_CU(cudaMemsetAsync(Sd.kind, 0, n, c->st));
    if (vw) SPH_CU(cudaMemcpyAsync(c->stage, vw, vb, cudaMemcpyDefault, c->st));
    SPH_CU(launch_walls_velocity(c->prec, c->dim, (int)n, Sd.kind, vw ? c->stage : nullptr, sv, c->st));
    if (c->P.adjoint_steps > 0) {
        if (vw) SPH_CU(cudaMemcpyAsync(c->orig_vw, c->stage, vb, cudaMemcpyDeviceToDevice, c->st));
        else SPH_CU(cudaMemsetAsync(c->orig_vw, 0, vb, c->st));
    }
    if (sigma0) SPH_CU(cudaMemcpyAsync(Sd.s0, sigma0, n * sizeof(double), cudaMemcpyDefault, c->st));
    else {
        SPH_CU(launch_sigma0(c->dim, (int)n, Sd.h, Sd.m, c->P.rho0, Sd.s0, c->st));
        c->launches += 2;
    }
    SPH_CU(launch_init_ids((int)n, Sd.id, c->st));
    SPH_CU(launch_check_input((int)n, Sd.h, Sd.m, c->P.h_min, c->P.h_max, c->err, c->st));
    SPH_CU(cudaMemsetAsync(c->err + 1, 0, sizeof(uint32_t), c->st));
    SPH_CU(launch_check_constants((int)n, Sd.h, Sd.m, Sd.s0, Sd.kind, c->err + 1, c->st));
    SPH_TRY(copy_constants(c));
    ++c->launches;
    if (Sd.drho) SPH_CU(cudaMemsetAsync(Sd.drho, 0, n * rs, c->st));
    c->launches += 3;
    if (c->P.adjoint_steps > 0) {
        SPH_CU(cudaMemcpyAsync(c->orig_h, Sd.h, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        SPH_CU(cudaMemcpyAsync(c->orig_m, Sd.m, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        SPH_CU(cudaMemcpyAsync(c->orig_s0, Sd.s0, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        SPH_CU(cudaMemcpyAsync(c->orig_kind, Sd.kind, n, cudaMemcpyDeviceToDevice, c->st));
    }
    c->have_state = 1;
    c->have_cells = 0;
    c->ad_given = a != nullptr;
    return SPH_OK;
}

sph_status sph_build_cells(sph_ctx* c)
{
    if (!c) return SPH_ERR_ARG;
    if (!c->have_state) return SPH_ERR_STATE;
    if (c->P.integrator == SPH_INT_DUAL) {
        // density and diagnostics of the loaded state; the first advection
        // step takes Dt_ad and dt_ac from its max |v|
        SPH_TRY(run_sort(c, 2, 0));
        SPH_TRY(run_forces(c, 0, 0, 0));
        c->dual_est = 0;
        c->have_cells = 1;
        return SPH_OK;
    }
    if (c->ad_given) {
        // a and dr given: only the diagnostics and dt_0 (from v and dr); the
        // sort and the density pass are left to the first step, which does
        // both itself
        const int n = (int)c->n;
        SPH_CU(launch_diag_only(c->prec, c->dim, n, cur_set(c), c->partials, c->G.sms, c->st));
        SPH_CU(launch_finalize(pair_blocks(c->prec, n, c->G.sms), c->partials, c->rows, c->P, c->diag, c->dt, 0,
                               c->st));
        c->launches += 2;
        c->cells_pending = 1;
        c->have_cells = 1;
        return SPH_OK;
    }
    sph_status s = run_sort(c, 0, 0);
    if (s != SPH_OK) return s;
    s = run_forces(c, 0, 1, 0);
    if (s != SPH_OK) return s;
    c->cells_pending = 0;
    c->have_cells = 1;
    return SPH_OK;
}

sph_status sph_step(sph_ctx* c, int32_t nsteps)
{
    if (!c || nsteps < 0) return SPH_ERR_ARG;
    const int32_t nsteps_in = nsteps;
    if (!c->have_cells) return SPH_ERR_STATE;
    if (c->P.integrator == SPH_INT_KDK && c->P.graphs && !c->prof_ev && nsteps >= 2) {
        const int par = c->cur;
        if (c->gstate[par] == 0) graph_capture(c, par);
        if (c->gstate[par] == 1) {
            SPH_TRY(graph_launch(c, c->gexec[par], nsteps / 2));
            c->launches += (int64_t)(nsteps / 2) * c->glaunches[par];
            nsteps &= 1;     // two steps per replay bring the sets back to this parity
        }
    }
    for (int32_t k = 0; k < nsteps; ++k) {
        if (c->P.integrator == SPH_INT_DUAL) {
            SPH_TRY(run_dual_step(c));
        } else {
            SPH_TRY(run_sort(c, 1, 0));
            SPH_TRY(run_forces(c, 1, 1, 1));
        }
        if (c->prof_ev) ++c->prof_step;
    }
    if (c->P.integrator == SPH_INT_KDK && nsteps_in > 0) c->cells_pending = 0;
    return SPH_OK;
}

sph_status sph_set_density_rate(sph_ctx* c, const double* drho)
{
    if (!c || !drho || c->P.integrator != SPH_INT_DUAL) return SPH_ERR_ARG;
    if (!c->have_state || c->have_cells) return SPH_ERR_STATE;
    const size_t n = (size_t)c->n;
    void* dst = c->prec == 64 ? (void*)c->set[c->cur].d.drho : (void*)c->set[c->cur].f.drho;
    SPH_CU(cudaMemcpyAsync(c->stage, drho, n * sizeof(double), cudaMemcpyDefault, c->st));
    SPH_CU(launch_scalar_in(c->prec, (int)n, c->stage, c->set[c->cur].d.kind, dst, c->st));
    ++c->launches;
    return SPH_OK;
}

sph_status sph_get_density_rate(sph_ctx* c, double* drho)
{
    if (!c || !drho || c->P.integrator != SPH_INT_DUAL) return SPH_ERR_ARG;
    if (!c->have_state) return SPH_ERR_STATE;
    const int n = (int)c->n;
    const StateSet<double>& Sd = c->set[c->cur].d;
    const void* src = c->prec == 64 ? (void*)Sd.drho : (void*)c->set[c->cur].f.drho;
    SPH_CU(launch_scalar_out(c->prec, n, src, Sd.id, c->stage, c->st));
    SPH_CU(cudaMemcpyAsync(drho, c->stage, (size_t)n * sizeof(double), cudaMemcpyDefault, c->st));
    ++c->launches;
    if (is_host_ptr(drho)) SPH_CU(cudaStreamSynchronize(c->st));
    return SPH_OK;
}

sph_status sph_set_dt(sph_ctx* c, double dt)
{
    if (!c || !(dt > 0) || !std::isfinite(dt)) return SPH_ERR_ARG;
    c->host_dt = dt;
    SPH_CU(cudaMemcpyAsync(c->dt, &c->host_dt, sizeof(double), cudaMemcpyHostToDevice, c->st));
    SPH_CU(cudaStreamSynchronize(c->st));
    return SPH_OK;
}

sph_status sph_set_eta(sph_ctx* c, double eta)
{
    if (!c || !(eta >= 0) || !std::isfinite(eta)) return SPH_ERR_ARG;
    if (eta == c->P.eta) return SPH_OK;    // unchanged: the captured graphs stay valid
    c->P.eta = eta;
    c->K64 = make_consts<double>(&c->P);
    c->K32 = make_consts<float>(&c->P);
    graph_release(c);       // the captured launches hold the old constants
    return SPH_OK;
}

sph_status sph_get_state(sph_ctx* c, double* x, double* v, double* a, double* dr, double* rho)
{
    if (!c) return SPH_ERR_ARG;
    if (!c->have_state) return SPH_ERR_STATE;
    const int n = (int)c->n;
    const size_t vb = 3 * (size_t)n * sizeof(double);
    if (rho && c->have_cells && c->cells_pending) {
        // built with a and dr given and not stepped yet: sort and run the
        // density pass now (a and dr travel with the sort)
        SPH_TRY(run_sort(c, 0, 1));
        SPH_CU(launch_density(c->prec, c->dim, n, cur_set(c), c->start, c->G, consts(c), c->vr, c->pos4, c->cell,
                              c->nbl, c->nbc, c->st, c->vol, c->pos4c, c->P.pair_tiles));
        ++c->launches;
        c->cells_pending = 0;
    }
    const StateSet<double>& Sd = c->set[c->cur].d;
    const void* sv = c->prec == 64 ? (void*)c->set[c->cur].d.v : (void*)c->set[c->cur].f.v;
    const void* sa = c->prec == 64 ? (void*)c->set[c->cur].d.a : (void*)c->set[c->cur].f.a;
    const void* sdr = c->prec == 64 ? (void*)c->set[c->cur].d.dr : (void*)c->set[c->cur].f.dr;
    if (rho && !c->have_cells) return SPH_ERR_STATE;
    bool host = false;
    struct Out { double* dst; const void* src; int prec; } outs[4] = {{x, Sd.x, 64}, {v, sv, c->prec},
                                                                    {a, sa, c->prec}, {dr, sdr, c->prec}};
    // rows in the caller's order, gathered from the sorted positions (pos in
    // the scratch of the sort); written in place into device memory, and
    // through the staging buffer and a copy into host memory (a copy reaches
    // about 3x the rate of kernel stores across the host link)
    int32_t* pos = c->perm_tmp;
    if (x || v || a || dr || rho) {
        SPH_CU(launch_inverse_perm(n, Sd.id, pos, c->st));
        ++c->launches;
    }
    for (auto& o : outs) {
        if (!o.dst) continue;
        double* dv = is_host_ptr(o.dst) ? nullptr : (double*)device_view(o.dst);
        SPH_CU(launch_vec_out_gather(o.prec, c->dim, n, o.src, pos, dv ? dv : c->stage, c->st));
        if (!dv) SPH_CU(cudaMemcpyAsync(o.dst, c->stage, vb, cudaMemcpyDefault, c->st));
        ++c->launches;
        host = host || is_host_ptr(o.dst);
    }
    if (rho) {
        double* dv = is_host_ptr(rho) ? nullptr : (double*)device_view(rho);
        SPH_CU(launch_rho_out_gather(c->prec, n, c->vr, Sd.kind, pos, c->P.rho0, dv ? dv : c->stage, c->st));
        if (!dv) SPH_CU(cudaMemcpyAsync(rho, c->stage, (size_t)n * sizeof(double), cudaMemcpyDefault, c->st));
        ++c->launches;
        host = host || is_host_ptr(rho);
    }
    if (host) SPH_CU(cudaStreamSynchronize(c->st));
    return SPH_OK;
}

sph_status sph_get_diag(sph_ctx* c, sph_diag* out)
{
    if (!c || !out) return SPH_ERR_ARG;
    double buf[DG_COUNT];
    SPH_CU(cudaMemcpyAsync(buf, c->diag, sizeof(buf), cudaMemcpyDeviceToHost, c->st));
    SPH_CU(cudaStreamSynchronize(c->st));
    out->mass = buf[DG_MASS];
    for (int d = 0; d < 3; ++d) out->momentum[d] = buf[DG_MOM + d];
    out->kinetic = buf[DG_KE];
    out->vmax = buf[DG_VMAX];
    out->vt_max = buf[DG_VTMAX];
    out->dr_max = buf[DG_DRMAX];
    out->n_chi = buf[DG_NCHI];
    out->dt = buf[DG_DT];
    out->dt_next = buf[DG_DTNEXT];
    out->steps = buf[DG_STEPS];
    out->substeps = buf[DG_SUBSTEPS];
    for (int d = 0; d < 3; ++d) out->body_force[d] = buf[DG_FBODY + d];
    for (int d = 0; d < 3; ++d) out->body_impulse[d] = buf[DG_IMPULSE + d];
    out->time = buf[DG_TIME];
    return SPH_OK;
}

sph_status sph_sync(sph_ctx* c)
{
    if (!c) return SPH_ERR_ARG;
    uint32_t e = 0;
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_ERR_CUDA;
    if (cudaMemcpy(&e, c->err, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess) return SPH_ERR_CUDA;
    if (!e) return SPH_OK;
    if (cudaMemset(c->err, 0, sizeof(uint32_t)) != cudaSuccess) return SPH_ERR_CUDA;
    if (e & ERRB_INPUT) return SPH_ERR_INPUT;
    if (e & ERRB_NAN) return SPH_ERR_NAN;
    if (e & ERRB_DOMAIN) return SPH_ERR_DOMAIN;
    return SPH_ERR_OVERFLOW;
}

static void prof_free(sph_ctx* c)
{
    if (!c->prof_ev) return;
    for (cudaEvent_t e : *c->prof_ev)
        if (e) cudaEventDestroy(e);
    delete c->prof_ev;
    delete c->prof_used;
    c->prof_ev = nullptr;
    c->prof_used = nullptr;
}

sph_status sph_profile_begin(sph_ctx* c, int32_t max_steps)
{
    if (!c || max_steps < 1) return SPH_ERR_ARG;
    prof_free(c);
    size_t nev = 2 * (size_t)max_steps * SPH_K_NCLASS;
    c->prof_ev = new (std::nothrow) std::vector<cudaEvent_t>(nev, nullptr);
    c->prof_used = new (std::nothrow) std::vector<int>((size_t)max_steps * SPH_K_NCLASS, 0);
    if (!c->prof_ev || !c->prof_used) {
        prof_free(c);
        return SPH_ERR_ARG;
    }
    for (auto& e : *c->prof_ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            prof_free(c);
            return SPH_ERR_CUDA;
        }
    }
    c->prof_max = max_steps;
    c->prof_step = 0;
    return SPH_OK;
}

sph_status sph_profile_end(sph_ctx* c, double* ms, int64_t* count)
{
    if (!c) return SPH_ERR_ARG;
    if (!c->prof_ev) return SPH_ERR_STATE;
    double acc[SPH_K_NCLASS] = {0};
    int64_t cnt[SPH_K_NCLASS] = {0};
    sph_status st = SPH_OK;
    if (cudaStreamSynchronize(c->st) != cudaSuccess) st = SPH_ERR_CUDA;
    int steps = c->prof_step < c->prof_max ? c->prof_step : c->prof_max;
    for (int s = 0; s < steps && st == SPH_OK; ++s)
        for (int k = 0; k < SPH_K_NCLASS; ++k) {
            size_t i = (size_t)s * SPH_K_NCLASS + k;
            if (!(*c->prof_used)[i]) continue;
            float t = 0.f;
            if (cudaEventElapsedTime(&t, (*c->prof_ev)[2 * i], (*c->prof_ev)[2 * i + 1]) != cudaSuccess) {
                st = SPH_ERR_CUDA;
                break;
            }
            acc[k] += t;
            ++cnt[k];
        }
    prof_free(c);
    for (int k = 0; k < SPH_K_NCLASS; ++k) {
        if (ms) ms[k] = acc[k];
        if (count) count[k] = cnt[k];
    }
    return st;
}

const char* sph_kernel_class_name(int32_t k)
{
    static const char* names[SPH_K_NCLASS] = {"kick_drift_key", "scan", "scatter_order", "permute", "density",
                                              "forces", "finalize", "advect", "acoustic"};
    return (k >= 0 && k < SPH_K_NCLASS) ? names[k] : "?";
}

void sph_destroy(sph_ctx* c)
{
    if (!c) return;
    graph_release(c);
    if (c->gst) {
        cudaStreamSynchronize(c->gst);
        cudaEventDestroy(c->gev[0]);
        cudaEventDestroy(c->gev[1]);
        cudaStreamDestroy(c->gst);
    }
    prof_free(c);
    delete[] c->tape;
    delete c;
}

const char* sph_status_str(sph_status s)
{
    switch (s) {
    case SPH_OK: return "ok";
    case SPH_ERR_ARG: return "invalid argument";
    case SPH_ERR_CUDA: return "CUDA error";
    case SPH_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case SPH_ERR_OVERFLOW: return "cell capacity overflow";
    case SPH_ERR_NAN: return "non-finite particle state";
    case SPH_ERR_DOMAIN: return "particle outside the domain";
    case SPH_ERR_STATE: return "call out of order";
    case SPH_ERR_INPUT: return "invalid particle data (h outside [h_min, h_max] or mass not positive)";
    }
    return "unknown status";
}

sph_status sph_save_ckpt(sph_ctx* c, sph_ckpt* ck)
{
    if (!c || !ck || !ck->x || !ck->v || !ck->a || !ck->dr) return SPH_ERR_ARG;
    if (!c->have_state || !c->have_cells) return SPH_ERR_STATE;
    SPH_TRY(sph_get_state(c, ck->x, ck->v, ck->a, ck->dr, nullptr));
    sph_diag d;
    SPH_TRY(sph_get_diag(c, &d));
    ck->dt_next = d.dt_next;
    ck->steps = d.steps;
    return SPH_OK;
}

sph_status sph_step_adjoint(sph_ctx* c, const double* x0, const double* v0, const double* a0, const double* dr0,
                            int32_t nsteps, double* xbar, double* vbar, double* abar, double* drbar, double* etabar)
{
    if (!c || !x0 || !v0 || !a0 || !dr0 || !xbar || !vbar || !abar || !drbar) return SPH_ERR_ARG;
    if (c->P.adjoint_steps < 1 || nsteps < 1 || nsteps > c->P.adjoint_steps) return SPH_ERR_ARG;
    if (c->P.tv_mode == SPH_TV_BACKGROUND) return SPH_ERR_ARG;
    if (!c->have_state) return SPH_ERR_STATE;
    SPH_TRY(reload_state(c, x0, v0, a0, dr0));
    SPH_TRY(sph_build_cells(c));
    AdjView& A = c->adj;
    SPH_TRY(cot_in(c, xbar, A.xc));      // the forward replay leaves the cotangents alone
    SPH_TRY(cot_in(c, vbar, A.vc));
    SPH_TRY(cot_in(c, abar, A.ac));
    SPH_TRY(cot_in(c, drbar, A.drc));
    bool replayed = false;
    if (c->P.graphs && !c->prof_ev) {
        if (c->astate == 0 || c->asteps != nsteps || c->acur0 != c->cur) adjoint_capture(c, nsteps);
        if (c->astate == 1 && c->asteps == nsteps && c->acur0 == c->cur) {
            SPH_TRY(graph_launch(c, c->aexec, 1));
            c->launches += c->alaunches;
            c->cur = c->acur1;
            replayed = true;
        }
    }
    if (!replayed) SPH_TRY(adjoint_segment(c, nsteps));
    SPH_TRY(cot_out(c, A.xc, xbar));
    SPH_TRY(cot_out(c, A.vc, vbar));
    SPH_TRY(cot_out(c, A.ac, abar));
    SPH_TRY(cot_out(c, A.drc, drbar));
    double eta = 0.0;
    SPH_CU(cudaMemcpyAsync(&eta, A.eta, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    SPH_CU(cudaStreamSynchronize(c->st));
    if (etabar) *etabar = eta;
    return SPH_OK;
}

sph_status sph_force_pass_adjoint(sph_ctx* c, const double* x, const double* v, const double* abar,
                                  const double* drbar, double* xbar, double* vbar, double* etabar)
{
    if (!c || !x || !v || !abar || !drbar || !xbar || !vbar) return SPH_ERR_ARG;
    if (c->P.adjoint_steps < 1 || c->P.tv_mode == SPH_TV_BACKGROUND) return SPH_ERR_ARG;
    if (!c->have_state) return SPH_ERR_STATE;
    SPH_TRY(reload_state(c, x, v, nullptr, nullptr));
    SPH_TRY(sph_build_cells(c));
    SPH_TRY(save_tape(c, 0));
    SPH_CU(cudaMemsetAsync(c->tape[0].dt, 0, sizeof(double), c->st));
    AdjView& A = c->adj;
    SPH_CU(cudaMemsetAsync(A.eta, 0, sizeof(double), c->st));
    SPH_TRY(cot_in(c, xbar, A.xc));
    SPH_TRY(cot_in(c, vbar, A.vc));
    SPH_TRY(cot_in(c, abar, A.ac));
    SPH_TRY(cot_in(c, drbar, A.drc));
    SPH_CU(launch_adjoint_step(c->prec, c->dim, (int)c->n, tape_view(c->tape[0]), cells_only(c->G), consts(c), A, 0,
                              c->st));
    c->launches += 3;
    SPH_TRY(cot_out(c, A.xc, xbar));
    SPH_TRY(cot_out(c, A.vc, vbar));
    double eta = 0.0;
    SPH_CU(cudaMemcpyAsync(&eta, A.eta, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    SPH_CU(cudaStreamSynchronize(c->st));
    if (etabar) *etabar = eta;
    return SPH_OK;
}

int64_t sph_launch_count(const sph_ctx* c) { return c ? c->launches : -1; }

}  // extern "C"

// ------------------------------------------------------ density without allocation
//
// Some callers cannot hand this library a workspace: a host framework that owns
// all device memory and whose plug-ins may not call cudaMalloc behind its
// allocator's back, or a real-time loop in which a cudaMalloc/cudaFree (which may
// synchronise the whole device) would stall the frame.  For them,
// sph_density_noalloc runs the density pass on a scratch area that this library
// reserves statically in device memory, sized for SPH_NOALLOC_MAX_PARTICLES
// particles and SPH_NOALLOC_MAX_CELLS cells (24 MiB); every GPU that loads the library
// holds it until the process exits.
namespace {

constexpr size_t kNoAllocScratchBytes = 24u << 20;   // covers 65,536 particles in 3-D (22.6 MiB)

// Device-global scratch; host code must use the address from
// cudaGetSymbolAddress, never the name itself (that is a host-side stand-in).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device.  Outside stream
// capture every call looks it up again (cheap once the library's device code
// is loaded), so an address cached before a device reset -- after which the
// device code is loaded anew, possibly elsewhere -- is never used.  During a
// capture the lookup (which may load the device code) is not made: the
// address of the last call outside capture on this device is used, and a
// capture with no earlier call on the device is refused (SPH_ERR_STATE).
sph_status noalloc_scratch(cudaStream_t st, void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SPH_ERR_CUDA;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return SPH_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SPH_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
    } else if (!g_noalloc_addr[dev]) {
        return SPH_ERR_STATE;
    }
    *out = g_noalloc_addr[dev];
    return SPH_OK;
}

}  // namespace

extern "C" sph_status sph_density_noalloc(const sph_params* p, int64_t n, const double* x, const double* h,
                                          const double* m, const int8_t* kind, const double* sigma0, double* rho,
                                          void* stream)
{
    sph_status s = check_params(p, n);
    if (s != SPH_OK) return s;
    if (p->precision != 64 || !x || !h || !m || !rho) return SPH_ERR_ARG;
    if (n > SPH_NOALLOC_MAX_PARTICLES) return SPH_ERR_WORKSPACE;
    // the cell sort of this view does not refine the cells into sub-cells
    const Grid G = cells_only(make_grid(p));
    if (G.ncell > SPH_NOALLOC_MAX_CELLS) return SPH_ERR_WORKSPACE;
    void* base = nullptr;
    s = noalloc_scratch((cudaStream_t)stream, &base);
    if (s != SPH_OK) return s;

    // Lay out a context-like view over the scratch (host struct only).
    sph_ctx c;
    std::memset(&c, 0, sizeof(c));
    c.P = *p;
    c.P.adjoint_steps = 0;
    c.n = n;
    c.dim = p->dim;
    c.prec = 64;
    c.st = (cudaStream_t)stream;
    c.G = G;
    c.K64 = make_consts<double>(p);
    c.density_only = 1;
    if (carve(&c, nullptr) > kNoAllocScratchBytes) return SPH_ERR_WORKSPACE;
    carve(&c, (char*)base);

    const int ni = (int)n;
    const size_t nc1 = (size_t)G.ncell + 1;
    StateSet<double>& S0 = c.set[0].d;
    // The scratch keeps the previous call's contents: clear what is summed into.
    SPH_CU(cudaMemsetAsync(c.count, 0, nc1 * sizeof(int32_t), c.st));
    SPH_CU(cudaMemsetAsync(c.prefix, 0, nc1 * sizeof(int32_t), c.st));
    SPH_CU(cudaMemsetAsync(c.err, 0, 4 * sizeof(uint32_t), c.st));
    SPH_CU(cudaMemsetAsync(c.err + 1, 1, 1, c.st));   // the sort moves h, m, sigma0 and kind
    SPH_CU(cudaMemsetAsync(S0.v, 0, (size_t)c.dim * n * sizeof(double), c.st));
    SPH_CU(launch_vec_in(64, c.dim, ni, x, S0.x, c.st));
    SPH_CU(cudaMemcpyAsync(S0.h, h, n * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
    SPH_CU(cudaMemcpyAsync(S0.m, m, n * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
    if (kind) SPH_CU(cudaMemcpyAsync(S0.kind, kind, n, cudaMemcpyDeviceToDevice, c.st));
    else SPH_CU(cudaMemsetAsync(S0.kind, 0, n, c.st));
    if (sigma0) SPH_CU(cudaMemcpyAsync(S0.s0, sigma0, n * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
    else SPH_CU(launch_sigma0(c.dim, ni, S0.h, S0.m, p->rho0, S0.s0, c.st));
    SPH_CU(launch_init_ids(ni, S0.id, c.st));
    c.cur = 0;
    s = run_sort(&c, 0, 0);
    if (s != SPH_OK) return s;
    const StateSet<double>& S1 = c.set[c.cur].d;
    SPH_CU(launch_density(64, c.dim, ni, cur_set(&c), c.start, c.G, consts(&c), c.vr, c.pos4, c.cell, nullptr,
                          nullptr, c.st));
    SPH_CU(launch_rho_out(64, ni, c.vr, S1.kind, S1.id, p->rho0, rho, c.st));
    return SPH_OK;
}
