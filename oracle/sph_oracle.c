/*
 * sph_oracle.c -- plain FP64 CPU oracle of the transport-velocity WCSPH
 * kick-drift-kick step of Wang, Haidn & Hu, "The efficient implementation of
 * transport velocity formulation" (arXiv 2411.13992).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct program the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * table or constant with the CUDA library, and the library never calls it.
 *
 * Every quantity is FP64 and every operation is a plain IEEE operation: the
 * file is compiled with -ffp-contract=off, so x86 and Arm builds give the same
 * bits.  OpenMP only splits the outer loop over particles i; the arithmetic
 * for one i does not depend on the thread count.
 *
 * Passages followed (section / equation of the paper):
 *   Wendland kernel, h = 1.3 dp ........................ Sec. 4 (opening paragraph)
 *   equation of state p = c^2 (rho - rho0) ............. Eq. 2
 *   Riemann pressure force ............................. Eq. 3 (second row)
 *   low-dissipation Riemann solver + limiter, eta = 3 .. Eq. 5-6
 *   viscous force ...................................... Eq. 7
 *   density reinitialisation (summation) ............... Eq. 8
 *   advection / acoustic time-step criteria ............ Eq. 9-11, h = h_min
 *   h-scaled transport-velocity displacement ........... Eq. 14
 *   transport-velocity limiter ......................... Eq. 15
 *   limited correction, h = h_min ...................... Eq. 16
 *   kick-drift-kick integration with the correction
 *   applied once per step .............................. Sec. 1, Sec. 3
 *   dual-criteria time stepping: advection steps with
 *   density reinitialisation and the correction, acoustic
 *   substeps with the Riemann pressure force and the
 *   Riemann continuity equation (U*) ................... Sec. 2.4, Eq. 3 (first row), Eq. 5 (first row),
 *                                                          Eq. 9-11, Sec. 3 (correction per advection step)
 *   background pressure p0 = alpha rho0 |v|_ad^2 ....... Eq. 12-13, alpha = 7
 *   force on the body (drag and lift coefficients) ..... Eq. 18, Sec. 4.4
 *   free stream in a periodic box: fringe-region forcing (Nordstrom et al.
 *   1999), standing in for the free-stream boundary the paper cites without
 *   specifying it ....................................... Sec. 4.4
 *
 * Readings where the paper is silent or ambiguous (each is also listed in the
 * design notes of the repository):
 *   - e_ij points from i to j and is used only for the Riemann states U_l, U_r;
 *     grad W_ij means grad_i W_ij = W'(r) (x_i - x_j)/r in Eq. 3, 7, 14-16.
 *   - Wendland C2 with support 2h:
 *       W = a_D (1 - q/2)^4 (2q + 1), q = r/h,
 *       a_2 = 7/(4 pi h^2), a_3 = 21/(16 pi h^3).
 *   - sum W^0_ij in Eq. 8 is the perfect-lattice sum at the particle's own
 *     spacing (passed in per particle as sigma0).
 *   - V_j = m_j / rho_j; rho_bar = (rho_i + rho_j)/2; c_bar = c.
 *   - pair smoothing length h_ij = (h_i + h_j)/2 (or max, by flag).
 *   - the correction computed at the end of step n is added in the drift of
 *     step n+1; walls never move.
 *   - j = i is in the density sum and out of the force sums; two distinct
 *     particles at exactly the same position (r = 0) contribute nothing to the
 *     force sums (the limit of grad W is zero; the viscous limit is skipped).
 *   - wall particles (kind != 0): in a fluid-wall pair rho_j := rho_i,
 *     p_j := p_i, V_j := m_j/rho_i, and the wall's prescribed velocity stands
 *     for v_j.  Walls count in sigma_i and R_i.  PARITY UNPINNED: the paper
 *     gives no wall boundary condition, so only the library-vs-oracle parity
 *     checks this branch.
 *   - pair smoothing length for variable resolution: PARITY UNPINNED beyond
 *     the conservation and brute-force checks (the paper does not state it).
 *   - dual-criteria step (the paper names the scheme and its two criteria;
 *     the order of operations is read as follows): at the start of an
 *     advection step the neighbour set is rebuilt and then frozen for the
 *     whole step (W and W' are evaluated at the current distance, so a pair
 *     that leaves the support stops contributing and a pair that enters it
 *     is not seen until the next advection step); the density is
 *     reinitialised by summation, the viscous acceleration is evaluated once
 *     and held, and the transport displacement is computed and added to the
 *     positions once.  Each acoustic substep dt = min(dt_ac, Dt_ad - t) then
 *     does rho += dt/2 drho; x += dt/2 v; v += dt (a_pressure + a_viscous
 *     + g); x += dt/2 v; drho from the Riemann continuity equation;
 *     rho += dt/2 drho; drho is carried to the next substep and across
 *     advection steps (zero at the start).  The last substep ends exactly at
 *     Dt_ad.  U* is Eq. 5 (first row) with p_L, p_R read as p_l, p_r and no
 *     limiter; a wall j stands in with rho_j = rho_i, p_j = p_i and its
 *     prescribed velocity, as in the force sums.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
    int32_t dim;               /* 2 or 3 */
    int32_t periodic[3];       /* 1: periodic along that axis */
    double lo[3];              /* domain lower corner */
    double L[3];               /* domain lengths */
    double rho0;               /* reference density */
    double c;                  /* artificial sound speed (Eq. 2) */
    double eta;                /* dynamic viscosity (Eq. 7) */
    double g[3];               /* body force per unit mass */
    double h_min;              /* minimum smoothing length (Eq. 9-11, 15-16) */
    double riemann_eta;        /* slope of the dissipation limiter (Eq. 6) */
    int32_t tv_mode;           /* 0 none, 1 limited (Eq. 16), 2 unlimited (Eq. 14),
                                  3 background pressure p0 = rho0 c^2 (Eq. 12) */
    int32_t tv_h_per_particle; /* 0: h = h_min in Eq. 14-16, 1: h = h_i */
    double tv_xi;              /* coefficient xi of Eq. 14 / 16 */
    double tv_C;               /* limiter constant C (Eq. 15) */
    double tv_thresh;          /* limiter threshold (Eq. 15) */
    int32_t h_pair_max;        /* 0: h_ij = (h_i+h_j)/2, 1: max(h_i,h_j) */
    int32_t pad0;
    double cfl_ad, cfl_ac;     /* Eq. 9, 11 */
    double u_ref;              /* reference velocity (Eq. 10) */
    double dt_tv;              /* step size in the background-pressure mode (tv_mode 3) */
    double tv_p0;              /* background pressure of Eq. 12; 0: rho0 c^2 (kick-drift-kick) */
    /* free stream (flow past the cylinder, Sec. 4.4; the paper's free-stream
     * boundary is not specified there): a fringe region along axis 0 in a
     * periodic box forces the fluid toward the free stream (see orc_fringe) */
    double fs_lambda;          /* peak forcing rate lambda_max (0: off) */
    double fs_u[3];            /* free-stream velocity */
    double fs_x[4];            /* x_start, x_end, rise length, fall length of the fringe */
} orc_params;

static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int orc_get_threads(void) { return g_threads; }

/* ---------------------------------------------------------------- kernel */

static double kernel_alpha(double h, int dim)
{
    if (dim == 2) return 7.0 / (4.0 * ORC_PI * h * h);
    return 21.0 / (16.0 * ORC_PI * h * h * h);
}

/* Wendland C2 kernel W(r, h) with support 2h. */
double orc_kernel_W(double r, double h, int dim)
{
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return kernel_alpha(h, dim) * t * t * t * t * (2.0 * q + 1.0);
}

/* dW/dr of the Wendland C2 kernel; <= 0 on [0, 2h). */
double orc_kernel_dW(double r, double h, int dim)
{
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return kernel_alpha(h, dim) / h * (-5.0 * q) * t * t * t;
}

/* Perfect-lattice sum  sum_k W(|k| dp, h) dp^D  for dp = 1, h = h_over_dp,
 * over the integer lattice including the origin.  sigma0 for a particle of
 * spacing dp is this value divided by dp^D (the reference sum of Eq. 8). */
double orc_lattice_sum(int dim, double h_over_dp)
{
    int K = (int)ceil(2.0 * h_over_dp) + 1;
    double s = 0.0;
    int kz0 = dim == 3 ? -K : 0, kz1 = dim == 3 ? K : 0;
    for (int kz = kz0; kz <= kz1; ++kz)
        for (int ky = -K; ky <= K; ++ky)
            for (int kx = -K; kx <= K; ++kx) {
                double r = sqrt((double)(kx * kx + ky * ky + kz * kz));
                s += orc_kernel_W(r, h_over_dp, dim);
            }
    return s;
}

/* ------------------------------------------------------------- geometry */

double orc_pair_h(const orc_params* P, double hi, double hj)
{
    if (P->h_pair_max) return hi > hj ? hi : hj;
    return 0.5 * (hi + hj);
}

/* r_ij = x_i - x_j, minimum image along periodic axes. */
void orc_min_image(const orc_params* P, const double* xi, const double* xj, double* rij)
{
    for (int d = 0; d < 3; ++d) {
        double dx = 0.0;
        if (d < P->dim) {
            dx = xi[d] - xj[d];
            if (P->periodic[d]) {
                if (dx > 0.5 * P->L[d]) dx -= P->L[d];
                else if (dx < -0.5 * P->L[d]) dx += P->L[d];
            }
        }
        rij[d] = dx;
    }
}

static double norm3(const double* r) { return sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]); }
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Put x back into [lo, lo + L) along periodic axes. */
void orc_wrap(const orc_params* P, double* x)
{
    for (int d = 0; d < P->dim; ++d) {
        if (!P->periodic[d]) continue;
        if (x[d] < P->lo[d]) x[d] += P->L[d];
        else if (x[d] >= P->lo[d] + P->L[d]) x[d] -= P->L[d];
    }
}

/* ----------------------------------------------------------- neighbours */

static int is_neighbour(const orc_params* P, const double* x, const double* h, int64_t i, int64_t j)
{
    if (i == j) return 1;
    double rij[3];
    orc_min_image(P, x + 3 * i, x + 3 * j, rij);
    return norm3(rij) < 2.0 * orc_pair_h(P, h[i], h[j]);
}

static int cmp_i64(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

typedef struct {
    int nc[3];
    double base[3], edge[3];
    int64_t* start; /* [ncell + 1] */
    int64_t* list;  /* particles sorted by cell */
} cellgrid;

/* Own cell list: every j with r_ij < 2 h_ij lies in the 3^D block of cells
 * around i's cell when the cell edge is >= 2 h_max.  Returns 0 when the grid
 * would have fewer than 3 cells along a periodic axis (caller falls back to
 * the brute-force search). */
static int cells_build(const orc_params* P, int64_t n, const double* x, const double* h, cellgrid* G)
{
    double hmax = 0.0;
    for (int64_t i = 0; i < n; ++i) hmax = h[i] > hmax ? h[i] : hmax;
    double reach = 2.0 * hmax;
    for (int d = 0; d < 3; ++d) {
        G->nc[d] = 1; G->base[d] = 0.0; G->edge[d] = 1.0;
        if (d >= P->dim) continue;
        if (P->periodic[d]) {
            int nc = (int)floor(P->L[d] / reach);
            if (nc < 3) return 0;
            G->nc[d] = nc; G->base[d] = P->lo[d]; G->edge[d] = P->L[d] / nc;
        } else {
            double mn = x[d], mx = x[d];
            for (int64_t i = 0; i < n; ++i) {
                mn = x[3 * i + d] < mn ? x[3 * i + d] : mn;
                mx = x[3 * i + d] > mx ? x[3 * i + d] : mx;
            }
            G->base[d] = mn; G->edge[d] = reach;
            G->nc[d] = (int)floor((mx - mn) / reach) + 1;
        }
    }
    int64_t ncell = (int64_t)G->nc[0] * G->nc[1] * G->nc[2];
    G->start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    G->list = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t* key = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        for (int d = 0; d < 3; ++d) {
            c[d] = 0;
            if (d >= P->dim) continue;
            c[d] = (int64_t)floor((x[3 * i + d] - G->base[d]) / G->edge[d]);
            if (c[d] < 0) c[d] = 0;
            if (c[d] >= G->nc[d]) c[d] = G->nc[d] - 1;
        }
        key[i] = c[0] + (int64_t)G->nc[0] * (c[1] + (int64_t)G->nc[1] * c[2]);
        G->start[key[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) G->start[c + 1] += G->start[c];
    int64_t* fill = (int64_t*)malloc((size_t)ncell * sizeof(int64_t));
    memcpy(fill, G->start, (size_t)ncell * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) G->list[fill[key[i]]++] = i;
    free(fill);
    free(key);
    return 1;
}

static void cells_free(cellgrid* G) { free(G->start); free(G->list); }

/* Candidates of i from the cell list, written to buf (ascending, neighbours
 * only).  Returns the count. */
static int64_t cells_collect(const orc_params* P, const cellgrid* G, const double* x, const double* h,
                             int64_t i, int64_t* buf)
{
    int64_t ci[3];
    for (int d = 0; d < 3; ++d) {
        ci[d] = 0;
        if (d >= P->dim) continue;
        ci[d] = (int64_t)floor((x[3 * i + d] - G->base[d]) / G->edge[d]);
        if (ci[d] < 0) ci[d] = 0;
        if (ci[d] >= G->nc[d]) ci[d] = G->nc[d] - 1;
    }
    int64_t cnt = 0;
    int r2 = P->dim == 3 ? 1 : 0;
    for (int dz = -r2; dz <= r2; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int64_t c[3] = {ci[0] + dx, ci[1] + dy, ci[2] + dz};
                int skip = 0;
                for (int d = 0; d < 3; ++d) {
                    if (c[d] < 0 || c[d] >= G->nc[d]) {
                        if (d < P->dim && P->periodic[d]) c[d] = (c[d] + G->nc[d]) % G->nc[d];
                        else skip = 1;
                    }
                }
                if (skip) continue;
                int64_t cell = c[0] + (int64_t)G->nc[0] * (c[1] + (int64_t)G->nc[1] * c[2]);
                for (int64_t k = G->start[cell]; k < G->start[cell + 1]; ++k) {
                    int64_t j = G->list[k];
                    if (is_neighbour(P, x, h, i, j)) buf[cnt++] = j;
                }
            }
    qsort(buf, (size_t)cnt, sizeof(int64_t), cmp_i64);
    return cnt;
}

/* Neighbour lists in CSR form, self included, each list ascending in j.
 * mode 0: brute force over all pairs (minimum image);  mode 1: cell list.
 * Call with idx == NULL to get the total count (start[] is filled either way);
 * then call again with idx of that capacity.  Both modes give identical lists. */
int64_t orc_neighbours(const orc_params* P, int64_t n, const double* x, const double* h, int mode,
                       int64_t* start, int64_t* idx)
{
    cellgrid G;
    int use_cells = (mode == 1) && n > 0 && cells_build(P, n, x, h, &G);
    int64_t* count = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t maxbuf = n > 0 ? n : 1;
#pragma omp parallel num_threads(g_threads)
    {
        int64_t* buf = use_cells ? (int64_t*)malloc((size_t)maxbuf * sizeof(int64_t)) : NULL;
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            int64_t cnt = 0;
            if (use_cells) {
                cnt = cells_collect(P, &G, x, h, i, buf);
            } else {
                for (int64_t j = 0; j < n; ++j) cnt += is_neighbour(P, x, h, i, j);
            }
            count[i] = cnt;
        }
#pragma omp single
        {
            start[0] = 0;
            for (int64_t i = 0; i < n; ++i) start[i + 1] = start[i] + count[i];
        }
        if (idx) {
#pragma omp for schedule(dynamic, 256)
            for (int64_t i = 0; i < n; ++i) {
                int64_t* out = idx + start[i];
                if (use_cells) {
                    int64_t cnt = cells_collect(P, &G, x, h, i, buf);
                    memcpy(out, buf, (size_t)cnt * sizeof(int64_t));
                } else {
                    int64_t cnt = 0;
                    for (int64_t j = 0; j < n; ++j)
                        if (is_neighbour(P, x, h, i, j)) out[cnt++] = j;
                }
            }
        }
        free(buf);
    }
    free(count);
    if (use_cells) cells_free(&G);
    return start[n];
}

/* --------------------------------------------------------------- density */

/* Eq. 8 with Eq. 2: sigma_i = sum_j W(r_ij, h_ij) over all neighbours of i
 * (self included, walls included), rho_i = rho0 sigma_i / sigma0_i.
 * Wall particles get rho = rho0 (their own density is never used). */
void orc_density(const orc_params* P, int64_t n, const double* x, const double* h, const int8_t* kind,
                 const double* sigma0, const int64_t* start, const int64_t* idx, double* rho, double* sigma)
{
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = start[i]; k < start[i + 1]; ++k) {
            int64_t j = idx[k];
            double rij[3];
            orc_min_image(P, x + 3 * i, x + 3 * j, rij);
            s += orc_kernel_W(norm3(rij), orc_pair_h(P, h[i], h[j]), P->dim);
        }
        if (sigma) sigma[i] = s;
        rho[i] = kind[i] ? P->rho0 : P->rho0 * s / sigma0[i];
    }
}

/* Eq. 2: artificial equation of state. */
double orc_eos(const orc_params* P, double rho) { return P->c * P->c * (rho - P->rho0); }

/* Eq. 6: dissipation limiter of the low-dissipation Riemann solver. */
double orc_riemann_beta(const orc_params* P, double ul, double ur)
{
    double b = P->riemann_eta * fmax((ul - ur) / P->c, 0.0);
    return fmin(b, 1.0);
}

/* Eq. 5 (second row): interface pressure. */
double orc_riemann_pstar(const orc_params* P, double pl, double pr, double rhobar, double ul, double ur)
{
    double beta = orc_riemann_beta(P, ul, ur);
    return 0.5 * (pl + pr) + 0.5 * beta * rhobar * P->c * (ul - ur);
}

/* Eq. 15: transport-velocity limiter as a function of s = h^2 |R|^2. */
double orc_tv_limiter(const orc_params* P, double s)
{
    if (P->tv_mode == 0) return 0.0;
    if (P->tv_mode == 2 || P->tv_mode == 3) return 1.0;
    if (s > P->tv_thresh) return fmin(P->tv_C * s, 1.0);
    return 0.0;
}

/* Free-stream forcing rate of the fringe region technique (Nordstrom, Nordin
 * & Henningson, SIAM J. Sci. Comput. 20 (1999) 1365): the momentum equation
 * gets lambda(x) (U_inf - v) with
 *   lambda(x) = lambda_max [S((x - x_start)/d_rise) - S((x - x_end)/d_fall + 1)],
 *   S(t) = 0 (t <= 0), 1 / (1 + exp(1/(t - 1) + 1/t)) (0 < t < 1), 1 (t >= 1),
 * a smooth step from 0 to 1 over [0, 1] (S(t) + S(1 - t) = 1).  In a periodic
 * box the region, placed downstream of the body, returns the wake to the free
 * stream before it re-enters upstream.  The paper's free-stream boundary (Sec.
 * 4.4) is not specified in it; this published forcing stands in for it. */
static double fringe_step(double t)
{
    if (t <= 0.0) return 0.0;
    if (t >= 1.0) return 1.0;
    return 1.0 / (1.0 + exp(1.0 / (t - 1.0) + 1.0 / t));
}

double orc_fringe(const orc_params* P, double x)
{
    if (!(P->fs_lambda > 0.0)) return 0.0;
    return P->fs_lambda * (fringe_step((x - P->fs_x[0]) / P->fs_x[2]) - fringe_step((x - P->fs_x[1]) / P->fs_x[3] + 1.0));
}

/* Pressure (Eq. 3, 5, 6) and viscous (Eq. 7) accelerations plus g, and the
 * zero-order residual R_i = sum_j V_j grad_i W_ij with the limited
 * displacement dr_i = xi chi_i h^2 R_i (Eq. 14-16), for every fluid i.
 * Walls get zeros.  chi may be NULL. */
void orc_forces(const orc_params* P, int64_t n, const double* x, const double* v, const double* h,
                const double* m, const int8_t* kind, const double* vw, const double* rho,
                const int64_t* start, const int64_t* idx, double* a, double* R, double* chi, double* dr)
{
    const double c2 = P->c * P->c;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double ai[3] = {0, 0, 0}, Ri[3] = {0, 0, 0};
        if (kind[i]) {
            for (int d = 0; d < 3; ++d) { a[3 * i + d] = 0; R[3 * i + d] = 0; dr[3 * i + d] = 0; }
            if (chi) chi[i] = 0;
            continue;
        }
        for (int d = 0; d < P->dim; ++d) ai[d] = P->g[d];
        const double rho_i = rho[i];
        const double p_i = c2 * (rho_i - P->rho0);
        const double* vi = v + 3 * i;
        for (int64_t k = start[i]; k < start[i + 1]; ++k) {
            int64_t j = idx[k];
            if (j == i) continue;
            double rij[3];
            orc_min_image(P, x + 3 * i, x + 3 * j, rij);
            double r = norm3(rij);
            if (r == 0.0) continue;
            double dw = orc_kernel_dW(r, orc_pair_h(P, h[i], h[j]), P->dim);
            double gradW[3], e[3];
            for (int d = 0; d < 3; ++d) { gradW[d] = dw * rij[d] / r; e[d] = -rij[d] / r; }
            int wall = kind[j] != 0;
            double rho_j = wall ? rho_i : rho[j];
            double p_j = wall ? p_i : c2 * (rho_j - P->rho0);
            const double* vj = wall ? vw + 3 * j : v + 3 * j;
            double V_j = m[j] / rho_j;
            double ul = dot3(vi, e), ur = dot3(vj, e);
            double rhobar = 0.5 * (rho_i + rho_j);
            double pstar = orc_riemann_pstar(P, p_i, p_j, rhobar, ul, ur);
            double cp = -2.0 * m[j] * pstar / (rho_i * rho_j);
            double cv = 2.0 * m[j] * P->eta / (rho_i * rho_j) * dw / r;
            for (int d = 0; d < 3; ++d) {
                ai[d] += cp * gradW[d] + cv * (vi[d] - vj[d]);
                Ri[d] += V_j * gradW[d];
            }
        }
        if (P->fs_lambda > 0.0) {
            /* free-stream forcing of the fringe region (orc_fringe) */
            double lam = orc_fringe(P, x[3 * i]);
            for (int d = 0; d < P->dim; ++d) ai[d] += lam * (P->fs_u[d] - vi[d]);
        }
        double htv = P->tv_h_per_particle ? h[i] : P->h_min;
        double s = htv * htv * dot3(Ri, Ri);
        double ch = orc_tv_limiter(P, s);
        /* Eq. 12 in kick-drift-kick: the background-pressure acceleration
         * a_bg = -2 sum_j m_j p0 / (rho_i rho_j) grad W_ij = -(2 p0 / rho_i) R_i
         * moves the particle by dt^2/2 a_bg in the drift. */
        double p0 = P->tv_p0 > 0.0 ? P->tv_p0 : P->rho0 * c2;
        double bg = -(P->dt_tv * P->dt_tv * p0 / rho_i);
        for (int d = 0; d < 3; ++d) {
            a[3 * i + d] = ai[d];
            R[3 * i + d] = Ri[d];
            dr[3 * i + d] = P->tv_mode == 3 ? bg * Ri[d] : P->tv_xi * ch * htv * htv * Ri[d];
        }
        if (chi) chi[i] = ch;
    }
}

/* Force of the fluid on the wall particles (the body of Eq. 18, e.g. the
 * cylinder of Sec. 4.4): minus the sum over fluid i of m_i times the pressure
 * (Eq. 3, 5, 6) and viscous (Eq. 7) terms of i's wall neighbours, each pair
 * term as in orc_forces (the wall stands in with rho_j = rho_i, p_j = p_i and
 * its prescribed velocity).  F[3] out.  The drag and lift coefficients of
 * Eq. 18 are C_D = 2 F_x / (rho0 U^2 D), C_L = 2 F_y / (rho0 U^2 D). */
void orc_wall_force(const orc_params* P, int64_t n, const double* x, const double* v, const double* h,
                    const double* m, const int8_t* kind, const double* vw, const double* rho,
                    const int64_t* start, const int64_t* idx, double* F)
{
    const double c2 = P->c * P->c;
    double Fx = 0.0, Fy = 0.0, Fz = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (kind[i]) continue;
        const double rho_i = rho[i];
        const double p_i = c2 * (rho_i - P->rho0);
        const double* vi = v + 3 * i;
        double fi[3] = {0, 0, 0};
        for (int64_t k = start[i]; k < start[i + 1]; ++k) {
            int64_t j = idx[k];
            if (j == i || !kind[j]) continue;
            double rij[3];
            orc_min_image(P, x + 3 * i, x + 3 * j, rij);
            double r = norm3(rij);
            if (r == 0.0) continue;
            double dw = orc_kernel_dW(r, orc_pair_h(P, h[i], h[j]), P->dim);
            double gradW[3], e[3];
            for (int d = 0; d < 3; ++d) { gradW[d] = dw * rij[d] / r; e[d] = -rij[d] / r; }
            const double rho_j = rho_i, p_j = p_i;
            const double* vj = vw + 3 * j;
            double ul = dot3(vi, e), ur = dot3(vj, e);
            double pstar = orc_riemann_pstar(P, p_i, p_j, 0.5 * (rho_i + rho_j), ul, ur);
            double cp = -2.0 * m[j] * pstar / (rho_i * rho_j);
            double cv = 2.0 * m[j] * P->eta / (rho_i * rho_j) * dw / r;
            for (int d = 0; d < 3; ++d) fi[d] += cp * gradW[d] + cv * (vi[d] - vj[d]);
        }
        Fx -= m[i] * fi[0];
        Fy -= m[i] * fi[1];
        Fz -= m[i] * fi[2];
    }
    F[0] = Fx;
    F[1] = Fy;
    F[2] = Fz;
}

/* ------------------------------------------------------------ integration */

/* Half (or any) kick of fluid velocities: v += hdt a. */
void orc_kick(const orc_params* P, int64_t n, double hdt, double* v, const double* a, const int8_t* kind)
{
    (void)P;
    for (int64_t i = 0; i < n; ++i) {
        if (kind[i]) continue;
        for (int d = 0; d < 3; ++d) v[3 * i + d] = v[3 * i + d] + hdt * a[3 * i + d];
    }
}

/* Drift of fluid positions with the transport-velocity displacement:
 * x += dt v + dr, then periodic wrap. */
void orc_drift(const orc_params* P, int64_t n, double dt, double* x, const double* v, const double* dr,
               const int8_t* kind)
{
    for (int64_t i = 0; i < n; ++i) {
        if (kind[i]) continue;
        for (int d = 0; d < P->dim; ++d) x[3 * i + d] = x[3 * i + d] + dt * v[3 * i + d] + dr[3 * i + d];
        orc_wrap(P, x + 3 * i);
    }
}

/* Eq. 9-11 with h = h_min: the single step size min(dt_ad, dt_ac). */
double orc_time_step(const orc_params* P, int64_t n, const double* v, const int8_t* kind)
{
    double vmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (kind[i]) continue;
        double s = sqrt(dot3(v + 3 * i, v + 3 * i));
        vmax = s > vmax ? s : vmax;
    }
    double nu = P->eta / P->rho0;
    double vad = fmax(vmax, fmax(nu / P->h_min, P->u_ref));
    double dt_ad = P->cfl_ad * P->h_min / vad;
    double dt_ac = P->cfl_ac * P->h_min / (vmax + P->c);
    return fmin(dt_ad, dt_ac);
}

/* Diagnostics over fluid particles:
 * out[0] mass, out[1..3] momentum, out[4] kinetic energy 1/2 sum m |v|^2,
 * out[5] max |v|, out[6] max |dr| / (dt |v|) (the overcorrection ratio: the
 * transport displacement over the advection displacement, Sec. 3),
 * out[7] number of particles with chi > 0. */
void orc_diagnostics(const orc_params* P, int64_t n, const double* v, const double* m, const int8_t* kind,
                     const double* dr, const double* chi, double dt, double* out)
{
    (void)P;
    for (int k = 0; k < 8; ++k) out[k] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (kind[i]) continue;
        const double* vi = v + 3 * i;
        double v2 = dot3(vi, vi), sp = sqrt(v2);
        out[0] += m[i];
        for (int d = 0; d < 3; ++d) out[1 + d] += m[i] * vi[d];
        out[4] += 0.5 * m[i] * v2;
        out[5] = sp > out[5] ? sp : out[5];
        if (sp > 0.0 && dt > 0.0) {
            double ratio = sqrt(dot3(dr + 3 * i, dr + 3 * i)) / (dt * sp);
            out[6] = ratio > out[6] ? ratio : out[6];
        }
        if (chi && chi[i] > 0.0) out[7] += 1.0;
    }
}

/* --------------------------------------------------------------- driver */

typedef struct {
    int64_t* start;
    int64_t* idx;
} nbrlist;

static int nbr_build(const orc_params* P, int64_t n, const double* x, const double* h, int mode, nbrlist* L)
{
    L->start = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!L->start) return -1;
    int64_t tot = orc_neighbours(P, n, x, h, mode, L->start, NULL);
    L->idx = (int64_t*)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int64_t));
    if (!L->idx) { free(L->start); return -1; }
    orc_neighbours(P, n, x, h, mode, L->start, L->idx);
    return 0;
}

static void nbr_free(nbrlist* L) { free(L->start); free(L->idx); }

/* Force pass on the current positions: neighbours, density, forces.
 * Gives a, R, chi, dr and rho.  Returns 0 on success. */
int orc_force_pass(const orc_params* P, int64_t n, const double* x, const double* v, const double* h,
                   const double* m, const int8_t* kind, const double* vw, const double* sigma0, int mode,
                   double* rho, double* a, double* R, double* chi, double* dr)
{
    nbrlist L;
    if (nbr_build(P, n, x, h, mode, &L)) return -1;
    orc_density(P, n, x, h, kind, sigma0, L.start, L.idx, rho, NULL);
    orc_forces(P, n, x, v, h, m, kind, vw, rho, L.start, L.idx, a, R, chi, dr);
    nbr_free(&L);
    return 0;
}

/* One kick-drift-kick step of size dt, in place on x, v, a, dr:
 *   v += dt/2 a;  x += dt v + dr (wrap);  rho, a, R, chi, dr from the new x
 *   and the half-step v;  v += dt/2 a.
 * Returns 0 on success. */
int orc_step(const orc_params* P, int64_t n, double* x, double* v, double* a, double* dr, const double* h,
             const double* m, const int8_t* kind, const double* vw, const double* sigma0, double dt, int mode,
             double* rho, double* R, double* chi)
{
    double hdt = 0.5 * dt;
    orc_params Q = *P;
    Q.dt_tv = dt;       /* the background-pressure displacement uses this step's dt */
    orc_kick(&Q, n, hdt, v, a, kind);
    orc_drift(&Q, n, dt, x, v, dr, kind);
    if (orc_force_pass(&Q, n, x, v, h, m, kind, vw, sigma0, mode, rho, a, R, chi, dr)) return -1;
    orc_kick(&Q, n, hdt, v, a, kind);
    return 0;
}

/* ===================================================================
 * Adjoint (reverse mode) of the step with the neighbour lists and dt
 * frozen.  Not in the paper: derived by hand from the formulas above.
 * Subgradients at the kinks: d beta/d dU = eta_R / c inside
 * 0 < eta_R dU / c < 1 and 0 elsewhere (Eq. 6); d chi / d s = C inside
 * thresh < s < 1/C and 0 elsewhere (Eq. 15, limited form).
 * =================================================================== */

/* d^2 W / dr^2 of the Wendland C2 kernel. */
double orc_kernel_d2W(double r, double h, int dim)
{
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return kernel_alpha(h, dim) / (h * h) * (-5.0) * t * t * (1.0 - 2.0 * q);
}

double orc_riemann_dbeta(const orc_params* P, double du)
{
    double b = P->riemann_eta * du / P->c;
    return (b > 0.0 && b < 1.0) ? P->riemann_eta / P->c : 0.0;
}

double orc_tv_dlimiter(const orc_params* P, double s)
{
    if (P->tv_mode != 1) return 0.0;
    return (s > P->tv_thresh && P->tv_C * s < 1.0) ? P->tv_C : 0.0;
}

/* Reverse of orc_density + orc_forces at fixed neighbour lists.  Given the
 * cotangents Abar of a and Dbar of dr (fluid particles), add to xbar the
 * cotangents of the positions, to vbar those of the velocities the forces
 * used, and to *etabar that of the dynamic viscosity.  rho and R are the
 * forward values on the same positions. */
void orc_forces_adjoint(const orc_params* P, int64_t n, const double* x, const double* v, const double* h,
                        const double* m, const int8_t* kind, const double* vw, const double* rho,
                        const double* sigma0, const int64_t* start, const int64_t* idx, const double* R,
                        const double* Abar, const double* Dbar, double* xbar, double* vbar, double* etabar)
{
    const double c = P->c, c2 = c * c;
    double* rhob = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double* Rb = (double*)calloc((size_t)(n > 0 ? 3 * n : 1), sizeof(double));
    double etab = 0.0;
    /* 1. transport-velocity displacement dr = xi chi(s) H^2 R, s = H^2 |R|^2 */
    for (int64_t i = 0; i < n; ++i) {
        if (kind[i]) continue;
        double H = P->tv_h_per_particle ? h[i] : P->h_min;
        double H2 = H * H;
        const double* Ri = R + 3 * i;
        const double* Di = Dbar + 3 * i;
        double s = H2 * dot3(Ri, Ri);
        double chi = orc_tv_limiter(P, s), dchi = orc_tv_dlimiter(P, s);
        double DR = dot3(Di, Ri);
        for (int d = 0; d < 3; ++d) Rb[3 * i + d] = P->tv_xi * H2 * (chi * Di[d] + dchi * DR * 2.0 * H2 * Ri[d]);
    }
    /* 2. pair terms of a_i and R_i */
    for (int64_t i = 0; i < n; ++i) {
        if (kind[i]) continue;
        const double rho_i = rho[i];
        const double p_i = c2 * (rho_i - P->rho0);
        const double* vi = v + 3 * i;
        const double* Ai = Abar + 3 * i;
        const double* Rbi = Rb + 3 * i;
        for (int64_t k = start[i]; k < start[i + 1]; ++k) {
            int64_t j = idx[k];
            if (j == i) continue;
            double rij[3];
            orc_min_image(P, x + 3 * i, x + 3 * j, rij);
            double q = norm3(rij);
            if (q == 0.0) continue;
            double hij = orc_pair_h(P, h[i], h[j]);
            double w = orc_kernel_dW(q, hij, P->dim);
            double w2 = orc_kernel_d2W(q, hij, P->dim);
            double u[3], dv[3];
            int wall = kind[j] != 0;
            double rho_j = wall ? rho_i : rho[j];
            double p_j = wall ? p_i : c2 * (rho_j - P->rho0);
            const double* vj = wall ? vw + 3 * j : v + 3 * j;
            for (int d = 0; d < 3; ++d) {
                u[d] = rij[d] / q;
                dv[d] = vi[d] - vj[d];
            }
            double dU = -dot3(dv, u);                       /* U_l - U_r */
            double beta = orc_riemann_beta(P, -dot3(vi, u), -dot3(vj, u));
            double dbeta = orc_riemann_dbeta(P, dU);
            double rbar_ = 0.5 * (rho_i + rho_j);
            double pstar = 0.5 * (p_i + p_j) + 0.5 * beta * rbar_ * c * dU;
            double K = m[j] / (rho_i * rho_j);
            double Au = dot3(Ai, u), Adv = dot3(Ai, dv), Ru = dot3(Rbi, u);
            double Pb = -2.0 * K * w * Au;
            double Kb = -2.0 * pstar * w * Au + 2.0 * P->eta * (w / q) * Adv;
            double wb = -2.0 * K * pstar * Au + (m[j] / rho_j) * Ru;
            double wqb = 2.0 * K * P->eta * Adv;
            etab += 2.0 * K * (w / q) * Adv;
            double dUb = Pb * 0.5 * rbar_ * c * (beta + dU * dbeta);
            double rbarb = Pb * 0.5 * beta * c * dU;
            double ub[3], dvb[3], rb[3];
            for (int d = 0; d < 3; ++d) {
                ub[d] = -2.0 * K * pstar * w * Ai[d] + (m[j] / rho_j) * w * Rbi[d] - dUb * dv[d];
                dvb[d] = 2.0 * K * P->eta * (w / q) * Ai[d] - dUb * u[d];
            }
            double rho_i_b = -K / rho_i * Kb + 0.5 * rbarb + c2 * 0.5 * Pb;
            double rho_j_b = -K / rho_j * Kb + 0.5 * rbarb + c2 * 0.5 * Pb - (m[j] / (rho_j * rho_j)) * w * Ru;
            rhob[i] += rho_i_b;
            if (wall) rhob[i] += rho_j_b;          /* rho_j stands for rho_i, p_j for p_i */
            else rhob[j] += rho_j_b;
            double uu = dot3(ub, u);
            for (int d = 0; d < 3; ++d)
                rb[d] = (ub[d] - uu * u[d]) / q + w2 * wb * u[d] + (w2 / q - w / (q * q)) * wqb * u[d];
            for (int d = 0; d < 3; ++d) {
                xbar[3 * i + d] += rb[d];
                vbar[3 * i + d] += dvb[d];
                if (!wall) {
                    xbar[3 * j + d] -= rb[d];
                    vbar[3 * j + d] -= dvb[d];
                }
            }
        }
    }
    /* 3. density summation rho_i = rho0 sigma_i / sigma0_i */
    for (int64_t i = 0; i < n; ++i) {
        if (kind[i]) continue;
        double sb = rhob[i] * P->rho0 / sigma0[i];
        for (int64_t k = start[i]; k < start[i + 1]; ++k) {
            int64_t j = idx[k];
            if (j == i) continue;
            double rij[3];
            orc_min_image(P, x + 3 * i, x + 3 * j, rij);
            double q = norm3(rij);
            if (q == 0.0) continue;
            double w = orc_kernel_dW(q, orc_pair_h(P, h[i], h[j]), P->dim);
            for (int d = 0; d < 3; ++d) {
                double g = sb * w * rij[d] / q;
                xbar[3 * i + d] += g;
                if (!kind[j]) xbar[3 * j + d] -= g;
            }
        }
    }
    *etabar += etab;
    free(rhob);
    free(Rb);
}

/* Adjoint of orc_step.  On entry xbar, vbar, abar, drbar hold the
 * cotangents of the step's outputs (x', v', a', dr'); on return those of its
 * inputs (x, v, a, dr).  *etabar is incremented.  The forward internals are
 * recomputed from the inputs x, v, a, dr (unchanged).  Walls get zeros. */
int orc_step_adjoint(const orc_params* P, int64_t n, const double* x, const double* v, const double* a,
                     const double* dr, const double* h, const double* m, const int8_t* kind, const double* vw,
                     const double* sigma0, double dt, int mode, double* xbar, double* vbar, double* abar,
                     double* drbar, double* etabar)
{
    if (P->tv_mode == 3) return -2;     /* the background-pressure mode has no adjoint here */
    size_t nb = (size_t)(n > 0 ? 3 * n : 1) * sizeof(double);
    double* xp = (double*)malloc(nb);
    double* vh = (double*)malloc(nb);
    double* A = (double*)malloc(nb);
    double* Rf = (double*)malloc(nb);
    double* af = (double*)malloc(nb);
    double* drf = (double*)malloc(nb);
    double* rho = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!xp || !vh || !A || !Rf || !af || !drf || !rho) return -1;
    memcpy(xp, x, nb);
    memcpy(vh, v, nb);
    double hdt = 0.5 * dt;
    orc_kick(P, n, hdt, vh, a, kind);
    orc_drift(P, n, dt, xp, vh, dr, kind);
    nbrlist L;
    if (nbr_build(P, n, xp, h, mode, &L)) return -1;
    orc_density(P, n, xp, h, kind, sigma0, L.start, L.idx, rho, NULL);
    orc_forces(P, n, xp, vh, h, m, kind, vw, rho, L.start, L.idx, af, Rf, NULL, drf);
    /* v' = vh + hdt a'  ->  abar' += hdt vbar', vhbar = vbar' */
    for (int64_t i = 0; i < 3 * n; ++i) A[i] = abar[i] + hdt * vbar[i];
    /* vbar now holds vhbar; xbar holds xbar' */
    orc_forces_adjoint(P, n, xp, vh, h, m, kind, vw, rho, sigma0, L.start, L.idx, Rf, A, drbar, xbar, vbar,
                       etabar);
    /* x' = x + dt vh + dr ;  vh = v + hdt a */
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < 3; ++d) {
            int64_t o = 3 * i + d;
            if (kind[i]) {
                xbar[o] = vbar[o] = abar[o] = drbar[o] = 0.0;
                continue;
            }
            drbar[o] = xbar[o];
            vbar[o] += dt * xbar[o];
            abar[o] = hdt * vbar[o];
        }
    }
    nbr_free(&L);
    free(xp); free(vh); free(A); free(Rf); free(af); free(drf); free(rho);
    return 0;
}

/* Adjoint of the initial force pass (a, dr from x, v): given Abar, Dbar,
 * add to xbar and vbar and increment *etabar. */
int orc_force_pass_adjoint(const orc_params* P, int64_t n, const double* x, const double* v, const double* h,
                           const double* m, const int8_t* kind, const double* vw, const double* sigma0, int mode,
                           const double* Abar, const double* Dbar, double* xbar, double* vbar, double* etabar)
{
    if (P->tv_mode == 3) return -2;
    size_t nb = (size_t)(n > 0 ? 3 * n : 1) * sizeof(double);
    double* Rf = (double*)malloc(nb);
    double* af = (double*)malloc(nb);
    double* drf = (double*)malloc(nb);
    double* rho = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!Rf || !af || !drf || !rho) return -1;
    nbrlist L;
    if (nbr_build(P, n, x, h, mode, &L)) return -1;
    orc_density(P, n, x, h, kind, sigma0, L.start, L.idx, rho, NULL);
    orc_forces(P, n, x, v, h, m, kind, vw, rho, L.start, L.idx, af, Rf, NULL, drf);
    orc_forces_adjoint(P, n, x, v, h, m, kind, vw, rho, sigma0, L.start, L.idx, Rf, Abar, Dbar, xbar, vbar,
                       etabar);
    nbr_free(&L);
    free(Rf); free(af); free(drf); free(rho);
    return 0;
}


/* ===================================================================
 * Dual-criteria time stepping (Sec. 2.4; the correction once per
 * advection step, Sec. 3).
 * =================================================================== */

/* Eq. 7 alone: viscous acceleration of every fluid i (walls: zeros). */
void orc_viscous(const orc_params* P, int64_t n, const double* x, const double* v, const double* h,
                 const double* m, const int8_t* kind, const double* vw, const double* rho, const int64_t* start,
                 const int64_t* idx, double* a_nu)
{
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double ai[3] = {0, 0, 0};
        if (!kind[i]) {
            const double rho_i = rho[i];
            const double* vi = v + 3 * i;
            for (int64_t k = start[i]; k < start[i + 1]; ++k) {
                int64_t j = idx[k];
                if (j == i) continue;
                double rij[3];
                orc_min_image(P, x + 3 * i, x + 3 * j, rij);
                double r = norm3(rij);
                if (r == 0.0) continue;
                double dw = orc_kernel_dW(r, orc_pair_h(P, h[i], h[j]), P->dim);
                int wall = kind[j] != 0;
                double rho_j = wall ? rho_i : rho[j];
                const double* vj = wall ? vw + 3 * j : v + 3 * j;
                double cv = 2.0 * m[j] * P->eta / (rho_i * rho_j) * dw / r;
                for (int d = 0; d < 3; ++d) ai[d] += cv * (vi[d] - vj[d]);
            }
        }
        for (int d = 0; d < 3; ++d) a_nu[3 * i + d] = ai[d];
    }
}

/* Eq. 3 (second row) with the interface pressure of Eq. 5-6 alone: the
 * pressure acceleration of every fluid i (walls: zeros). */
void orc_pressure(const orc_params* P, int64_t n, const double* x, const double* v, const double* h,
                  const double* m, const int8_t* kind, const double* vw, const double* rho, const int64_t* start,
                  const int64_t* idx, double* a_p)
{
    const double c2 = P->c * P->c;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double ai[3] = {0, 0, 0};
        if (!kind[i]) {
            const double rho_i = rho[i];
            const double p_i = c2 * (rho_i - P->rho0);
            const double* vi = v + 3 * i;
            for (int64_t k = start[i]; k < start[i + 1]; ++k) {
                int64_t j = idx[k];
                if (j == i) continue;
                double rij[3];
                orc_min_image(P, x + 3 * i, x + 3 * j, rij);
                double r = norm3(rij);
                if (r == 0.0) continue;
                double dw = orc_kernel_dW(r, orc_pair_h(P, h[i], h[j]), P->dim);
                double e[3];
                for (int d = 0; d < 3; ++d) e[d] = -rij[d] / r;
                int wall = kind[j] != 0;
                double rho_j = wall ? rho_i : rho[j];
                double p_j = wall ? p_i : c2 * (rho_j - P->rho0);
                const double* vj = wall ? vw + 3 * j : v + 3 * j;
                double pstar = orc_riemann_pstar(P, p_i, p_j, 0.5 * (rho_i + rho_j), dot3(vi, e), dot3(vj, e));
                double cp = -2.0 * m[j] * pstar / (rho_i * rho_j);
                for (int d = 0; d < 3; ++d) ai[d] += cp * dw * rij[d] / r;
            }
        }
        for (int d = 0; d < 3; ++d) a_p[3 * i + d] = ai[d];
    }
}

/* Eq. 5 (first row) with p_L, p_R read as p_l, p_r: interface velocity. */
double orc_riemann_ustar(const orc_params* P, double pl, double pr, double rhobar, double ul, double ur)
{
    return 0.5 * (ul + ur) + 0.5 * (pl - pr) / (rhobar * P->c);
}

/* Eq. 3 (first row): drho_i/dt = 2 rho_i sum_j V_j (U*_ij - U_l) dW/dr for
 * every fluid i (walls: zero). */
void orc_continuity(const orc_params* P, int64_t n, const double* x, const double* v, const double* h,
                    const double* m, const int8_t* kind, const double* vw, const double* rho, const int64_t* start,
                    const int64_t* idx, double* drho)
{
    const double c2 = P->c * P->c;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        const double rho_i = rho[i];
        if (!kind[i]) {
            const double p_i = c2 * (rho_i - P->rho0);
            const double* vi = v + 3 * i;
            for (int64_t k = start[i]; k < start[i + 1]; ++k) {
                int64_t j = idx[k];
                if (j == i) continue;
                double rij[3];
                orc_min_image(P, x + 3 * i, x + 3 * j, rij);
                double r = norm3(rij);
                if (r == 0.0) continue;
                double dw = orc_kernel_dW(r, orc_pair_h(P, h[i], h[j]), P->dim);
                double e[3];
                for (int d = 0; d < 3; ++d) e[d] = -rij[d] / r;
                int wall = kind[j] != 0;
                double rho_j = wall ? rho_i : rho[j];
                double p_j = wall ? p_i : c2 * (rho_j - P->rho0);
                const double* vj = wall ? vw + 3 * j : v + 3 * j;
                double ul = dot3(vi, e);
                double ustar = orc_riemann_ustar(P, p_i, p_j, 0.5 * (rho_i + rho_j), ul, dot3(vj, e));
                s += m[j] / rho_j * (ustar - ul) * dw;
            }
        }
        drho[i] = kind[i] ? 0.0 : 2.0 * rho_i * s;
    }
}

/* Eq. 9-10 with h = h_min: the advection step size; *vad_out (may be NULL)
 * receives the advection speed |v|_ad. */
double orc_advection_step(const orc_params* P, int64_t n, const double* v, const int8_t* kind, double* vad_out)
{
    double vmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (kind[i]) continue;
        double sp = sqrt(dot3(v + 3 * i, v + 3 * i));
        vmax = sp > vmax ? sp : vmax;
    }
    double nu = P->eta / P->rho0;
    double vad = fmax(vmax, fmax(nu / P->h_min, P->u_ref));
    if (vad_out) *vad_out = vad;
    return P->cfl_ad * P->h_min / vad;
}

/* Eq. 11 with h = h_min: the acoustic step size. */
double orc_acoustic_step(const orc_params* P, int64_t n, const double* v, const int8_t* kind)
{
    double vmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (kind[i]) continue;
        double sp = sqrt(dot3(v + 3 * i, v + 3 * i));
        vmax = sp > vmax ? sp : vmax;
    }
    return P->cfl_ac * P->h_min / (vmax + P->c);
}

#define ORC_BG_ALPHA 7.0   /* alpha of Eq. 13 */

/* One advection step of the dual-criteria scheme, in place on x, v, rho,
 * drho (the state); a receives the last substep's acceleration, dr, R, chi
 * the correction of this step, *Dt_out the advection step size.  Returns the
 * number of acoustic substeps, or -1 if memory runs out. */
int64_t orc_dual_step(const orc_params* P, int64_t n, double* x, double* v, double* rho, double* drho,
                      const double* h, const double* m, const int8_t* kind, const double* vw, const double* sigma0,
                      int mode, double* a, double* dr, double* R, double* chi, double* Dt_out)
{
    nbrlist L;
    if (nbr_build(P, n, x, h, mode, &L)) return -1;
    double* a_nu = (double*)malloc((size_t)(3 * n > 0 ? 3 * n : 1) * sizeof(double));
    double* a_p = (double*)malloc((size_t)(3 * n > 0 ? 3 * n : 1) * sizeof(double));
    if (!a_nu || !a_p) { free(a_nu); free(a_p); nbr_free(&L); return -1; }
    /* advection step: density reinitialisation (Eq. 8), step size (Eq. 9-10),
     * viscous acceleration (Eq. 7), transport correction (Eq. 14-16, or
     * Eq. 12 with p0 of Eq. 13), applied once */
    orc_density(P, n, x, h, kind, sigma0, L.start, L.idx, rho, NULL);
    double vad;
    const double Dt = orc_advection_step(P, n, v, kind, &vad);
    orc_params Q = *P;
    Q.dt_tv = Dt;
    Q.tv_p0 = ORC_BG_ALPHA * P->rho0 * vad * vad;
    orc_viscous(&Q, n, x, v, h, m, kind, vw, rho, L.start, L.idx, a_nu);
    orc_forces(&Q, n, x, v, h, m, kind, vw, rho, L.start, L.idx, a_p, R, chi, dr);
    for (int64_t i = 0; i < n; ++i) {
        if (kind[i]) continue;
        for (int d = 0; d < P->dim; ++d) x[3 * i + d] = x[3 * i + d] + dr[3 * i + d];
    }
    /* acoustic substeps (Eq. 11) */
    double t = 0.0;
    int64_t k = 0;
    for (;;) {
        double dt = orc_acoustic_step(P, n, v, kind);
        const double rem = Dt - t;
        const int last = dt >= rem;
        if (last) dt = rem;
        const double hdt = 0.5 * dt;
        for (int64_t i = 0; i < n; ++i) {
            if (kind[i]) continue;
            rho[i] = rho[i] + hdt * drho[i];
            for (int d = 0; d < P->dim; ++d) x[3 * i + d] = x[3 * i + d] + hdt * v[3 * i + d];
        }
        orc_pressure(P, n, x, v, h, m, kind, vw, rho, L.start, L.idx, a_p);
        for (int64_t i = 0; i < n; ++i) {
            for (int d = 0; d < 3; ++d) {
                double ad = kind[i] || d >= P->dim ? 0.0 : a_p[3 * i + d] + a_nu[3 * i + d] + P->g[d];
                a[3 * i + d] = ad;
                if (!kind[i]) v[3 * i + d] = v[3 * i + d] + dt * ad;
            }
        }
        for (int64_t i = 0; i < n; ++i) {
            if (kind[i]) continue;
            for (int d = 0; d < P->dim; ++d) x[3 * i + d] = x[3 * i + d] + hdt * v[3 * i + d];
        }
        orc_continuity(P, n, x, v, h, m, kind, vw, rho, L.start, L.idx, drho);
        for (int64_t i = 0; i < n; ++i) {
            if (kind[i]) continue;
            rho[i] = rho[i] + hdt * drho[i];
        }
        t = t + dt;
        ++k;
        if (last) break;
    }
    for (int64_t i = 0; i < n; ++i)
        if (!kind[i]) orc_wrap(P, x + 3 * i);
    if (Dt_out) *Dt_out = Dt;
    free(a_nu);
    free(a_p);
    nbr_free(&L);
    return k;
}
