/*
 * FP64 CPU oracle for the Minimod acoustic isotropic constant-density
 * propagator (arXiv 2007.06048).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline / reference leg load it;
 * the library never does.  The two share no code, header, table or constant.
 *
 * What it computes, by the paper's sections:
 *   Eq. 1   (1/v^2) p_tt - lap p = f
 *   Eq. 5   p^{n+1} - Q p^n + p^{n-1} = dt^2 v^2 f^n,   Q = 2 + dt^2 v^2 lap
 *   Sec. 3  the 25-point star Laplacian  sum_m c_am [p(+m) + p(-m) - 2 p]  on
 *           each axis a, with c_am from the order-2R Taylor expansion
 *   Alg. 1  p^0 = 0; each step solves the left-hand side everywhere and then
 *           adds the source term f^n
 *   Alg. 2  an inner region updated with Eq. 5 and six damping regions
 *           (left/right, back/front, top/bottom) around it
 *
 * Readings where the paper is silent (also listed in the design notes):
 *   R2  u = 0 outside the grid (homogeneous Dirichlet).
 *   R3  the damping regions solve u_tt + 2 eta u_t = v^2 (lap u + f), centred
 *       in time, which gives
 *          u^{n+1} = [2 u^n - (1 - eta dt) u^{n-1} + c lap u^n] / (1 + eta dt)
 *       with c = dt^2 v^2, eta = eta_x(i) + eta_y(j) + eta_z(k),
 *       eta_a(i) = eta_max,a (d/L)^2, d = max(L - i, i - (n_a - 1 - L), 0),
 *       eta_max,a = 3 vmax ln(1/R) / (2 L h_a).  Where eta = 0 this is Eq. 5.
 *   R4  the damping layers are part of the grid; the inner region is
 *       [L, n_a - 1 - L] on every axis.
 *   R5  a point source: the discrete f^n at x_s is w[n] / (hx hy hz), so the
 *       add of Alg. 1 is  c(x_s) w[n] / (hx hy hz (1 + eta(x_s) dt)),  i.e.
 *       the source sits inside the damped update's numerator.
 *   R7  receivers record u^{n+1} at grid points after the add of step n.
 *   R16 optimised stencils (Sec. 3 allows weights of lower formal order
 *       with a smaller dispersion error and gives none): c_1..c_R minimise
 *       the squared relative error of the 1-D second-derivative symbol,
 *          int_0^kmax ( sum_m 2 c_m (1 - cos m k) / k^2 - 1 )^2 dk,
 *       over the band kh in [0, kmax], subject to sum_m m^2 c_m = 1 (exact
 *       for quadratics, second order); orc_optimized_coeffs.  Any weight set
 *       can drive the Laplacian and the stepper (coef argument).
 *   R17 CPML (Sec. 3 names a convolutional PML, with no formula): the
 *       second-order equation with complex-frequency-shifted stretching
 *       s_a = 1 + d_a / (alpha_a + i w) on each axis,
 *          u_tt = v^2 sum_a [ D2_a u + D1_a psi_a + zeta_a ] + v^2 f,
 *          psi_a  = chi_a * D1_a u,   zeta_a = chi_a * (D2_a u + D1_a psi_a),
 *          chi_a(t) = -d_a exp(-(d_a + alpha_a) t),
 *       with the recursive convolutions  m^n = b m^{n-1} + g q^n,
 *       b = exp(-(d + alpha) dt),  g = d (b - 1) / (d + alpha),  D2_a the
 *       order-8 second difference, D1_a the order-8 centred first difference
 *       (weights 4/5, -1/5, 4/105, -1/280), psi = 0 outside the grid.  Per
 *       step: psi^n from u^n, then zeta^n and u^{n+1} = 2u^n - u^{n-1} +
 *       C (sum_a (D2_a u^n + D1_a psi_a^n + zeta_a^n) + s^n).  Profiles on L
 *       cells per face: d_a = d0_a (x/L)^2, alpha_a = pi f0 (1 - x/L), x the
 *       depth into the layer (x = L at the outer cell, 0 from cell L
 *       inward), d0_a = 3 v_max ln(1/R) / (2 L h_a).  With a free surface the
 *       top layer is absent (reading R15).  orc_forward_cpml.
 *   R15 free surface (the paper's option at the surface, Sec. 3): p = 0 on
 *       the plane k = 0, imposed as the odd image  u(i, j, -m) = -u(i, j, m)
 *       for the stencil and u(i, j, 0) = 0 after every step (sources added
 *       there vanish, receivers there read 0); the top damping layer is
 *       removed (eta_z = 0 for k < L), the other five faces keep theirs.
 *
 *   R18 the variable-density first-order system of Sec. 3 (the paper's
 *       "acoustic_iso" on a staggered Yee grid): p at the grid points, the
 *       particle-velocity components half a cell along their axes, leapfrog
 *       with the velocities at half steps, order-8 staggered weights, damping
 *       or CPML layers, optionally the free surface (p odd and v_z even
 *       about k = 0); stated in full before orc_forward_vd.
 *
 * Index convention: i along x (fastest), j along y, k along z (depth, k = 0 at
 * the surface); user arrays are [nz][ny][nx].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_R 8

/* ------------------------------------------------------------------------ */
/* Sec. 3: second-derivative weights from the Taylor expansion.             */
/*                                                                          */
/*   f(x+mh) + f(x-mh) - 2 f(x) = sum_{p>=1} 2 (mh)^{2p} f^{(2p)}(x) / (2p)! */
/*                                                                          */
/* so  sum_m c_m [f(x+mh) + f(x-mh) - 2 f(x)] = h^2 f''(x) + O(h^{2R+2})    */
/* exactly when  sum_m c_m m^2 = 1  and  sum_m c_m m^{2p} = 0, p = 2..R.    */
/* The R x R system is solved by Gaussian elimination with partial pivots.  */
/* Output: c[0] = -2 sum_m c_m (the centre weight), c[m] = c_m, m = 1..R.  */
/* ------------------------------------------------------------------------ */
int orc_fd_coeffs(int order, double *c)
{
    if (order < 2 || order % 2 != 0 || order / 2 > ORC_MAX_R || !c) return -1;
    const int R = order / 2;
    double A[ORC_MAX_R][ORC_MAX_R + 1];
    for (int p = 1; p <= R; ++p) {
        for (int m = 1; m <= R; ++m) A[p - 1][m - 1] = pow((double)m, 2.0 * p);
        A[p - 1][R] = (p == 1) ? 1.0 : 0.0;
    }
    for (int col = 0; col < R; ++col) {
        int piv = col;
        for (int r = col + 1; r < R; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) return -2;
        if (piv != col)
            for (int q = 0; q <= R; ++q) { double t = A[col][q]; A[col][q] = A[piv][q]; A[piv][q] = t; }
        for (int r = 0; r < R; ++r) {
            if (r == col) continue;
            const double f = A[r][col] / A[col][col];
            for (int q = col; q <= R; ++q) A[r][q] -= f * A[col][q];
        }
    }
    double sum = 0.0;
    for (int m = 1; m <= R; ++m) { c[m] = A[m - 1][R] / A[m - 1][m - 1]; sum += c[m]; }
    c[0] = -2.0 * sum;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Reading R16: least-squares weights over the band [0, kmax] (radians per  */
/* cell) with the consistency constraint sum_m m^2 c_m = 1.  The integral   */
/* is a composite trapezoid rule on nq intervals; a_m(k) = 2(1 - cos mk)/k^2 */
/* (a_m(0) = m^2).  Stationarity of the Lagrangian gives the symmetric      */
/* system  [G g; g^T 0] [c; lambda] = [b; 1],  G_mn = int a_m a_n,          */
/* b_m = int a_m, g_m = m^2, solved by Gaussian elimination with pivots.    */
/* Output as orc_fd_coeffs: c[0] = -2 sum c_m, c[m] = c_m.                  */
/* ------------------------------------------------------------------------ */
int orc_optimized_coeffs(int order, double kmax, int nq, double *c)
{
    if (order < 2 || order % 2 != 0 || order / 2 > ORC_MAX_R || !c) return -1;
    if (!(kmax > 0.0 && kmax <= 3.14159265358979323846) || nq < 2) return -1;
    const int R = order / 2, n = R + 1;
    double A[ORC_MAX_R + 1][ORC_MAX_R + 2];
    for (int r = 0; r < n; ++r)
        for (int q = 0; q <= n; ++q) A[r][q] = 0.0;
    for (int q = 0; q <= nq; ++q) {
        const double k = kmax * q / nq;
        const double w = (q == 0 || q == nq) ? 0.5 * kmax / nq : kmax / nq;
        double a[ORC_MAX_R + 1];
        for (int m = 1; m <= R; ++m)
            a[m] = (q == 0) ? (double)m * m : 2.0 * (1.0 - cos(m * k)) / (k * k);
        for (int i = 1; i <= R; ++i) {
            for (int j = 1; j <= R; ++j) A[i - 1][j - 1] += w * a[i] * a[j];
            A[i - 1][n] += w * a[i];
        }
    }
    for (int m = 1; m <= R; ++m) { A[m - 1][R] = (double)m * m; A[R][m - 1] = (double)m * m; }
    A[R][R] = 0.0;
    A[R][n] = 1.0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) return -2;
        if (piv != col)
            for (int q = 0; q <= n; ++q) { double t = A[col][q]; A[col][q] = A[piv][q]; A[piv][q] = t; }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const double f = A[r][col] / A[col][col];
            for (int q = col; q <= n; ++q) A[r][q] -= f * A[col][q];
        }
    }
    double sum = 0.0;
    for (int m = 1; m <= R; ++m) { c[m] = A[m - 1][n] / A[m - 1][m - 1]; sum += c[m]; }
    c[0] = -2.0 * sum;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Reading R3: damping profile along one axis of n cells, L = nbl.          */
/* ------------------------------------------------------------------------ */
int orc_damping_profile(int n, int nbl, double h, double vmax, double refl, double *eta)
{
    if (n < 1 || nbl < 0 || 2 * nbl > n || h <= 0 || !eta) return -1;
    if (nbl == 0) { for (int i = 0; i < n; ++i) eta[i] = 0.0; return 0; }
    if (!(refl > 0.0 && refl < 1.0) || vmax <= 0) return -1;
    const double eta_max = 3.0 * vmax * log(1.0 / refl) / (2.0 * nbl * h);
    for (int i = 0; i < n; ++i) {
        int d = 0;
        if (nbl - i > d) d = nbl - i;
        if (i - (n - 1 - nbl) > d) d = i - (n - 1 - nbl);
        const double s = (double)d / (double)nbl;
        eta[i] = eta_max * s * s;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Wavefields live in a zero-padded copy: R extra cells on every side hold  */
/* the u = 0 of reading R2 literally, so the stencil needs no bounds tests. */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz, R;
    long px, py, pz;   /* padded extents */
    long sy, sz;       /* strides of j and k in the padded array */
} grid_t;

static grid_t make_grid(int nx, int ny, int nz, int R)
{
    grid_t g;
    g.nx = nx; g.ny = ny; g.nz = nz; g.R = R;
    g.px = nx + 2L * R; g.py = ny + 2L * R; g.pz = nz + 2L * R;
    g.sy = g.px; g.sz = g.px * g.py;
    return g;
}

static inline long at(const grid_t *g, int i, int j, int k)
{
    return ((long)k + g->R) * g->sz + ((long)j + g->R) * g->sy + ((long)i + g->R);
}

static double *padded_zeros(const grid_t *g)
{
    return (double *)calloc((size_t)(g->px * g->py * g->pz), sizeof(double));
}

/* Reading R15: fill the R planes above the surface with the odd image of
 * the planes below it (every padded x-y position, so edges stay zero).    */
static void mirror_top(const grid_t *g, double *u)
{
    for (int m = 1; m <= g->R && m < g->nz; ++m)
        for (int j = -g->R; j < g->ny + g->R; ++j)
            for (int i = -g->R; i < g->nx + g->R; ++i)
                u[at(g, i, j, -m)] = -u[at(g, i, j, m)];
}

/* Reading R15: p = 0 on the surface plane k = 0. */
static void zero_top(const grid_t *g, double *u)
{
    for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i) u[at(g, i, j, 0)] = 0.0;
}

/* Sec. 3 Laplacian at one point: per axis  sum_m c_am [p(+m) + p(-m) - 2p]. */
static inline double lap_at(const grid_t *g, const double *u, long o,
                            const double *cx, const double *cy, const double *cz)
{
    const double p = u[o];
    double lx = 0.0, ly = 0.0, lz = 0.0;
    for (int m = 1; m <= g->R; ++m) {
        lx += cx[m] * (u[o + m] + u[o - m] - 2.0 * p);
        ly += cy[m] * (u[o + m * g->sy] + u[o - m * g->sy] - 2.0 * p);
        lz += cz[m] * (u[o + m * g->sz] + u[o - m * g->sz] - 2.0 * p);
    }
    return lx + ly + lz;
}

/* coef: NULL for the Taylor weights of the order, else c_1..c_R (unit spacing). */
static int axis_weights(int order, const double *coef, double hx, double hy, double hz,
                        double *cx, double *cy, double *cz)
{
    double c[ORC_MAX_R + 1];
    if (orc_fd_coeffs(order, c) != 0) return -1;
    if (coef) {
        double sum = 0.0;
        for (int m = 1; m <= order / 2; ++m) { c[m] = coef[m - 1]; sum += c[m]; }
        c[0] = -2.0 * sum;
    }
    for (int m = 0; m <= order / 2; ++m) {
        cx[m] = c[m] / (hx * hx);
        cy[m] = c[m] / (hy * hy);
        cz[m] = c[m] / (hz * hz);
    }
    return 0;
}

/* Sec. 3 Laplacian of a whole field u [nz][ny][nx] into out, u = 0 outside. */
int orc_laplacian(int nx, int ny, int nz, double hx, double hy, double hz, int order,
                  const double *u, double *out, int free_surface, const double *coef)
{
    if (nx < 1 || ny < 1 || nz < 1 || !u || !out) return -1;
    double cx[ORC_MAX_R + 1], cy[ORC_MAX_R + 1], cz[ORC_MAX_R + 1];
    if (axis_weights(order, coef, hx, hy, hz, cx, cy, cz) != 0) return -1;
    const grid_t g = make_grid(nx, ny, nz, order / 2);
    double *pu = padded_zeros(&g);
    if (!pu) return -3;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                pu[at(&g, i, j, k)] = u[((long)k * ny + j) * nx + i];
    if (free_surface) mirror_top(&g, pu);
    #pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                out[((long)k * ny + j) * nx + i] = lap_at(&g, pu, at(&g, i, j, k), cx, cy, cz);
    free(pu);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Forward modelling: Alg. 1 with the wavefield solution step of Alg. 2.    */
/*                                                                          */
/* vel      [nz][ny][nx] FP32 velocities (m/s), promoted to FP64 here       */
/* src_ijk  [nsrc][3] grid indices, wavelet [nsrc][nt] FP32                 */
/* rec_ijk  [nrec][3] grid indices, traces [nt][nrec] FP64 output           */
/* u_prev0, u_cur0   optional initial u^{-1}, u^0 ([nz][ny][nx]); NULL = 0  */
/* u_prev_out, u_cur_out  optional final u^{nt-1}, u^{nt}                   */
/* nthreads  OpenMP threads, 0 = runtime default                            */
/* Returns 0, or a negative code for bad arguments / no memory.             */
/* ------------------------------------------------------------------------ */
int orc_forward(int nx, int ny, int nz, double hx, double hy, double hz,
                double dt, int nt, int order, int nbl, double refl,
                const float *vel,
                int nsrc, const int *src_ijk, const float *wavelet,
                int nrec, const int *rec_ijk, double *traces,
                const double *u_prev0, const double *u_cur0,
                double *u_prev_out, double *u_cur_out, int nthreads, int free_surface,
                const double *coef)
{
    if (nx < 1 || ny < 1 || nz < 1 || nt < 0 || dt <= 0 || !vel) return -1;
    if (hx <= 0 || hy <= 0 || hz <= 0) return -1;
    if (free_surface && nz <= order / 2) return -1;
    if (2 * nbl > nx || 2 * nbl > ny || 2 * nbl > nz || nbl < 0) return -1;
    if (nsrc < 0 || nrec < 0 || (nsrc > 0 && (!src_ijk || !wavelet))) return -1;
    if (nrec > 0 && (!rec_ijk || !traces)) return -1;
    for (int s = 0; s < nsrc; ++s) {
        const int *p = src_ijk + 3 * s;
        if (p[0] < 0 || p[0] >= nx || p[1] < 0 || p[1] >= ny || p[2] < 0 || p[2] >= nz) return -1;
    }
    for (int r = 0; r < nrec; ++r) {
        const int *p = rec_ijk + 3 * r;
        if (p[0] < 0 || p[0] >= nx || p[1] < 0 || p[1] >= ny || p[2] < 0 || p[2] >= nz) return -1;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    double cx[ORC_MAX_R + 1], cy[ORC_MAX_R + 1], cz[ORC_MAX_R + 1];
    if (axis_weights(order, coef, hx, hy, hz, cx, cy, cz) != 0) return -1;
    const grid_t g = make_grid(nx, ny, nz, order / 2);
    const long N = (long)nx * ny * nz;

    /* c = dt^2 v^2 (Eq. 5) and the model maximum used by reading R3. */
    double vmax = 0.0;
    for (long q = 0; q < N; ++q) if ((double)vel[q] > vmax) vmax = (double)vel[q];
    double *ex = (double *)malloc(sizeof(double) * nx);
    double *ey = (double *)malloc(sizeof(double) * ny);
    double *ez = (double *)malloc(sizeof(double) * nz);
    double *C = padded_zeros(&g), *ua = padded_zeros(&g), *ub = padded_zeros(&g), *uc = padded_zeros(&g);
    int rc = 0;
    if (!ex || !ey || !ez || !C || !ua || !ub || !uc) { rc = -3; goto done; }
    if (orc_damping_profile(nx, nbl, hx, vmax, refl, ex) || orc_damping_profile(ny, nbl, hy, vmax, refl, ey) ||
        orc_damping_profile(nz, nbl, hz, vmax, refl, ez)) { rc = -1; goto done; }
    if (free_surface)   /* reading R15: no absorbing layer under the free surface */
        for (int k = 0; k < nbl && k < nz - 1 - nbl; ++k) ez[k] = 0.0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long q = ((long)k * ny + j) * nx + i;
                const double v = (double)vel[q];
                C[at(&g, i, j, k)] = dt * dt * v * v;
                if (u_prev0) ua[at(&g, i, j, k)] = u_prev0[q];
                if (u_cur0) ub[at(&g, i, j, k)] = u_cur0[q];
            }
    if (free_surface) { zero_top(&g, ua); zero_top(&g, ub); }

    /* Alg. 2 region bounds: inner = [x3,x4] x [y3,y4] x [z3,z4]. */
    const int x3 = nbl, x4 = nx - 1 - nbl, y3 = nbl, y4 = ny - 1 - nbl, z3 = nbl, z4 = nz - 1 - nbl;
    const double cell = hx * hy * hz;
    double *up = ua, *ucur = ub, *un = uc;   /* u^{n-1}, u^n, u^{n+1} */

    for (int n = 0; n < nt; ++n) {          /* Alg. 1 time loop */
        if (free_surface) mirror_top(&g, ucur);
        #pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const long o = at(&g, i, j, k);
                    const double L = lap_at(&g, ucur, o, cx, cy, cz);
                    const int inner = i >= x3 && i <= x4 && j >= y3 && j <= y4 && k >= z3 && k <= z4;
                    if (inner) {
                        /* Eq. 5 solved for p^{n+1} (its right-hand side is added below). */
                        un[o] = 2.0 * ucur[o] - up[o] + C[o] * L;
                    } else {
                        /* Damping regions of Alg. 2, reading R3. */
                        const double e = (ex[i] + ey[j] + ez[k]) * dt;
                        un[o] = (2.0 * ucur[o] - (1.0 - e) * up[o] + C[o] * L) / (1.0 + e);
                    }
                }
        /* Alg. 1: add the source term of Eq. 5's right-hand side (reading R5). */
        for (int s = 0; s < nsrc; ++s) {
            const int *p = src_ijk + 3 * s;
            const long o = at(&g, p[0], p[1], p[2]);
            const double e = (ex[p[0]] + ey[p[1]] + ez[p[2]]) * dt;
            un[o] += C[o] * (double)wavelet[(long)s * nt + n] / (cell * (1.0 + e));
        }
        if (free_surface) zero_top(&g, un);
        /* Reading R7: receivers sample u^{n+1}. */
        for (int r = 0; r < nrec; ++r) {
            const int *p = rec_ijk + 3 * r;
            traces[(long)n * nrec + r] = un[at(&g, p[0], p[1], p[2])];
        }
        double *t = up; up = ucur; ucur = un; un = t;
    }

    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long q = ((long)k * ny + j) * nx + i;
                if (u_prev_out) u_prev_out[q] = up[at(&g, i, j, k)];
                if (u_cur_out) u_cur_out[q] = ucur[at(&g, i, j, k)];
            }
done:
    free(ex); free(ey); free(ez); free(C); free(ua); free(ub); free(uc);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Reading R17: CPML forward run.  Memory variables are full padded volumes */
/* (zero where the profiles vanish).  Arguments as orc_forward; f0 sets the */
/* frequency shift alpha_max = pi f0 (0: none).                             */
/* ------------------------------------------------------------------------ */
static const double orc_d1[5] = {0.0, 4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0};
static int check_positions(int nx, int ny, int nz, int n, const int *ijk);

/* CPML coefficients b, g of one axis (n cells, L per face; the top face of z
 * is dropped when top_free). */
static void cpml_profile(int n, int L, double h, double vmax, double refl, double f0, double dt, int top_free,
                         double *b, double *g)
{
    const double d0 = L > 0 ? 3.0 * vmax * log(1.0 / refl) / (2.0 * L * h) : 0.0;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        int x = 0;
        if (!top_free && L - i > x) x = L - i;
        if (i - (n - 1 - L) > x) x = i - (n - 1 - L);
        if (L == 0 || x == 0) { b[i] = 1.0; g[i] = 0.0; continue; }
        const double s = (double)x / L;
        const double d = d0 * s * s, alpha = pi * f0 * (1.0 - s);
        b[i] = exp(-(d + alpha) * dt);
        g[i] = d * (b[i] - 1.0) / (d + alpha);
    }
}

int orc_forward_cpml(int nx, int ny, int nz, double hx, double hy, double hz,
                     double dt, int nt, int nbl, double refl, double f0,
                     const float *vel,
                     int nsrc, const int *src_ijk, const float *wavelet,
                     int nrec, const int *rec_ijk, double *traces,
                     double *u_cur_out, int nthreads, int free_surface)
{
    const int order = 8, R = 4;
    if (nx < 1 || ny < 1 || nz < 1 || nt < 0 || dt <= 0 || !vel || f0 < 0) return -1;
    if (hx <= 0 || hy <= 0 || hz <= 0) return -1;
    if (2 * nbl > nx || 2 * nbl > ny || 2 * nbl > nz || nbl < 0) return -1;
    if (nbl > 0 && !(refl > 0.0 && refl < 1.0)) return -1;
    if (free_surface && nz <= R) return -1;
    if (nsrc < 0 || nrec < 0 || (nsrc > 0 && (!src_ijk || !wavelet)) || (nrec > 0 && (!rec_ijk || !traces)))
        return -1;
    if (check_positions(nx, ny, nz, nsrc, src_ijk) || check_positions(nx, ny, nz, nrec, rec_ijk)) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    double cx[ORC_MAX_R + 1], cy[ORC_MAX_R + 1], cz[ORC_MAX_R + 1];
    if (axis_weights(order, NULL, hx, hy, hz, cx, cy, cz) != 0) return -1;
    const grid_t g = make_grid(nx, ny, nz, R);
    const long N = (long)nx * ny * nz;
    double vmax = 0.0;
    for (long q = 0; q < N; ++q) if ((double)vel[q] > vmax) vmax = (double)vel[q];
    double *bx = malloc(sizeof(double) * nx), *gx = malloc(sizeof(double) * nx);
    double *by = malloc(sizeof(double) * ny), *gy = malloc(sizeof(double) * ny);
    double *bz = malloc(sizeof(double) * nz), *gz = malloc(sizeof(double) * nz);
    double *C = padded_zeros(&g), *ua = padded_zeros(&g), *ub = padded_zeros(&g), *uc = padded_zeros(&g);
    double *psi[3], *zeta[3];
    int rc = 0;
    for (int a = 0; a < 3; ++a) { psi[a] = padded_zeros(&g); zeta[a] = padded_zeros(&g); }
    if (!bx || !gx || !by || !gy || !bz || !gz || !C || !ua || !ub || !uc) { rc = -3; goto done; }
    for (int a = 0; a < 3; ++a) if (!psi[a] || !zeta[a]) { rc = -3; goto done; }
    cpml_profile(nx, nbl, hx, vmax, refl, f0, dt, 0, bx, gx);
    cpml_profile(ny, nbl, hy, vmax, refl, f0, dt, 0, by, gy);
    cpml_profile(nz, nbl, hz, vmax, refl, f0, dt, free_surface, bz, gz);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const double v = (double)vel[((long)k * ny + j) * nx + i];
                C[at(&g, i, j, k)] = dt * dt * v * v;
            }
    const double cell = hx * hy * hz;
    const long stride[3] = {1, g.sy, g.sz};
    const double hh[3] = {hx, hy, hz};
    const double *cw[3] = {cx, cy, cz};
    double *up = ua, *ucur = ub, *un = uc;
    for (int n = 0; n < nt; ++n) {
        if (free_surface) mirror_top(&g, ucur);
        /* pass 1: psi_a^n = b psi_a^{n-1} + g D1_a u^n wherever the profile is on */
        #pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const long o = at(&g, i, j, k);
                    const int idx[3] = {i, j, k};
                    const double *B[3] = {bx, by, bz}, *G[3] = {gx, gy, gz};
                    for (int a = 0; a < 3; ++a) {
                        const double gg = G[a][idx[a]];
                        if (gg == 0.0) continue;
                        double d1 = 0.0;
                        for (int m = 1; m <= R; ++m) d1 += orc_d1[m] * (ucur[o + m * stride[a]] - ucur[o - m * stride[a]]);
                        psi[a][o] = B[a][idx[a]] * psi[a][o] + gg * d1 / hh[a];
                    }
                }
        /* pass 2: zeta_a^n and u^{n+1} */
        #pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const long o = at(&g, i, j, k);
                    const int idx[3] = {i, j, k};
                    const double *B[3] = {bx, by, bz}, *G[3] = {gx, gy, gz};
                    double total = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        double d2 = 0.0;
                        for (int m = 1; m <= R; ++m)
                            d2 += cw[a][m] * (ucur[o + m * stride[a]] + ucur[o - m * stride[a]] - 2.0 * ucur[o]);
                        const double gg = G[a][idx[a]];
                        if (gg == 0.0) { total += d2; continue; }
                        double dpsi = 0.0;
                        for (int m = 1; m <= R; ++m)
                            dpsi += orc_d1[m] * (psi[a][o + m * stride[a]] - psi[a][o - m * stride[a]]);
                        dpsi /= hh[a];
                        zeta[a][o] = B[a][idx[a]] * zeta[a][o] + gg * (d2 + dpsi);
                        total += d2 + dpsi + zeta[a][o];
                    }
                    un[o] = 2.0 * ucur[o] - up[o] + C[o] * total;
                }
        for (int s = 0; s < nsrc; ++s) {
            const int *p = src_ijk + 3 * s;
            const long o = at(&g, p[0], p[1], p[2]);
            un[o] += C[o] * (double)wavelet[(long)s * nt + n] / cell;
        }
        if (free_surface) zero_top(&g, un);
        for (int r = 0; r < nrec; ++r) {
            const int *p = rec_ijk + 3 * r;
            traces[n * (long)nrec + r] = un[at(&g, p[0], p[1], p[2])];   /* reading R7 */
        }
        double *t = up; up = ucur; ucur = un; un = t;
    }
    if (u_cur_out)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) u_cur_out[((long)k * ny + j) * nx + i] = ucur[at(&g, i, j, k)];
done:
    free(bx); free(gx); free(by); free(gy); free(bz); free(gz);
    free(C); free(ua); free(ub); free(uc);
    for (int a = 0; a < 3; ++a) { free(psi[a]); free(zeta[a]); }
    return rc;
}

/* Threads the OpenMP runtime would use (1 without OpenMP). */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the forward map w -> traces (transpose of Alg. 1 with the     */
/* readings above).  Writing the forward step as                            */
/*   D u^{n+1} = 2 u^n - E u^{n-1} + C (L u^n + s^n),  d^n = R u^{n+1},     */
/* D = 1 + e, E = 1 - e, C = dt^2 v^2, s^n = S w^n / (hx hy hz), the        */
/* transpose runs backward from mu^{nt+1} = mu^{nt+2} = 0:                  */
/*   D mu^n = 2 mu^{n+1} - E mu^{n+2} + L (C mu^{n+1}) + R^T r^{n-1}        */
/* for n = nt .. 1, and the adjoint source is                               */
/*   a[s][n-1] = C(x_s) mu^n(x_s) / (hx hy hz).                             */
/* L is symmetric (u = 0 outside), so L^T = L.                              */
/* resid [nt][nrec] FP64 in; adj [nsrc][nt] FP64 out.                       */
/* If grad_c != NULL it also needs u_hist = u^{-1} .. u^{nt} (nt+2 padded   */
/* volumes, as produced by orc_forward_history) and accumulates the         */
/* gradient of J = 1/2 sum |d - d_obs|^2 with respect to c:                 */
/*   dJ/dc(x) = sum_{n=1..nt} mu^n(x) (L u^{n-1} + s^{n-1})(x).             */
/* ------------------------------------------------------------------------ */
static int adjoint_core(int nx, int ny, int nz, double hx, double hy, double hz,
                        double dt, int nt, int order, int nbl, double refl,
                        const float *vel, int nsrc, const int *src_ijk, const float *wavelet,
                        int nrec, const int *rec_ijk, const double *resid, double *adj,
                        double *const *u_hist, double *grad_c, int free_surface)
{
    double cx[ORC_MAX_R + 1], cy[ORC_MAX_R + 1], cz[ORC_MAX_R + 1];
    if (axis_weights(order, NULL, hx, hy, hz, cx, cy, cz) != 0) return -1;
    const grid_t g = make_grid(nx, ny, nz, order / 2);
    const long N = (long)nx * ny * nz;
    double vmax = 0.0;
    for (long q = 0; q < N; ++q) if ((double)vel[q] > vmax) vmax = (double)vel[q];
    double *ex = (double *)malloc(sizeof(double) * nx);
    double *ey = (double *)malloc(sizeof(double) * ny);
    double *ez = (double *)malloc(sizeof(double) * nz);
    double *C = padded_zeros(&g), *m0 = padded_zeros(&g), *m1 = padded_zeros(&g), *m2 = padded_zeros(&g);
    double *cm = padded_zeros(&g);
    int rc = 0;
    if (!ex || !ey || !ez || !C || !m0 || !m1 || !m2 || !cm) { rc = -3; goto done; }
    if (orc_damping_profile(nx, nbl, hx, vmax, refl, ex) || orc_damping_profile(ny, nbl, hy, vmax, refl, ey) ||
        orc_damping_profile(nz, nbl, hz, vmax, refl, ez)) { rc = -1; goto done; }
    if (free_surface)
        for (int k = 0; k < nbl && k < nz - 1 - nbl; ++k) ez[k] = 0.0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const double v = (double)vel[((long)k * ny + j) * nx + i];
                C[at(&g, i, j, k)] = dt * dt * v * v;
            }
    const double cell = hx * hy * hz;
    /* m1 = mu^{n+1}, m2 = mu^{n+2}, m0 receives mu^n */
    for (int n = nt; n >= 1; --n) {
        #pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const long o = at(&g, i, j, k);
                    cm[o] = C[o] * m1[o];
                }
        if (free_surface) mirror_top(&g, cm);   /* the restricted L is symmetric: L^T = L */
        #pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const long o = at(&g, i, j, k);
                    const double e = (ex[i] + ey[j] + ez[k]) * dt;
                    m0[o] = (2.0 * m1[o] - (1.0 - e) * m2[o] + lap_at(&g, cm, o, cx, cy, cz)) / (1.0 + e);
                }
        for (int r = 0; r < nrec; ++r) {          /* R^T r^{n-1}, inside the division */
            const int *p = rec_ijk + 3 * r;
            const long o = at(&g, p[0], p[1], p[2]);
            const double e = (ex[p[0]] + ey[p[1]] + ez[p[2]]) * dt;
            m0[o] += resid[(long)(n - 1) * nrec + r] / (1.0 + e);
        }
        if (free_surface) zero_top(&g, m0);     /* the transpose of the surface projection */
        for (int s = 0; s < nsrc; ++s) {
            const int *p = src_ijk + 3 * s;
            const long o = at(&g, p[0], p[1], p[2]);
            if (adj) adj[(long)s * nt + (n - 1)] = C[o] * m0[o] / cell;
        }
        if (grad_c) {
            /* term of forward step n-1: mu^n (L u^{n-1} + s^{n-1}); u_hist[m+1] = u^m */
            const double *u = u_hist[n];   /* u^{n-1} */
            if (free_surface) mirror_top(&g, u_hist[n]);
            #pragma omp parallel for collapse(2) schedule(static)
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        const long o = at(&g, i, j, k);
                        grad_c[((long)k * ny + j) * nx + i] += m0[o] * lap_at(&g, u, o, cx, cy, cz);
                    }
            for (int s = 0; s < nsrc; ++s) {
                const int *p = src_ijk + 3 * s;
                const long o = at(&g, p[0], p[1], p[2]);
                grad_c[((long)p[2] * ny + p[1]) * nx + p[0]] += m0[o] * (double)wavelet[(long)s * nt + (n - 1)] / cell;
            }
        }
        double *t = m2; m2 = m1; m1 = m0; m0 = t;
    }
done:
    free(ex); free(ey); free(ez); free(C); free(m0); free(m1); free(m2); free(cm);
    return rc;
}

static int check_positions(int nx, int ny, int nz, int n, const int *ijk)
{
    for (int s = 0; s < n; ++s) {
        const int *p = ijk + 3 * s;
        if (p[0] < 0 || p[0] >= nx || p[1] < 0 || p[1] >= ny || p[2] < 0 || p[2] >= nz) return -1;
    }
    return 0;
}

int orc_adjoint(int nx, int ny, int nz, double hx, double hy, double hz,
                double dt, int nt, int order, int nbl, double refl, const float *vel,
                int nsrc, const int *src_ijk, int nrec, const int *rec_ijk,
                const double *resid, double *adj, int nthreads, int free_surface)
{
    if (nx < 1 || ny < 1 || nz < 1 || nt < 0 || dt <= 0 || !vel || nsrc < 0 || nrec < 0) return -1;
    if (free_surface && nz <= order / 2) return -1;
    if (2 * nbl > nx || 2 * nbl > ny || 2 * nbl > nz || nbl < 0) return -1;
    if ((nsrc && (!src_ijk || !adj)) || (nrec && (!rec_ijk || !resid))) return -1;
    if (check_positions(nx, ny, nz, nsrc, src_ijk) || check_positions(nx, ny, nz, nrec, rec_ijk)) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    return adjoint_core(nx, ny, nz, hx, hy, hz, dt, nt, order, nbl, refl, vel, nsrc, src_ijk, NULL,
                        nrec, rec_ijk, resid, adj, NULL, NULL, free_surface);
}

/* Gradient of J = 1/2 sum_n |R u^{n+1} - d_obs^n|^2 with respect to the
 * velocity, for the residual resid = R u^{n+1} - d_obs^n given by the caller:
 *   dJ/dv(x) = 2 dt^2 v(x) dJ/dc(x)  (c = dt^2 v^2).
 * Runs the forward storing every state u^{-1} .. u^{nt} (small grids only),
 * then the adjoint recurrence of orc_adjoint.  grad_v [nz][ny][nx] FP64. */
int orc_gradient(int nx, int ny, int nz, double hx, double hy, double hz,
                 double dt, int nt, int order, int nbl, double refl, const float *vel,
                 int nsrc, const int *src_ijk, const float *wavelet,
                 int nrec, const int *rec_ijk, const double *resid, double *grad_v, int nthreads,
                 int free_surface)
{
    if (free_surface && nz <= order / 2) return -1;
    if (nx < 1 || ny < 1 || nz < 1 || nt < 0 || dt <= 0 || !vel || !grad_v || nsrc < 0 || nrec < 0) return -1;
    if (2 * nbl > nx || 2 * nbl > ny || 2 * nbl > nz || nbl < 0) return -1;
    if ((nsrc && (!src_ijk || !wavelet)) || (nrec && (!rec_ijk || !resid))) return -1;
    if (check_positions(nx, ny, nz, nsrc, src_ijk) || check_positions(nx, ny, nz, nrec, rec_ijk)) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const grid_t g = make_grid(nx, ny, nz, order / 2);
    const long N = (long)nx * ny * nz;
    int rc = 0;
    double **hist = (double **)calloc((size_t)nt + 2, sizeof(double *));
    double *dense = (double *)malloc(sizeof(double) * (size_t)N);
    double *prev = (double *)calloc((size_t)N, sizeof(double));
    double *gc = (double *)calloc((size_t)N, sizeof(double));
    if (!hist || !dense || !prev || !gc) { rc = -3; goto done; }
    for (int m = 0; m < nt + 2; ++m)
        if (!(hist[m] = padded_zeros(&g))) { rc = -3; goto done; }
    /* hist[m+1] = u^m, m = -1 .. nt: one forward step at a time from the last state */
    for (int m = 0; m < nt; ++m) {
        double *cur = dense;
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const long q = ((long)k * ny + j) * nx + i;
                    prev[q] = hist[m][at(&g, i, j, k)];
                    cur[q] = hist[m + 1][at(&g, i, j, k)];
                }
        /* the step m of the full run: u^{m+1} from u^m, u^{m-1} with w[m] */
        float *wm = NULL;
        if (nsrc) {
            wm = (float *)malloc(sizeof(float) * nsrc);
            if (!wm) { rc = -3; goto done; }
            for (int s = 0; s < nsrc; ++s) wm[s] = wavelet[(long)s * nt + m];
        }
        double *up = (double *)malloc(sizeof(double) * (size_t)N), *un = (double *)malloc(sizeof(double) * (size_t)N);
        if (!up || !un) { free(up); free(un); free(wm); rc = -3; goto done; }
        rc = orc_forward(nx, ny, nz, hx, hy, hz, dt, 1, order, nbl, refl, vel, nsrc, src_ijk, wm,
                         0, NULL, NULL, prev, cur, up, un, nthreads, free_surface, NULL);
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i)
                    hist[m + 2][at(&g, i, j, k)] = un[((long)k * ny + j) * nx + i];
        free(up); free(un); free(wm);
        if (rc) goto done;
    }
    rc = adjoint_core(nx, ny, nz, hx, hy, hz, dt, nt, order, nbl, refl, vel, nsrc, src_ijk, wavelet,
                      nrec, rec_ijk, resid, NULL, hist, gc, free_surface);
    if (rc) goto done;
    for (long q = 0; q < N; ++q) grad_v[q] = 2.0 * dt * dt * (double)vel[q] * gc[q];
done:
    if (hist) for (int m = 0; m < nt + 2; ++m) free(hist[m]);
    free(hist); free(dense); free(prev); free(gc);
    return rc;
}

/* ======================================================================== */
/* Reading R18: the first-order variable-density system of Sec. 3 on a      */
/* staggered (Yee) grid.                                                    */
/*                                                                          */
/*   (1/(rho v^2)) p_t - div vel = f,     rho vel_t - grad p = 0            */
/*                                                                          */
/* i.e.  p_t = K (div vel + f),  vel_t = b grad p,  K = rho v^2, b = 1/rho. */
/* p, K, rho live at the grid points (i, j, k); the component along axis a  */
/* lives half a cell further along a (vx[k][j][i] at x = (i + 1/2) hx).     */
/* Leapfrog in time: vel at half steps n - 1/2, p at whole steps n.         */
/*   D+_a p (i + 1/2) = sum_m a_m [p(i + m) - p(i - m + 1)] / h_a           */
/*   D-_a q (i)       = sum_m a_m [q(i + m - 1) - q(i - m)] / h_a           */
/* with the staggered weights a_m below and p = vel = 0 outside the grid    */
/* (reading R2), so that D-_a = -(D+_a)^T.  Buoyancy at a half point is the */
/* mean of b at its two grid points (b at the grid point itself past the    */
/* last one).  The source f = delta(x - x_s) w(t): sample w[n] drives the   */
/* step from p^n to p^{n+1}; receivers record p^{n+1} (reading R7).         */
/*                                                                          */
/* Boundary layers (the grid includes them, reading R4):                    */
/*   damping: p and each component relax at eta = eta_x + eta_y + eta_z    */
/*     taken at their own (possibly half-cell) positions, centred in time:  */
/*       vel_a^{n+1/2} = [(1 - e/2) vel_a^{n-1/2} + dt b_a D+_a p^n]/(1+e/2) */
/*       p^{n+1} = [(1 - e/2) p^n + dt K (sum_a D-_a vel_a^{n+1/2} + s^n)]  */
/*                 / (1 + e/2),     e = dt eta,  s^n = w[n] / (hx hy hz)    */
/*     with the profile of reading R3 at the continuous depth x into the    */
/*     layer (x <= L): eta = eta_max (x/L)^2.                               */
/*   CPML: each derivative gains a memory variable on its axis's layers,    */
/*       psi_a^n = B psi_a^{n-1} + G D+_a p^n      (at vel_a's points)      */
/*       vel_a^{n+1/2} = vel_a^{n-1/2} + dt b_a (D+_a p^n + psi_a^n)        */
/*       phi_a^{n+1/2} = B phi_a^{n-1/2} + G D-_a vel_a^{n+1/2} (at p's)    */
/*       p^{n+1} = p^n + dt K (sum_a (D-_a vel_a + phi_a) + s^n)            */
/*     B = exp(-(d + alpha) dt), G = d (B - 1)/(d + alpha), with d, alpha   */
/*     of reading R17 at the continuous depth x into the layer.             */
/* ======================================================================== */

/* Staggered first-derivative weights of order 2R:
 *   sum_m a_m [f(x + (m - 1/2) h) - f(x - (m - 1/2) h)] = h f'(x) + O(h^{2R+1})
 * exactly when  sum_m 2 (m - 1/2) a_m = 1  and  sum_m (m - 1/2)^{2q+1} a_m = 0,
 * q = 1..R-1 (Taylor expansion of the odd part).  Output a[0] = 0, a[m]. */
int orc_staggered_coeffs(int order, double *a)
{
    if (order < 2 || order % 2 != 0 || order / 2 > ORC_MAX_R || !a) return -1;
    const int R = order / 2;
    double A[ORC_MAX_R][ORC_MAX_R + 1];
    for (int q = 0; q < R; ++q) {
        for (int m = 1; m <= R; ++m) A[q][m - 1] = pow(m - 0.5, 2.0 * q + 1.0);
        A[q][R] = (q == 0) ? 0.5 : 0.0;
    }
    for (int col = 0; col < R; ++col) {
        int piv = col;
        for (int r = col + 1; r < R; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) return -2;
        if (piv != col)
            for (int q = 0; q <= R; ++q) { double t = A[col][q]; A[col][q] = A[piv][q]; A[piv][q] = t; }
        for (int r = 0; r < R; ++r) {
            if (r == col) continue;
            const double f = A[r][col] / A[col][col];
            for (int q = col; q <= R; ++q) A[r][q] -= f * A[col][q];
        }
    }
    a[0] = 0.0;
    for (int m = 1; m <= R; ++m) a[m] = A[m - 1][R] / A[m - 1][m - 1];
    return 0;
}

/* Depth into the layers (cells) of the continuous position x on an axis of
 * n points with L-cell layers, capped at L. */
static double layer_depth(double x, int n, int L, int top_free)
{
    double d = 0.0;
    if (!top_free && L - x > d) d = L - x;
    if (x - (n - 1 - L) > d) d = x - (n - 1 - L);
    return d > L ? (double)L : d;
}

/* Profiles of one axis at the grid points (half = 0) or the half points
 * i + 1/2 (half = 1): damping eta, or the CPML pair B, G. */
static void vd_profile(int n, int L, double h, double vmax, double refl, double f0, double dt, int half,
                       int top_free, double *eta, double *B, double *G)
{
    const double d0 = L > 0 ? 3.0 * vmax * log(1.0 / refl) / (2.0 * L * h) : 0.0;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        const double x = L > 0 ? layer_depth(i + 0.5 * half, n, L, top_free) : 0.0;
        const double s = L > 0 ? x / L : 0.0;
        const double d = d0 * s * s;
        eta[i] = d;
        if (x == 0.0) { B[i] = 1.0; G[i] = 0.0; continue; }
        const double alpha = pi * f0 * (1.0 - s);
        B[i] = exp(-(d + alpha) * dt);
        G[i] = d * (B[i] - 1.0) / (d + alpha);
    }
}

/* Free surface of the staggered system (reading R18 with the surface option
 * of Sec. 3, as reading R15): p = 0 on the plane k = 0.  Above it p and the
 * horizontal velocities are odd images, p(-m) = -p(m); v_z, which sits at
 * the half points k + 1/2, is an even image, v_z(-m) = v_z(m - 1) (index -m
 * is the position -m + 1/2, the mirror of m - 1/2).  Only p is read across
 * the surface by the velocity update and only v_z by the pressure update. */
static void vd_mirror_p(const grid_t *g, double *p)
{
    for (int m = 1; m <= g->R && m < g->nz; ++m)
        for (int j = -g->R; j < g->ny + g->R; ++j)
            for (int i = -g->R; i < g->nx + g->R; ++i)
                p[at(g, i, j, -m)] = -p[at(g, i, j, m)];
}

static void vd_mirror_vz(const grid_t *g, double *vz)
{
    for (int m = 1; m <= g->R && m - 1 < g->nz; ++m)
        for (int j = -g->R; j < g->ny + g->R; ++j)
            for (int i = -g->R; i < g->nx + g->R; ++i)
                vz[at(g, i, j, -m)] = vz[at(g, i, j, m - 1)];
}

/* Forward run of reading R18 (order 8).
 * vel, rho   [nz][ny][nx] FP32 (m/s, kg/m^3)
 * cpml       0: damping layers, 1: CPML with frequency shift alpha_max = pi f0
 * state0     optional [4][nz][ny][nx] initial p^0, vx, vy, vz at -1/2 (NULL = 0)
 * state_out  optional final p^{nt}, vx, vy, vz at nt - 1/2
 * traces     [nt][nrec] FP64: p^{n+1} at the receivers.
 * free_surface  1: p = 0 on k = 0 (images above it), no top layer; the
 *            plane k = 0 of p is set to 0 after every step (sources there
 *            vanish, receivers read 0) and in the initial state. */
int orc_forward_vd(int nx, int ny, int nz, double hx, double hy, double hz,
                   double dt, int nt, int nbl, double refl, int cpml, double f0,
                   const float *vel, const float *rho,
                   int nsrc, const int *src_ijk, const float *wavelet,
                   int nrec, const int *rec_ijk, double *traces,
                   const double *state0, double *state_out, int nthreads, int free_surface)
{
    const int R = 4;
    if (free_surface && nz <= R) return -1;
    if (nx < 1 || ny < 1 || nz < 1 || nt < 0 || dt <= 0 || !vel || !rho || f0 < 0) return -1;
    if (hx <= 0 || hy <= 0 || hz <= 0 || (cpml != 0 && cpml != 1)) return -1;
    if (2 * nbl > nx || 2 * nbl > ny || 2 * nbl > nz || nbl < 0) return -1;
    if (nbl > 0 && !(refl > 0.0 && refl < 1.0)) return -1;
    if (nsrc < 0 || nrec < 0 || (nsrc > 0 && (!src_ijk || !wavelet)) || (nrec > 0 && (!rec_ijk || !traces)))
        return -1;
    if (check_positions(nx, ny, nz, nsrc, src_ijk) || check_positions(nx, ny, nz, nrec, rec_ijk)) return -1;
    const long N = (long)nx * ny * nz;
    for (long q = 0; q < N; ++q) if (!(rho[q] > 0.0f) || !(vel[q] > 0.0f)) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    double aw[ORC_MAX_R + 1];
    if (orc_staggered_coeffs(2 * R, aw) != 0) return -1;
    const grid_t g = make_grid(nx, ny, nz, R);
    const int n3[3] = {nx, ny, nz};
    const double hh[3] = {hx, hy, hz};
    const long stride[3] = {1, g.sy, g.sz};
    double vmax = 0.0;
    for (long q = 0; q < N; ++q) if ((double)vel[q] > vmax) vmax = (double)vel[q];

    int rc = 0;
    double *prof[3][2][3];   /* [axis][half][eta, B, G] */
    for (int a = 0; a < 3; ++a)
        for (int s = 0; s < 2; ++s)
            for (int t = 0; t < 3; ++t) prof[a][s][t] = (double *)malloc(sizeof(double) * n3[a]);
    double *K = padded_zeros(&g), *Bc = padded_zeros(&g), *p = padded_zeros(&g);
    double *v[3], *bh[3], *psi[3], *phi[3];
    for (int a = 0; a < 3; ++a) {
        v[a] = padded_zeros(&g); bh[a] = padded_zeros(&g);
        psi[a] = cpml ? padded_zeros(&g) : NULL; phi[a] = cpml ? padded_zeros(&g) : NULL;
    }
    for (int a = 0; a < 3; ++a) {
        for (int s = 0; s < 2; ++s)
            for (int t = 0; t < 3; ++t) if (!prof[a][s][t]) rc = -3;
        if (!v[a] || !bh[a] || (cpml && (!psi[a] || !phi[a]))) rc = -3;
    }
    if (!K || !Bc || !p) rc = -3;
    if (rc) goto done;
    for (int a = 0; a < 3; ++a)
        for (int s = 0; s < 2; ++s)
            vd_profile(n3[a], nbl, hh[a], vmax, refl, f0, dt, s, a == 2 && free_surface, prof[a][s][0],
                       prof[a][s][1], prof[a][s][2]);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long q = ((long)k * ny + j) * nx + i, o = at(&g, i, j, k);
                const double vv = (double)vel[q], rr = (double)rho[q];
                K[o] = rr * vv * vv;
                Bc[o] = 1.0 / rr;
                if (state0) {
                    p[o] = state0[q];
                    for (int a = 0; a < 3; ++a) v[a][o] = state0[(a + 1) * N + q];
                }
            }
    /* buoyancy at the half points: mean of the two neighbours, or the point's own past the last one */
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const long o = at(&g, i, j, k);
                const int idx[3] = {i, j, k};
                for (int a = 0; a < 3; ++a)
                    bh[a][o] = idx[a] + 1 < n3[a] ? 0.5 * (Bc[o] + Bc[o + stride[a]]) : Bc[o];
            }
    const double cell = hx * hy * hz;
    if (free_surface) zero_top(&g, p);
    for (int n = 0; n < nt; ++n) {
        if (free_surface) vd_mirror_p(&g, p);
        /* particle velocities at n + 1/2 from p^n */
        #pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const long o = at(&g, i, j, k);
                    const int idx[3] = {i, j, k};
                    for (int a = 0; a < 3; ++a) {
                        double dp = 0.0;
                        for (int m = 1; m <= R; ++m)
                            dp += aw[m] * (p[o + m * stride[a]] - p[o - (m - 1) * stride[a]]);
                        dp /= hh[a];
                        if (cpml) {
                            const double Gc = prof[a][1][2][idx[a]];
                            if (Gc != 0.0) {
                                psi[a][o] = prof[a][1][1][idx[a]] * psi[a][o] + Gc * dp;
                                dp += psi[a][o];
                            }
                            v[a][o] += dt * bh[a][o] * dp;
                        } else {
                            double eta = 0.0;
                            for (int c = 0; c < 3; ++c) eta += prof[c][c == a][0][idx[c]];
                            const double e = dt * eta;
                            v[a][o] = ((1.0 - 0.5 * e) * v[a][o] + dt * bh[a][o] * dp) / (1.0 + 0.5 * e);
                        }
                    }
                }
        if (free_surface) vd_mirror_vz(&g, v[2]);
        /* pressure at n + 1 from the velocities at n + 1/2 */
        #pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const long o = at(&g, i, j, k);
                    const int idx[3] = {i, j, k};
                    double div = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        double dv = 0.0;
                        for (int m = 1; m <= R; ++m)
                            dv += aw[m] * (v[a][o + (m - 1) * stride[a]] - v[a][o - m * stride[a]]);
                        dv /= hh[a];
                        if (cpml) {
                            const double Gc = prof[a][0][2][idx[a]];
                            if (Gc != 0.0) {
                                phi[a][o] = prof[a][0][1][idx[a]] * phi[a][o] + Gc * dv;
                                dv += phi[a][o];
                            }
                        }
                        div += dv;
                    }
                    if (cpml) {
                        p[o] += dt * K[o] * div;
                    } else {
                        const double e = dt * (prof[0][0][0][i] + prof[1][0][0][j] + prof[2][0][0][k]);
                        p[o] = ((1.0 - 0.5 * e) * p[o] + dt * K[o] * div) / (1.0 + 0.5 * e);
                    }
                }
        for (int s = 0; s < nsrc; ++s) {
            const int *q = src_ijk + 3 * s;
            const long o = at(&g, q[0], q[1], q[2]);
            const double e = cpml ? 0.0 : dt * (prof[0][0][0][q[0]] + prof[1][0][0][q[1]] + prof[2][0][0][q[2]]);
            p[o] += dt * K[o] * (double)wavelet[(long)s * nt + n] / (cell * (1.0 + 0.5 * e));
        }
        if (free_surface) zero_top(&g, p);
        for (int r = 0; r < nrec; ++r) {
            const int *q = rec_ijk + 3 * r;
            traces[n * (long)nrec + r] = p[at(&g, q[0], q[1], q[2])];
        }
    }
    if (state_out)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const long q = ((long)k * ny + j) * nx + i, o = at(&g, i, j, k);
                    state_out[q] = p[o];
                    for (int a = 0; a < 3; ++a) state_out[(a + 1) * N + q] = v[a][o];
                }
done:
    for (int a = 0; a < 3; ++a) {
        for (int s = 0; s < 2; ++s)
            for (int t = 0; t < 3; ++t) free(prof[a][s][t]);
        free(v[a]); free(bh[a]); free(psi[a]); free(phi[a]);
    }
    free(K); free(Bc); free(p);
    return rc;
}
