/*
 * pfasst_oracle.c -- plain FP64 CPU oracle for SDC / multigrid / two-level PFASST.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference
 * that the CUDA library is checked against.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product path never does.
 * It shares no code, header or constant table with the CUDA library.
 *
 * Everything is written in the notation of "Interweaving PFASST and Parallel
 * Multigrid" (Minion, Speck, Bolten, Emmett, Ruprecht):
 *   - collocation / integration matrix Q .................. Sec. 2.1, Eq. (collocation), (collocationM)
 *   - SDC sweep with backward-Euler sub-steps ............. Sec. 2.2, Eq. (sdc-be)
 *   - compact sub-step equation (I - dt_m A) y = rhs ....... Sec. 2.2.2, Eq. (SDCcompactLIII)
 *   - collocation residual ................................ Sec. 2.2.2, Eq. (resid)
 *   - MLSDC / FAS correction .............................. Sec. 2.3
 *   - PFASST predictor, send-forward, coarse chain ........ Sec. 2.4
 *   - heat equation, 2nd-order FD, Dirichlet 0 ............ Sec. 4.1
 *   - geometric multigrid V-cycle (linear interpolation,
 *     full weighting, Jacobi / Gauss-Seidel smoothing) .... Sec. 4.1.1, 4.1.2, 4.2.1
 *   - 4th-order spatial interpolation, point-wise
 *     restriction in space and time between PFASST levels  Sec. 4.2.1
 * Equations are named by their labels in the paper's source.
 * Where the paper defers to other work (the FAS formula, the PFASST schedule,
 * the MG stopping rule) the reading used here is stated at the function.
 *
 * Arrays: a grid function on a d-dimensional grid with n interior points per
 * axis is stored as n^d doubles, x fastest ([z][y][x]); the zero Dirichlet
 * values on the walls are not stored.  Mesh width h = 1/(n+1).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Number of OpenMP threads the oracle's grid loops use (the CPU-baseline timings run it
 * single-threaded and on all cores); returns the count in effect. */
int orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

#define ORC_MAXS 16

/* ------------------------------------------------------------------------- */
/* Quadrature nodes and integration matrix (Sec. 2.1)                        */
/* ------------------------------------------------------------------------- */

/* Legendre polynomial P_N and its first two derivatives at x (long double). */
static void legendre(int N, long double x, long double *p, long double *dp, long double *d2p)
{
    long double p0 = 1.0L, p1 = x;
    if (N == 0) { *p = 1.0L; *dp = 0.0L; *d2p = 0.0L; return; }
    for (int k = 2; k <= N; ++k) {
        long double pk = ((2.0L * k - 1.0L) * x * p1 - (k - 1.0L) * p0) / k;
        p0 = p1;
        p1 = pk;
    }
    /* p1 = P_N, p0 = P_{N-1};  (1-x^2) P_N' = N (P_{N-1} - x P_N)
       (1-x^2) P_N'' = 2x P_N' - N(N+1) P_N  (Legendre's equation)        */
    long double w = 1.0L - x * x;
    *p = p1;
    *dp = N * (p0 - x * p1) / w;
    *d2p = (2.0L * x * (*dp) - N * (N + 1.0L) * p1) / w;
}

/* Gauss-Lobatto nodes on [0,1]: the two endpoints and the roots of P'_{s-1},
 * found by Newton's method from Chebyshev-Lobatto starting points. */
int orc_gauss_lobatto(int s, double *tau)
{
    if (s < 2 || s > ORC_MAXS) return -1;
    int N = s - 1;
    tau[0] = 0.0;
    tau[N] = 1.0;
    for (int j = 1; j < N; ++j) {
        long double x = -cosl(3.14159265358979323846264338327950288L * j / N);
        for (int it = 0; it < 100; ++it) {
            long double p, dp, d2p;
            legendre(N, x, &p, &dp, &d2p);
            long double dx = dp / d2p;
            x -= dx;
            if (fabsl(dx) < 1e-30L) break;
        }
        tau[j] = (double)((x + 1.0L) / 2.0L);
    }
    return 0;
}

/* Node families: 0 = Gauss-Lobatto (the workloads'), 1 = uniform nodes tau_m = m/M whose
 * quadrature rule does not use the left endpoint (Sec. 3: the paper's second- and
 * fourth-order methods; M = 1 is backward Euler). */
int orc_nodes(int s, int family, double *tau)
{
    if (s < 2 || s > ORC_MAXS) return -1;
    if (family == 0) return orc_gauss_lobatto(s, tau);
    if (family != 1) return -1;
    for (int m = 0; m < s; ++m) tau[m] = (double)m / (double)(s - 1);
    return 0;
}

/* Q[m][j] = integral from 0 to tau_m of the Lagrange basis polynomial l_j
 * (Sec. 2.1: q_{m,i} chosen for the highest order; first row is zero).
 * The basis polynomial is expanded in monomials and integrated exactly.  With
 * first = 1 the interpolation nodes are tau_1..tau_{s-1} (the rule without the left
 * endpoint) and column 0 is zero. */
static int qmatrix_from(int s, int first, const double *tau, double *Q)
{
    if (s < 2 || s > ORC_MAXS) return -1;
    for (int m = 0; m < s; ++m) Q[m * s] = 0.0;
    for (int j = first; j < s; ++j) {
        long double c[ORC_MAXS + 1];
        memset(c, 0, sizeof c);
        c[0] = 1.0L;
        int deg = 0;
        for (int i = first; i < s; ++i) {
            if (i == j) continue;
            long double den = (long double)tau[j] - (long double)tau[i];
            /* multiply c(x) by (x - tau_i)/den */
            for (int k = deg + 1; k >= 1; --k)
                c[k] = (c[k - 1] - (long double)tau[i] * c[k]) / den;
            c[0] = (-(long double)tau[i] * c[0]) / den;
            ++deg;
        }
        for (int m = 0; m < s; ++m) {
            long double t = tau[m], tp = t, acc = 0.0L;
            for (int k = 0; k <= deg; ++k) {
                acc += c[k] * tp / (k + 1);
                tp *= t;
            }
            Q[m * s + j] = (double)acc;
        }
    }
    return 0;
}

int orc_qmatrix(int s, const double *tau, double *Q) { return qmatrix_from(s, 0, tau, Q); }

int orc_qmatrix_family(int s, int family, const double *tau, double *Q)
{
    if (family != 0 && family != 1) return -1;
    return qmatrix_from(s, family == 1 ? 1 : 0, tau, Q);
}

/* Lagrange interpolation weights from nodes tc[0..sc) to the point t. */
static void lagrange_weights(int sc, const double *tc, double t, double *w)
{
    for (int j = 0; j < sc; ++j) {
        long double v = 1.0L;
        for (int i = 0; i < sc; ++i)
            if (i != j) v *= ((long double)t - tc[i]) / ((long double)tc[j] - tc[i]);
        w[j] = (double)v;
    }
}

void orc_lagrange_weights(int sc, const double *tc, double t, double *w) { lagrange_weights(sc, tc, t, w); }

/* ------------------------------------------------------------------------- */
/* Grid functions and the 2nd-order FD Laplacian (Sec. 4.1)                  */
/* ------------------------------------------------------------------------- */

static size_t npts(int dim, int n)
{
    size_t N = (size_t)n;
    if (dim >= 2) N *= (size_t)n;
    if (dim >= 3) N *= (size_t)n;
    return N;
}

/* extent of axis a (x=0, y=1, z=2): n if the axis exists, else 1 */
static int ext(int dim, int n, int a) { return a < dim ? n : 1; }

/* value at 0-based (i,j,k); zero outside the interior (Dirichlet 0) */
static double at(const double *u, int dim, int n, int i, int j, int k)
{
    if (i < 0 || i >= ext(dim, n, 0)) return 0.0;
    if (j < 0 || j >= ext(dim, n, 1)) return 0.0;
    if (k < 0 || k >= ext(dim, n, 2)) return 0.0;
    return u[((size_t)k * ext(dim, n, 1) + j) * ext(dim, n, 0) + i];
}

/* sum over existing axes of the two neighbours of point (i,j,k) */
static double nbsum(const double *u, int dim, int n, int i, int j, int k)
{
    double s = at(u, dim, n, i - 1, j, k) + at(u, dim, n, i + 1, j, k);
    if (dim >= 2) s += at(u, dim, n, i, j - 1, k) + at(u, dim, n, i, j + 1, k);
    if (dim >= 3) s += at(u, dim, n, i, j, k - 1) + at(u, dim, n, i, j, k + 1);
    return s;
}

/* Fourth-order Laplacian (Sec. 4.2 uses a fourth-order stencil; reading g23): per axis
 * (-u_{i-2} + 16 u_{i-1} - 30 u_i + 16 u_{i+1} - u_{i+2}) / (12 dx^2).  The wall value is
 * 0, and the one point beyond it that the stencil reaches takes the odd reflection
 * -u of its mirror image (0-based index -2 mirrors 0, index n+1 mirrors n-1), which
 * keeps every sine mode an eigenvector. */
static double at_odd(const double *u, int dim, int n, int a, int i, int j, int k, int q)
{
    int len = ext(dim, n, a), sign = 1;
    if (q == -1 || q == len) return 0.0;
    if (q < -1) { q = -2 - q; sign = -1; }
    if (q > len) { q = 2 * len - q; sign = -1; }
    if (a == 0) return sign * at(u, dim, n, q, j, k);
    if (a == 1) return sign * at(u, dim, n, i, q, k);
    return sign * at(u, dim, n, i, j, q);
}

/* h^2 Lap_h u at (i,j,k) for the spatial order `order` (2 or 4) */
static double lap_h2(const double *u, int dim, int n, int order, int i, int j, int k)
{
    double up = at(u, dim, n, i, j, k);
    if (order != 4) return nbsum(u, dim, n, i, j, k) - 2.0 * dim * up;
    double acc = 0.0;
    for (int a = 0; a < dim; ++a) {
        int c = a == 0 ? i : (a == 1 ? j : k);
        acc += (-at_odd(u, dim, n, a, i, j, k, c - 2) + 16.0 * at_odd(u, dim, n, a, i, j, k, c - 1) - 30.0 * up
                + 16.0 * at_odd(u, dim, n, a, i, j, k, c + 1) - at_odd(u, dim, n, a, i, j, k, c + 2)) / 12.0;
    }
    return acc;
}

/* -h^2 times the diagonal entry of Lap_h at (i,j,k): 2 d for order 2; for order 4,
 * 30/12 per axis, 29/12 on an axis where the point is first or last (the reflected
 * value beyond the wall is -u at the point itself) */
static double lap_diag_h2(int dim, int n, int order, int i, int j, int k)
{
    if (order != 4) return 2.0 * dim;
    double d = 0.0;
    for (int a = 0; a < dim; ++a) {
        int c = a == 0 ? i : (a == 1 ? j : k);
        d += (c == 0 || c == n - 1) ? 29.0 / 12.0 : 30.0 / 12.0;
    }
    return d;
}

/* out = nu * Lap_h u with the Laplacian of the given order (2: nu (u_{i-1} - 2u_i +
 * u_{i+1}) / dx^2 summed over axes, Sec. 4.1; 4: see lap_h2) */
void orc_apply_A_o(int dim, int n, int order, double nu, const double *u, double *out)
{
    double h = 1.0 / (n + 1), ih2 = 1.0 / (h * h);
    int nx = ext(dim, n, 0), ny = ext(dim, n, 1), nz = ext(dim, n, 2);
#pragma omp parallel for if (nz * ny > 64)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t p = ((size_t)k * ny + j) * nx + i;
                out[p] = nu * lap_h2(u, dim, n, order, i, j, k) * ih2;
            }
}

void orc_apply_A(int dim, int n, double nu, const double *u, double *out) { orc_apply_A_o(dim, n, 2, nu, u, out); }

/* out = (I - c Lap_h) e : the sub-step operator of Eq. (SDCcompactLIII) with c = dt_m * nu */
static void apply_L(int dim, int n, int order, double c, const double *e, double *out)
{
    double h = 1.0 / (n + 1), ih2 = 1.0 / (h * h);
    int nx = ext(dim, n, 0), ny = ext(dim, n, 1), nz = ext(dim, n, 2);
#pragma omp parallel for if (nz * ny > 64)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t p = ((size_t)k * ny + j) * nx + i;
                out[p] = e[p] - c * lap_h2(e, dim, n, order, i, j, k) * ih2;
            }
}

static double maxabs(const double *v, size_t N)
{
    double m = 0.0;
    for (size_t p = 0; p < N; ++p) {
        double a = fabs(v[p]);
        if (a > m || a != a) m = (a != a) ? INFINITY : a;
    }
    return m;
}

/* ------------------------------------------------------------------------- */
/* Geometric multigrid for (I - c Lap_h) u = b (Sec. 4.1.1: linear           */
/* interpolation, full weighting, Jacobi; Sec. 4.1.2: Gauss-Seidel)         */
/* ------------------------------------------------------------------------- */

typedef struct {
    int smoother;      /* 0 = weighted Jacobi, 1 = red-black Gauss-Seidel */
    double omega;      /* relaxation weight (Jacobi 2/3, GS 1)            */
    int nu1, nu2;      /* pre- and post-smoothing sweeps                  */
    int vcycles;       /* > 0: fixed number of V-cycles; 0: solve to tol  */
    double mg_tol;     /* full solve: ||b - L u||_inf <= tol*max(1,||b||) */
    double mg_stall;   /* stop when the new residual >= stall * old one   */
    int mg_maxcycles;  /* cap on V-cycles in full-solve mode              */
} orc_mg;

/* one weighted-Jacobi sweep: e <- e + omega D^{-1} (f - L e), D = diag(L) (1 + 2 d c/h^2
 * for order 2) */
static void smooth_jacobi(int dim, int n, int order, double c, double omega, const double *f, double *e,
                          double *tmp)
{
    double h = 1.0 / (n + 1), a = c / (h * h);
    int nx = ext(dim, n, 0), ny = ext(dim, n, 1), nz = ext(dim, n, 2);
    apply_L(dim, n, order, c, e, tmp);
#pragma omp parallel for if (nz * ny > 64)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t p = ((size_t)k * ny + j) * nx + i;
                e[p] += omega * (f[p] - tmp[p]) / (1.0 + a * lap_diag_h2(dim, n, order, i, j, k));
            }
}

/* one multicolour Gauss-Seidel sweep for the fourth-order operator (reading g24): colour
 * (I+J+K) mod 3 of the 1-based indices, colours 0, 1, 2 in turn; points of one colour
 * are at least 3 apart on every axis line, so none reads another of its colour, and
 * each solves its own row with the latest values of the other colours. */
static void smooth_gs3(int dim, int n, double c, double omega, const double *f, double *e)
{
    double h = 1.0 / (n + 1), a = c / (h * h);
    int nx = ext(dim, n, 0), ny = ext(dim, n, 1), nz = ext(dim, n, 2);
    for (int colour = 0; colour < 3; ++colour) {
#pragma omp parallel for if (nz * ny > 64)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int s1 = (i + 1) + (dim >= 2 ? j + 1 : 0) + (dim >= 3 ? k + 1 : 0);
                    if (s1 % 3 != colour) continue;
                    size_t p = ((size_t)k * ny + j) * nx + i;
                    double D = 1.0 + a * lap_diag_h2(dim, n, 4, i, j, k);
                    double Le = e[p] - a * lap_h2(e, dim, n, 4, i, j, k);
                    e[p] += omega * (f[p] - Le) / D;
                }
    }
}

/* one red-black Gauss-Seidel sweep: red points ((i+j+k) even in 1-based
 * interior indices) first, then black; each point solves its own row. */
static void smooth_rbgs(int dim, int n, double c, double omega, const double *f, double *e)
{
    double h = 1.0 / (n + 1), a = c / (h * h), D = 1.0 + 2.0 * dim * a;
    int nx = ext(dim, n, 0), ny = ext(dim, n, 1), nz = ext(dim, n, 2);
    for (int colour = 0; colour < 2; ++colour) {
#pragma omp parallel for if (nz * ny > 64)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int s1 = (i + 1) + (dim >= 2 ? j + 1 : 0) + (dim >= 3 ? k + 1 : 0);
                    if ((s1 & 1) != colour) continue;
                    size_t p = ((size_t)k * ny + j) * nx + i;
                    double gs = (f[p] + a * nbsum(e, dim, n, i, j, k)) / D;
                    e[p] = (1.0 - omega) * e[p] + omega * gs;
                }
    }
}

static void smooth(const orc_mg *mg, int dim, int n, int order, double c, const double *f, double *e, double *tmp)
{
    if (mg->smoother == 1 && order == 4) smooth_gs3(dim, n, c, mg->omega, f, e);
    else if (mg->smoother == 1) smooth_rbgs(dim, n, c, mg->omega, f, e);
    else smooth_jacobi(dim, n, order, c, mg->omega, f, e, tmp);
}

/* per-axis full-weighting taps: fine 1-based index 2J-1, 2J, 2J+1 with 1/4, 1/2, 1/4 */
/* full-weighting restriction of r (fine, n) to fc (coarse, (n-1)/2) */
static void restrict_fw(int dim, int n, const double *r, double *fc)
{
    int nc = (n - 1) / 2;
    int cx = ext(dim, nc, 0), cy = ext(dim, nc, 1), cz = ext(dim, nc, 2);
    static const double w[3] = {0.25, 0.5, 0.25};
#pragma omp parallel for if (cz * cy > 64)
    for (int K = 0; K < cz; ++K)
        for (int J = 0; J < cy; ++J)
            for (int I = 0; I < cx; ++I) {
                double acc = 0.0;
                for (int c = (dim >= 3 ? -1 : 0); c <= (dim >= 3 ? 1 : 0); ++c)
                    for (int b = (dim >= 2 ? -1 : 0); b <= (dim >= 2 ? 1 : 0); ++b)
                        for (int a = -1; a <= 1; ++a) {
                            double wt = w[a + 1] * (dim >= 2 ? w[b + 1] : 1.0) * (dim >= 3 ? w[c + 1] : 1.0);
                            /* coarse 0-based I <-> fine 0-based 2I+1 */
                            acc += wt * at(r, dim, n, 2 * I + 1 + a,
                                           dim >= 2 ? 2 * J + 1 + b : 0,
                                           dim >= 3 ? 2 * K + 1 + c : 0);
                        }
                fc[((size_t)K * cy + J) * cx + I] = acc;
            }
}

/* per-axis linear interpolation taps for fine 0-based index i:
 * 1-based i1 = i+1 even -> coarse 1-based i1/2 with weight 1;
 * odd -> coarse (i1-1)/2 and (i1+1)/2 with weight 1/2 each (walls are 0). */
static int lin_taps(int i, int *idx, double *w)
{
    int i1 = i + 1;
    if ((i1 & 1) == 0) { idx[0] = i1 / 2 - 1; w[0] = 1.0; return 1; }
    idx[0] = (i1 - 1) / 2 - 1; w[0] = 0.5;
    idx[1] = (i1 + 1) / 2 - 1; w[1] = 0.5;
    return 2;
}

/* e (fine, n) += P ec (coarse, (n-1)/2) with d-linear interpolation */
static void prolong_add(int dim, int n, const double *ec, double *e)
{
    int nc = (n - 1) / 2;
    int nx = ext(dim, n, 0), ny = ext(dim, n, 1), nz = ext(dim, n, 2);
#pragma omp parallel for if (nz * ny > 64)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int ix[2], iy[2] = {0, 0}, iz[2] = {0, 0};
                double wx[2], wy[2] = {1.0, 1.0}, wz[2] = {1.0, 1.0};
                int tx = lin_taps(i, ix, wx), ty = 1, tz = 1;
                if (dim >= 2) ty = lin_taps(j, iy, wy);
                if (dim >= 3) tz = lin_taps(k, iz, wz);
                double acc = 0.0;
                for (int c = 0; c < tz; ++c)
                    for (int b = 0; b < ty; ++b)
                        for (int a = 0; a < tx; ++a)
                            acc += wx[a] * wy[b] * wz[c] * at(ec, dim, nc, ix[a], iy[b], iz[c]);
                e[((size_t)k * ny + j) * nx + i] += acc;
            }
}

/* dense Gaussian elimination with partial pivoting: A (N x N, row-major) x = b */
static int dense_solve(int N, double *A, double *b, double *x)
{
    for (int col = 0; col < N; ++col) {
        int piv = col;
        for (int r = col + 1; r < N; ++r)
            if (fabs(A[r * N + col]) > fabs(A[piv * N + col])) piv = r;
        if (A[piv * N + col] == 0.0) return -1;
        if (piv != col) {
            for (int q = 0; q < N; ++q) {
                double t = A[col * N + q]; A[col * N + q] = A[piv * N + q]; A[piv * N + q] = t;
            }
            double t = b[col]; b[col] = b[piv]; b[piv] = t;
        }
        for (int r = col + 1; r < N; ++r) {
            double f = A[r * N + col] / A[col * N + col];
            for (int q = col; q < N; ++q) A[r * N + q] -= f * A[col * N + q];
            b[r] -= f * b[col];
        }
    }
    for (int r = N - 1; r >= 0; --r) {
        double s = b[r];
        for (int q = r + 1; q < N; ++q) s -= A[r * N + q] * x[q];
        x[r] = s / A[r * N + r];
    }
    return 0;
}

/* exact solve of (I - c Lap_h) e = f on a small grid: the operator is assembled
 * column by column by applying it to unit vectors, then eliminated densely. */
static void coarse_solve(int dim, int n, int order, double c, const double *f, double *e)
{
    int N = (int)npts(dim, n);
    double *A = malloc(sizeof(double) * N * N), *unit = calloc(N, sizeof(double));
    double *col = malloc(sizeof(double) * N), *rhs = malloc(sizeof(double) * N);
    for (int q = 0; q < N; ++q) {
        unit[q] = 1.0;
        apply_L(dim, n, order, c, unit, col);
        unit[q] = 0.0;
        for (int r = 0; r < N; ++r) A[r * N + q] = col[r];
    }
    memcpy(rhs, f, sizeof(double) * N);
    dense_solve(N, A, rhs, e);
    free(A); free(unit); free(col); free(rhs);
}

/* One V(nu1,nu2)-cycle for (I - c Lap_h) e = f on a grid with n = 2^p - 1
 * points per axis, with the operator rediscretised on every level ("standard
 * geometric multigrid", Sec. 4.1.1); the 3-point level is solved exactly.  `order`
 * is the Laplacian's order on this grid; every coarser grid is rediscretised with the
 * second-order stencil (reading g24). */
static void vcycle(const orc_mg *mg, int dim, int n, int order, double c, const double *f, double *e)
{
    if (n <= 3) { coarse_solve(dim, n, order, c, f, e); return; }
    size_t N = npts(dim, n);
    int nc = (n - 1) / 2;
    size_t Nc = npts(dim, nc);
    double *tmp = malloc(sizeof(double) * N);
    double *fc = malloc(sizeof(double) * Nc), *ec = calloc(Nc, sizeof(double));
    for (int s = 0; s < mg->nu1; ++s) smooth(mg, dim, n, order, c, f, e, tmp);
    apply_L(dim, n, order, c, e, tmp);
    for (size_t p = 0; p < N; ++p) tmp[p] = f[p] - tmp[p];       /* residual */
    restrict_fw(dim, n, tmp, fc);
    vcycle(mg, dim, nc, 2, c, fc, ec);
    prolong_add(dim, n, ec, e);
    for (int s = 0; s < mg->nu2; ++s) smooth(mg, dim, n, order, c, f, e, tmp);
    free(tmp); free(fc); free(ec);
}

/* ||b - (I - c Lap_h) u||_inf */
static double mg_resnorm(int dim, int n, int order, double c, const double *b, const double *u)
{
    size_t N = npts(dim, n);
    double *t = malloc(sizeof(double) * N);
    apply_L(dim, n, order, c, u, t);
    for (size_t p = 0; p < N; ++p) t[p] = b[p] - t[p];
    double r = maxabs(t, N);
    free(t);
    return r;
}

/* Solve (I - c Lap_h) u = b from the initial guess in u.
 * Fixed mode (vcycles > 0): exactly that many V-cycles (inexact solves, Sec. 2.3.1).
 * Full mode (vcycles == 0): V-cycles until ||b - L u|| <= tol * max(1, ||b||),
 * or until a cycle fails to bring the residual below stall * previous
 * (the 1e-12 / 75 % rule of Sec. 4.2.1), at most mg_maxcycles cycles.
 * Returns the number of V-cycles done. */
int orc_mg_solve_o(const orc_mg *mg, int dim, int n, int order, double c, const double *b, double *u)
{
    if (mg->vcycles > 0) {
        for (int v = 0; v < mg->vcycles; ++v) vcycle(mg, dim, n, order, c, b, u);
        return mg->vcycles;
    }
    double bn = maxabs(b, npts(dim, n));
    if (bn < 1.0) bn = 1.0;
    double r = mg_resnorm(dim, n, order, c, b, u);
    int cycles = 0;
    while (r > mg->mg_tol * bn && cycles < mg->mg_maxcycles) {
        vcycle(mg, dim, n, order, c, b, u);
        ++cycles;
        double rn = mg_resnorm(dim, n, order, c, b, u);
        if (rn >= mg->mg_stall * r) break;
        r = rn;
    }
    return cycles;
}

int orc_mg_solve(const orc_mg *mg, int dim, int n, double c, const double *b, double *u)
{
    return orc_mg_solve_o(mg, dim, n, 2, c, b, u);
}

/* One smoothing sweep, exported for the smoother pins. */
void orc_smooth_o(const orc_mg *mg, int dim, int n, int order, double c, const double *f, double *e)
{
    double *tmp = malloc(sizeof(double) * npts(dim, n));
    smooth(mg, dim, n, order, c, f, e, tmp);
    free(tmp);
}

void orc_smooth(const orc_mg *mg, int dim, int n, double c, const double *f, double *e)
{
    orc_smooth_o(mg, dim, n, 2, c, f, e);
}

void orc_restrict_fw(int dim, int n, const double *r, double *fc) { restrict_fw(dim, n, r, fc); }
void orc_prolong_add(int dim, int n, const double *ec, double *e) { prolong_add(dim, n, ec, e); }
void orc_apply_L(int dim, int n, double c, const double *e, double *out) { apply_L(dim, n, 2, c, e, out); }
void orc_apply_L_o(int dim, int n, int order, double c, const double *e, double *out)
{
    apply_L(dim, n, order, c, e, out);
}

/* ------------------------------------------------------------------------- */
/* SDC on one time slice (Sec. 2.2)                                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    int dim, n;        /* spatial grid of this level             */
    int s;             /* number of nodes (M + 1)                */
    double nu, dt;     /* diffusion coefficient, slice length    */
    int family;        /* 0 Gauss-Lobatto, 1 uniform (see orc_nodes) */
    int order;         /* Laplacian order: 2 (0 also means 2) or 4 */
} orc_level;

static int level_order(const orc_level *L) { return L->order == 4 ? 4 : 2; }

static void level_nodes(const orc_level *L, double *tau, double *Q)
{
    orc_nodes(L->s, L->family, tau);
    orc_qmatrix_family(L->s, L->family, tau, Q);
}

/* One SDC sweep with implicit-Euler sub-steps, Eq. (sdc-be) in the form (SDCcompactLIII):
 *   (I - dt_m nu Lap_h) u_{m+1} = u_m - dt_m F^k_{m+1} + dt sum_i (q_{m+1,i}-q_{m,i}) F^k_i
 *                                 + (tau_{m+1} - tau_m)
 * where u_m is the already-updated value, F^k = A U^k from before the sweep and
 * tau is the FAS correction (NULL on the finest level).  Each sub-step is solved
 * by multigrid from the initial guess u^k_{m+1} (Sec. 2.2.2, 2.3.1); afterwards
 * F_{m+1} = A u_{m+1} is re-evaluated.  U and F are s x N.  Returns V-cycles used. */
int orc_sweep(const orc_level *L, const orc_mg *mg, double *U, double *F, const double *fas)
{
    double tau[ORC_MAXS], Q[ORC_MAXS * ORC_MAXS];
    level_nodes(L, tau, Q);
    int s = L->s, M = s - 1;
    size_t N = npts(L->dim, L->n);
    double *Fk = malloc(sizeof(double) * N * s);
    double *b = malloc(sizeof(double) * N);
    memcpy(Fk, F, sizeof(double) * N * s);
    int cycles = 0;
    for (int m = 0; m < M; ++m) {
        double dtm = L->dt * (tau[m + 1] - tau[m]);
        for (size_t p = 0; p < N; ++p) {
            double I = 0.0;
            for (int i = 0; i < s; ++i) I += L->dt * (Q[(m + 1) * s + i] - Q[m * s + i]) * Fk[i * N + p];
            b[p] = U[m * N + p] - dtm * Fk[(m + 1) * N + p] + I;
            if (fas) b[p] += fas[(m + 1) * N + p] - fas[m * N + p];
        }
        cycles += orc_mg_solve_o(mg, L->dim, L->n, level_order(L), dtm * L->nu, b, U + (m + 1) * N);
        orc_apply_A_o(L->dim, L->n, level_order(L), L->nu, U + (m + 1) * N, F + (m + 1) * N);
    }
    free(Fk); free(b);
    return cycles;
}

/* Collocation residual, Eq. (resid): r_m = u_0 + dt sum_i q_{m,i} F_i (+ tau_m) - u_m,
 * returned as the max norm over all nodes and points. */
double orc_residual(const orc_level *L, const double *U, const double *F, const double *fas)
{
    double tau[ORC_MAXS], Q[ORC_MAXS * ORC_MAXS];
    level_nodes(L, tau, Q);
    int s = L->s;
    size_t N = npts(L->dim, L->n);
    double r = 0.0;
    for (int m = 0; m < s; ++m)
        for (size_t p = 0; p < N; ++p) {
            double v = U[p];
            for (int i = 0; i < s; ++i) v += L->dt * Q[m * s + i] * F[i * N + p];
            if (fas) v += fas[m * N + p];
            v -= U[m * N + p];
            double a = fabs(v);
            if (a > r || a != a) r = (a != a) ? INFINITY : a;
        }
    return r;
}

/* ------------------------------------------------------------------------- */
/* Transfers between PFASST levels (Sec. 4.2.1)                              */
/* ------------------------------------------------------------------------- */

/* point-wise restriction in space: coarse 1-based J <- fine 1-based 2J */
void orc_inject(int dim, int n, const double *uf, double *uc)
{
    int nc = (n - 1) / 2;
    int cx = ext(dim, nc, 0), cy = ext(dim, nc, 1), cz = ext(dim, nc, 2);
    for (int K = 0; K < cz; ++K)
        for (int J = 0; J < cy; ++J)
            for (int I = 0; I < cx; ++I)
                uc[((size_t)K * cy + J) * cx + I] =
                    at(uf, dim, n, 2 * I + 1, dim >= 2 ? 2 * J + 1 : 0, dim >= 3 ? 2 * K + 1 : 0);
}

/* coarse value at 1-based index J along one axis with odd reflection at the
 * walls (u(-x) = -u(x)): index 0 and nc+1 are the walls (0), -1 and nc+2 mirror. */
static int reflect(int J1, int nc, double *sign)
{
    *sign = 1.0;
    if (J1 == 0 || J1 == nc + 1) { *sign = 0.0; return 0; }
    if (J1 < 0) { *sign = -1.0; return -J1; }
    if (J1 > nc + 1) { *sign = -1.0; return 2 * (nc + 1) - J1; }
    return J1;
}

/* per-axis interpolation taps of fine 0-based index i onto coarse 1-based indices */
static int interp_taps(int order, int i, int nc, int *idx, double *w)
{
    int i1 = i + 1, t = 0;
    if ((i1 & 1) == 0) { idx[0] = i1 / 2; w[0] = 1.0; return 1; }
    int J = (i1 - 1) / 2;             /* fine point lies between coarse J and J+1 */
    if (order == 2) {
        int   off[2] = {0, 1};
        double ww[2] = {0.5, 0.5};
        for (int q = 0; q < 2; ++q) { idx[t] = J + off[q]; w[t] = ww[q]; ++t; }
    } else {
        int   off[4] = {-1, 0, 1, 2};
        double ww[4] = {-1.0 / 16, 9.0 / 16, 9.0 / 16, -1.0 / 16};
        for (int q = 0; q < 4; ++q) { idx[t] = J + off[q]; w[t] = ww[q]; ++t; }
    }
    (void)nc;
    return t;
}

/* uf (fine, n) += I_x uc (coarse, (n-1)/2), I_x = 4th-order (or linear) interpolation */
void orc_interp_add(int dim, int n, int order, double alpha, const double *uc, double *uf)
{
    int nc = (n - 1) / 2;
    int nx = ext(dim, n, 0), ny = ext(dim, n, 1), nz = ext(dim, n, 2);
    int cx = ext(dim, nc, 0), cy = ext(dim, nc, 1);
#pragma omp parallel for if (nz * ny > 64)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int ix[4], iy[4] = {1}, iz[4] = {1};
                double wx[4], wy[4] = {1.0}, wz[4] = {1.0};
                int tx = interp_taps(order, i, nc, ix, wx), ty = 1, tz = 1;
                if (dim >= 2) ty = interp_taps(order, j, nc, iy, wy);
                if (dim >= 3) tz = interp_taps(order, k, nc, iz, wz);
                double acc = 0.0;
                for (int c = 0; c < tz; ++c)
                    for (int b = 0; b < ty; ++b)
                        for (int a = 0; a < tx; ++a) {
                            double sx, sy = 1.0, sz = 1.0;
                            int X = reflect(ix[a], nc, &sx), Y = 1, Z = 1;
                            if (dim >= 2) Y = reflect(iy[b], nc, &sy);
                            if (dim >= 3) Z = reflect(iz[c], nc, &sz);
                            double sg = sx * sy * sz;
                            if (sg == 0.0) continue;
                            size_t q = ((size_t)(dim >= 3 ? Z - 1 : 0) * cy + (dim >= 2 ? Y - 1 : 0)) * cx + (X - 1);
                            acc += wx[a] * wy[b] * wz[c] * sg * uc[q];
                        }
                uf[((size_t)k * ny + j) * nx + i] += alpha * acc;
            }
}

/* ------------------------------------------------------------------------- */
/* Two-level PFASST (Sec. 2.4) with all P time slices emulated serially      */
/* ------------------------------------------------------------------------- */

typedef struct {
    int dim, n_f, s_f, s_c, slices, nlevels, interp_order;
    double nu, dt;
    orc_mg mg;
    int fam_f, fam_c;  /* node families of the fine and coarse level */
    int order_f;       /* Laplacian order of the fine level (2 or 4; 0 means 2); the coarse level is 2nd order */
    orc_mg mg_c;       /* multigrid settings of the coarse level's sub-step solves (reading g16:
                          the same as mg unless chosen otherwise) */
} orc_pfasst;

static int fine_order(const orc_pfasst *P) { return P->order_f == 4 ? 4 : 2; }

/* coarse node j coincides with fine node map[j] (coarse nodes are a subset) */
static int node_map(const orc_pfasst *P, int *map)
{
    int sf = P->s_f, sc = P->s_c;
    double tf[ORC_MAXS], tc[ORC_MAXS];
    orc_nodes(sf, P->fam_f, tf);
    orc_nodes(sc, P->fam_c, tc);
    for (int j = 0; j < sc; ++j) {
        map[j] = -1;
        for (int m = 0; m < sf; ++m)
            if (fabs(tf[m] - tc[j]) < 1e-14) map[j] = m;
        if (map[j] < 0) return -1;
    }
    return 0;
}

/* FAS restriction of one slice (Sec. 2.3; reading: the coarse problem is
 * U_c = U_c,0 + dt Q_c A_c U_c + tau with
 *   tau_j = R(dt sum_i Qf[map j][i] F_f,i) - dt sum_i Qc[j][i] A_c (R U_f)_i ),
 * R = point-wise injection in space and time. Writes Uc, Fc, fas and Uc0 = Uc. */
static void fas_restrict(const orc_pfasst *P, const double *Uf, const double *Ff,
                         double *Uc, double *Fc, double *fas, double *Uc0)
{
    int dim = P->dim, nf = P->n_f, nc = (nf - 1) / 2, sf = P->s_f, sc = P->s_c;
    size_t Nf = npts(dim, nf), Nc = npts(dim, nc);
    double tf[ORC_MAXS], tc[ORC_MAXS], Qf[ORC_MAXS * ORC_MAXS], Qc[ORC_MAXS * ORC_MAXS];
    int map[ORC_MAXS];
    orc_nodes(sf, P->fam_f, tf); orc_qmatrix_family(sf, P->fam_f, tf, Qf);
    orc_nodes(sc, P->fam_c, tc); orc_qmatrix_family(sc, P->fam_c, tc, Qc);
    node_map(P, map);
    double *tmpf = malloc(sizeof(double) * Nf), *tmpc = malloc(sizeof(double) * Nc);
    for (int j = 0; j < sc; ++j) {
        orc_inject(dim, nf, Uf + (size_t)map[j] * Nf, Uc + j * Nc);
        orc_apply_A(dim, nc, P->nu, Uc + j * Nc, Fc + j * Nc);
    }
    for (int j = 0; j < sc; ++j) {
        for (size_t p = 0; p < Nf; ++p) {
            double I = 0.0;
            for (int i = 0; i < sf; ++i) I += P->dt * Qf[map[j] * sf + i] * Ff[i * Nf + p];
            tmpf[p] = I;
        }
        orc_inject(dim, nf, tmpf, tmpc);
        for (size_t p = 0; p < Nc; ++p) {
            double I = 0.0;
            for (int i = 0; i < sc; ++i) I += P->dt * Qc[j * sc + i] * Fc[i * Nc + p];
            fas[j * Nc + p] = tmpc[p] - I;
        }
    }
    memcpy(Uc0, Uc, sizeof(double) * Nc * sc);
    free(tmpf); free(tmpc);
}

/* Interpolate the coarse correction of one slice to every fine node, including
 * node 0 (Sec. 4.2.1): U_f,m += sum_j T[m][j] I_x (U_c,j - U_c0,j), with T the
 * Lagrange weights of the coarse nodes at the fine nodes; then F_f = A_f U_f. */
static void interp_correction(const orc_pfasst *P, double *Uf, double *Ff, const double *Uc, const double *Uc0)
{
    int dim = P->dim, nf = P->n_f, nc = (nf - 1) / 2, sf = P->s_f, sc = P->s_c;
    size_t Nf = npts(dim, nf), Nc = npts(dim, nc);
    double tf[ORC_MAXS], tc[ORC_MAXS], w[ORC_MAXS];
    orc_nodes(sf, P->fam_f, tf);
    orc_nodes(sc, P->fam_c, tc);
    double *d = malloc(sizeof(double) * Nc);
    for (int j = 0; j < sc; ++j) {
        for (size_t p = 0; p < Nc; ++p) d[p] = Uc[j * Nc + p] - Uc0[j * Nc + p];
        for (int m = 0; m < sf; ++m) {
            lagrange_weights(sc, tc, tf[m], w);
            if (w[j] != 0.0) orc_interp_add(dim, nf, P->interp_order, w[j], d, Uf + (size_t)m * Nf);
        }
    }
    for (int m = 0; m < sf; ++m) orc_apply_A_o(dim, nf, fine_order(P), P->nu, Uf + (size_t)m * Nf, Ff + (size_t)m * Nf);
    free(d);
}

/* The interpolation step alone, for one slice (exported so that the tests can pin it). */
void orc_pfasst_interp_slice(const orc_pfasst *P, double *Uf, double *Ff, const double *Uc, const double *Uc0)
{
    interp_correction(P, Uf, Ff, Uc, Uc0);
}

static orc_level fine_level(const orc_pfasst *P)
{
    orc_level L = {P->dim, P->n_f, P->s_f, P->nu, P->dt, P->fam_f, fine_order(P)};
    return L;
}
static orc_level coarse_level(const orc_pfasst *P)
{
    orc_level L = {P->dim, (P->n_f - 1) / 2, P->s_c, P->nu, P->dt, P->fam_c, 2};
    return L;
}

/* Spread the initial value u0 to every node of every slice and set F = A U
 * (the start of the predictor, Sec. 2.4). */
void orc_pfasst_spread(const orc_pfasst *P, const double *u0, double *Uf, double *Ff)
{
    size_t Nf = npts(P->dim, P->n_f);
    for (int p = 0; p < P->slices; ++p)
        for (int m = 0; m < P->s_f; ++m) {
            double *u = Uf + ((size_t)p * P->s_f + m) * Nf;
            memcpy(u, u0, sizeof(double) * Nf);
            orc_apply_A_o(P->dim, P->n_f, fine_order(P), P->nu, u, Ff + ((size_t)p * P->s_f + m) * Nf);
        }
}

/* Predictor (Sec. 2.4): restrict the spread values (with FAS), then in stage
 * s = 0..P-1 every slice p >= s takes the new coarse end value of slice p-1 as
 * its initial value (s > 0) and does one coarse sweep, so slice p does p+1
 * coarse sweeps; finally the coarse correction is interpolated to the fine level.
 * With one level the predictor is the spread alone. */
void orc_pfasst_predict(const orc_pfasst *P, double *Uf, double *Ff,
                        double *Uc, double *Fc, double *fas, double *Uc0)
{
    if (P->nlevels < 2) return;
    int sf = P->s_f, sc = P->s_c, Pn = P->slices;
    size_t Nf = npts(P->dim, P->n_f), Nc = npts(P->dim, (P->n_f - 1) / 2);
    orc_level C = coarse_level(P);
    for (int p = 0; p < Pn; ++p)
        fas_restrict(P, Uf + (size_t)p * sf * Nf, Ff + (size_t)p * sf * Nf,
                     Uc + (size_t)p * sc * Nc, Fc + (size_t)p * sc * Nc,
                     fas + (size_t)p * sc * Nc, Uc0 + (size_t)p * sc * Nc);
    for (int s = 0; s < Pn; ++s) {
        if (s > 0)
            for (int p = Pn - 1; p >= s; --p) {
                double *u0c = Uc + (size_t)p * sc * Nc;
                memcpy(u0c, Uc + ((size_t)(p - 1) * sc + sc - 1) * Nc, sizeof(double) * Nc);
                orc_apply_A(P->dim, C.n, P->nu, u0c, Fc + (size_t)p * sc * Nc);
            }
        for (int p = s; p < Pn; ++p)
            orc_sweep(&C, &P->mg_c, Uc + (size_t)p * sc * Nc, Fc + (size_t)p * sc * Nc, fas + (size_t)p * sc * Nc);
    }
    for (int p = 0; p < Pn; ++p)
        interp_correction(P, Uf + (size_t)p * sf * Nf, Ff + (size_t)p * sf * Nf,
                          Uc + (size_t)p * sc * Nc, Uc0 + (size_t)p * sc * Nc);
}

/* One PFASST iteration over all slices (Sec. 2.4; the schedule is the reading
 * of the pipelined algorithm with one fine and one coarse level):
 *   1. fine sweep on every slice (these run concurrently in PFASST);
 *   2. FAS restriction of every slice;
 *   3. coarse sweeps as a serial chain: slice p first receives the new coarse
 *      end value of slice p-1 (blocking communication on the coarse level);
 *   4. interpolation of the coarse correction to the fine level, F_f = A U_f;
 *   5. send forward: slice p >= 1 takes the fine end value of slice p-1;
 *   6. collocation residual of every slice (Eq. resid), written to res[p].
 * With one level, steps 2-4 are skipped (parallel SDC with send-forward). */
void orc_pfasst_iteration(const orc_pfasst *P, double *Uf, double *Ff,
                          double *Uc, double *Fc, double *fas, double *Uc0, double *res)
{
    int sf = P->s_f, sc = P->s_c, Pn = P->slices;
    size_t Nf = npts(P->dim, P->n_f), Nc = npts(P->dim, (P->n_f - 1) / 2);
    orc_level F = fine_level(P), C = coarse_level(P);
    for (int p = 0; p < Pn; ++p)
        orc_sweep(&F, &P->mg, Uf + (size_t)p * sf * Nf, Ff + (size_t)p * sf * Nf, NULL);
    if (P->nlevels >= 2) {
        for (int p = 0; p < Pn; ++p)
            fas_restrict(P, Uf + (size_t)p * sf * Nf, Ff + (size_t)p * sf * Nf,
                         Uc + (size_t)p * sc * Nc, Fc + (size_t)p * sc * Nc,
                         fas + (size_t)p * sc * Nc, Uc0 + (size_t)p * sc * Nc);
        for (int p = 0; p < Pn; ++p) {
            if (p > 0) {
                double *u0c = Uc + (size_t)p * sc * Nc;
                memcpy(u0c, Uc + ((size_t)(p - 1) * sc + sc - 1) * Nc, sizeof(double) * Nc);
                orc_apply_A(P->dim, C.n, P->nu, u0c, Fc + (size_t)p * sc * Nc);
            }
            orc_sweep(&C, &P->mg_c, Uc + (size_t)p * sc * Nc, Fc + (size_t)p * sc * Nc, fas + (size_t)p * sc * Nc);
        }
        for (int p = 0; p < Pn; ++p)
            interp_correction(P, Uf + (size_t)p * sf * Nf, Ff + (size_t)p * sf * Nf,
                              Uc + (size_t)p * sc * Nc, Uc0 + (size_t)p * sc * Nc);
    }
    for (int p = Pn - 1; p >= 1; --p) {
        double *u0f = Uf + (size_t)p * sf * Nf;
        memcpy(u0f, Uf + ((size_t)(p - 1) * sf + sf - 1) * Nf, sizeof(double) * Nf);
        orc_apply_A_o(P->dim, P->n_f, fine_order(P), P->nu, u0f, Ff + (size_t)p * sf * Nf);
    }
    for (int p = 0; p < Pn; ++p)
        res[p] = orc_residual(&F, Uf + (size_t)p * sf * Nf, Ff + (size_t)p * sf * Nf, NULL);
}

/* ------------------------------------------------------------------------- */
/* PFASST with up to three levels (Sec. 2.3 - 2.4, reading of the multi-level */
/* schedule): levels l = 0 (finest) .. L-1 (coarsest), grid n_l = (n_{l-1}-1)/2 */
/* ------------------------------------------------------------------------- */

typedef struct {
    int dim, n0, slices, nlevels, interp_order;
    int s[3], fam[3];          /* nodes and node family of every level        */
    double nu, dt;
    orc_mg mg;
    int order0;                /* Laplacian order of level 0 (2 or 4; 0 means 2); coarser levels: 2 */
    orc_mg mg_c;               /* multigrid settings of the sub-step solves on levels >= 1 */
} orc_ml;

static int ml_order(const orc_ml *P, int l) { return l == 0 && P->order0 == 4 ? 4 : 2; }

/* per level: U, F (slices x s_l x N_l), tau (FAS correction, unused on level 0) and
 * Ur (the restricted values the coarse correction is measured against) */
typedef struct {
    double *U[3], *F[3], *tau[3], *Ur[3];
} orc_mlstate;

static int ml_n(const orc_ml *P, int l)
{
    int n = P->n0;
    for (int i = 0; i < l; ++i) n = (n - 1) / 2;
    return n;
}

static orc_level ml_level(const orc_ml *P, int l)
{
    orc_level L = {P->dim, ml_n(P, l), P->s[l], P->nu, P->dt, P->fam[l], ml_order(P, l)};
    return L;
}

static size_t ml_slab(const orc_ml *P, int l) { return (size_t)P->s[l] * npts(P->dim, ml_n(P, l)); }

/* FAS restriction of slice p from level l to l+1 (reading g6 applied level by level):
 *   U_{l+1,j} = R U_{l,map j},  F_{l+1} = A U_{l+1},
 *   tau_{l+1,j} = R( dt sum_i Q_l[map j][i] F_{l,i} + tau_{l,map j} ) - dt sum_i Q_{l+1}[j][i] F_{l+1,i},
 * so that R U_l solves level l+1 whenever U_l solves level l. */
static void ml_fas(const orc_ml *P, const orc_mlstate *S, int l, int p)
{
    int dim = P->dim, nf = ml_n(P, l), nc = ml_n(P, l + 1), sf = P->s[l], sc = P->s[l + 1];
    size_t Nf = npts(dim, nf), Nc = npts(dim, nc);
    double tf[ORC_MAXS], tc[ORC_MAXS], Qf[ORC_MAXS * ORC_MAXS], Qc[ORC_MAXS * ORC_MAXS];
    int map[ORC_MAXS];
    orc_nodes(sf, P->fam[l], tf); orc_qmatrix_family(sf, P->fam[l], tf, Qf);
    orc_nodes(sc, P->fam[l + 1], tc); orc_qmatrix_family(sc, P->fam[l + 1], tc, Qc);
    for (int j = 0; j < sc; ++j) {
        map[j] = -1;
        for (int m = 0; m < sf; ++m)
            if (fabs(tf[m] - tc[j]) < 1e-14) map[j] = m;
    }
    const double *Uf = S->U[l] + p * ml_slab(P, l), *Ff = S->F[l] + p * ml_slab(P, l);
    const double *tauf = l > 0 ? S->tau[l] + p * ml_slab(P, l) : NULL;
    double *Uc = S->U[l + 1] + p * ml_slab(P, l + 1), *Fc = S->F[l + 1] + p * ml_slab(P, l + 1);
    double *tauc = S->tau[l + 1] + p * ml_slab(P, l + 1), *Ur = S->Ur[l + 1] + p * ml_slab(P, l + 1);
    double *tmpf = malloc(sizeof(double) * Nf), *tmpc = malloc(sizeof(double) * Nc);
    for (int j = 0; j < sc; ++j) {
        orc_inject(dim, nf, Uf + (size_t)map[j] * Nf, Uc + j * Nc);
        orc_apply_A(dim, nc, P->nu, Uc + j * Nc, Fc + j * Nc);
    }
    for (int j = 0; j < sc; ++j) {
        for (size_t q = 0; q < Nf; ++q) {
            double I = tauf ? tauf[(size_t)map[j] * Nf + q] : 0.0;
            for (int i = 0; i < sf; ++i) I += P->dt * Qf[map[j] * sf + i] * Ff[i * Nf + q];
            tmpf[q] = I;
        }
        orc_inject(dim, nf, tmpf, tmpc);
        for (size_t q = 0; q < Nc; ++q) {
            double I = 0.0;
            for (int i = 0; i < sc; ++i) I += P->dt * Qc[j * sc + i] * Fc[i * Nc + q];
            tauc[j * Nc + q] = tmpc[q] - I;
        }
    }
    memcpy(Ur, Uc, sizeof(double) * Nc * sc);
    free(tmpf); free(tmpc);
}

/* coarse correction of slice p from level l+1 to every node of level l (Lagrange in
 * time through the level-(l+1) nodes, I_x in space), then F_l = A U_l */
static void ml_interp(const orc_ml *P, const orc_mlstate *S, int l, int p)
{
    int dim = P->dim, nf = ml_n(P, l), sf = P->s[l], sc = P->s[l + 1];
    size_t Nf = npts(dim, nf), Nc = npts(dim, ml_n(P, l + 1));
    double tf[ORC_MAXS], tc[ORC_MAXS], w[ORC_MAXS];
    orc_nodes(sf, P->fam[l], tf);
    orc_nodes(sc, P->fam[l + 1], tc);
    double *Uf = S->U[l] + p * ml_slab(P, l), *Ff = S->F[l] + p * ml_slab(P, l);
    const double *Uc = S->U[l + 1] + p * ml_slab(P, l + 1), *Ur = S->Ur[l + 1] + p * ml_slab(P, l + 1);
    double *d = malloc(sizeof(double) * Nc);
    for (int j = 0; j < sc; ++j) {
        for (size_t q = 0; q < Nc; ++q) d[q] = Uc[j * Nc + q] - Ur[j * Nc + q];
        for (int m = 0; m < sf; ++m) {
            lagrange_weights(sc, tc, tf[m], w);
            if (w[j] != 0.0) orc_interp_add(dim, nf, P->interp_order, w[j], d, Uf + (size_t)m * Nf);
        }
    }
    for (int m = 0; m < sf; ++m) orc_apply_A_o(dim, nf, ml_order(P, l), P->nu, Uf + (size_t)m * Nf, Ff + (size_t)m * Nf);
    free(d);
}

/* The interpolation step alone, level l+1 -> l of slice p (exported for the tests). */
void orc_ml_interp_slice(const orc_ml *P, const orc_mlstate *S, int l, int p)
{
    ml_interp(P, S, l, p);
}

static void ml_sweep(const orc_ml *P, const orc_mlstate *S, int l, int p)
{
    orc_level L = ml_level(P, l);
    orc_sweep(&L, l > 0 ? &P->mg_c : &P->mg, S->U[l] + p * ml_slab(P, l), S->F[l] + p * ml_slab(P, l),
              l > 0 ? S->tau[l] + p * ml_slab(P, l) : NULL);
}

/* slice p >= 1 takes the end value of slice p-1 as its initial value on level l */
static void ml_receive(const orc_ml *P, const orc_mlstate *S, int l, int p)
{
    size_t N = npts(P->dim, ml_n(P, l)), sl = ml_slab(P, l);
    double *u0 = S->U[l] + p * sl;
    memcpy(u0, S->U[l] + (p - 1) * sl + (size_t)(P->s[l] - 1) * N, sizeof(double) * N);
    orc_apply_A_o(P->dim, ml_n(P, l), ml_order(P, l), P->nu, u0, S->F[l] + p * sl);
}

void orc_ml_spread(const orc_ml *P, const double *u0, const orc_mlstate *S)
{
    size_t N = npts(P->dim, P->n0);
    for (int p = 0; p < P->slices; ++p)
        for (int m = 0; m < P->s[0]; ++m) {
            double *u = S->U[0] + p * ml_slab(P, 0) + (size_t)m * N;
            memcpy(u, u0, sizeof(double) * N);
            orc_apply_A_o(P->dim, P->n0, ml_order(P, 0), P->nu, u, S->F[0] + p * ml_slab(P, 0) + (size_t)m * N);
        }
}

/* Predictor: FAS restriction of the spread values down to the coarsest level; there,
 * stage s = 0..P-1: slices p >= s receive the coarsest end value of p-1 (s > 0) and
 * sweep; then the corrections are interpolated up level by level. */
void orc_ml_predict(const orc_ml *P, const orc_mlstate *S)
{
    int L = P->nlevels, Pn = P->slices, lc = L - 1;
    if (L < 2) return;
    for (int l = 0; l < lc; ++l)
        for (int p = 0; p < Pn; ++p) ml_fas(P, S, l, p);
    for (int s = 0; s < Pn; ++s) {
        if (s > 0)
            for (int p = Pn - 1; p >= s; --p) ml_receive(P, S, lc, p);
        for (int p = s; p < Pn; ++p) ml_sweep(P, S, lc, p);
    }
    for (int l = lc - 1; l >= 0; --l)
        for (int p = 0; p < Pn; ++p) ml_interp(P, S, l, p);
}

/* One sweep on level l of every slice, as a standalone step: on the coarsest level of
 * two or more the serial chain (slice p first receives the end value of slice p-1),
 * elsewhere every slice on its own. */
void orc_ml_sweep_level(const orc_ml *P, const orc_mlstate *S, int l)
{
    int chain = P->nlevels >= 2 && l == P->nlevels - 1;
    for (int p = 0; p < P->slices; ++p) {
        if (chain && p > 0) ml_receive(P, S, l, p);
        ml_sweep(P, S, l, p);
    }
}

/* One PFASST iteration with L levels (reading g7b):
 *   1. sweep on level 0, every slice;
 *   2. for each intermediate level l = 1..L-2: FAS restriction l-1 -> l, sweep on l;
 *   3. FAS restriction to the coarsest level, whose sweeps run as the serial chain
 *      (slice p first receives the coarsest end value of slice p-1);
 *   4. interpolation of the corrections level by level up to level 0;
 *   5. send-forward on level 0, collocation residual of every slice into res.
 * Coarser levels are restricted afresh every iteration, so only level 0 sends forward. */
void orc_ml_iteration(const orc_ml *P, const orc_mlstate *S, double *res)
{
    int L = P->nlevels, Pn = P->slices, lc = L - 1;
    for (int p = 0; p < Pn; ++p) ml_sweep(P, S, 0, p);
    if (L >= 2) {
        for (int l = 1; l < lc; ++l)
            for (int p = 0; p < Pn; ++p) {
                ml_fas(P, S, l - 1, p);
                ml_sweep(P, S, l, p);
            }
        for (int p = 0; p < Pn; ++p) ml_fas(P, S, lc - 1, p);
        for (int p = 0; p < Pn; ++p) {
            if (p > 0) ml_receive(P, S, lc, p);
            ml_sweep(P, S, lc, p);
        }
        for (int l = lc - 1; l >= 0; --l)
            for (int p = 0; p < Pn; ++p) ml_interp(P, S, l, p);
    }
    for (int p = Pn - 1; p >= 1; --p) ml_receive(P, S, 0, p);
    orc_level F = ml_level(P, 0);
    for (int p = 0; p < Pn; ++p)
        res[p] = orc_residual(&F, S->U[0] + p * ml_slab(P, 0), S->F[0] + p * ml_slab(P, 0), NULL);
}
