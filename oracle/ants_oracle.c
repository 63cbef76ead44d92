/*
 * ants_oracle.c -- plain, slow FP64 CPU oracle for the maximum-likelihood
 * position/energy reconstruction of ANTS2 (Morozov et al., arXiv:1602.07247).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the test suite, the smoke check and the CPU baseline
 * leg of the benchmark do.  It shares no code, header, table or constant
 * with the CUDA path.
 *
 * What it follows (paper sections):
 *   - Sec. 5.1.1, centroid (COG) equation: x = sum X_i S_i/g_i / sum S_i/g_i.
 *   - Sec. 5.1.2, statistical reconstruction: best match between measured
 *     signals and LRF-model signals by Maximum Likelihood.
 *   - Sec. 5.1.2.2, contracting grids: regular grid centred on the start
 *     position, best node becomes the centre of a finer grid with the same
 *     node count, fixed number of iterations; the energy at each node is the
 *     ratio (sum of signals) / (sum of LRF values).
 *   - Sec. 6 / 6.1.1 / 6.1.2, LRFs are B-spline parameterised functions of
 *     1 (axial), 2 (XY) or 3 (XYZ) coordinates, computed from datasets of
 *     (position, signal) pairs; Sec. 6.2, one group = one shared LRF times a
 *     per-sensor relative gain; Sec. 6.3, the gains of a group refitted with
 *     its profile fixed.
 *   - Sec. 5.2, event filters on chi-squared, energy, signal sum and
 *     position; Sec. 8, iterative LRF reconstruction (reconstruct, filter,
 *     optionally shift the positions at random, refit, repeat).
 *   - Sec. 5.1.2 / 5.1.2.1 / 5.3, search variants (least squares, the
 *     strongest-sensor start, sensor cuts, passive sensors) and the
 *     continuous minimisation of the match (Migrad in the paper; here damped
 *     Fisher scoring with the energy profiled out).
 *   - Sec. 6.1.1 / 6.1.2, composite, axial+z and sliced LRFs; Sec. 6.2,
 *     sensor groups by distance and XY classes by symmetry.
 *   - Sec. 4.2.3 - 4.2.6 and 3.5, optical photon transport in a slab stack.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - B-spline: uniform cubic on [lo,hi] with n intervals, n+3 basis
 *     functions on the extended knots t_j = lo + (j-3)h; evaluated with the
 *     Cox-de Boor recursion; x == hi uses the last interval.
 *   - LRF fit: least squares by the normal equations (B^T B + lambda I) c =
 *     B^T v solved with a Cholesky factorisation; lambda = 0 unless the matrix
 *     is not positive definite, then lambda = 1e-10 * trace / n_coef.
 *   - Likelihood: Poisson, mu_i = E eta_i(x).  At fixed x the ML energy is
 *     E = S/H (S = sum s_i, H = sum eta_i), which is the ratio of Sec. 5.1.2.2;
 *     substituting it, the search maximises F(x) = sum s_i ln eta_i - S ln H.
 *     eta_i <= 1e-30 is replaced by 1e-30.
 *   - Contracting grid: N x N (x N_z) nodes, flat index (iz, iy, ix) row
 *     major, node = centre + (index - (N-1)/2) * step; step *= shrink after
 *     each iteration; nodes outside the LRF domain score -inf; ties go to the
 *     lowest flat index; the result is the best node of the last grid.
 *   - Start: COG with the detector's relative gains, clamped into the XY
 *     domain of an XY/XYZ LRF; z starts at a given z0.
 *   - Reported logL: sum_i [ s_i ln mu_i - mu_i - lgamma(s_i+1) ] at the
 *     result, with s_i = 0 terms equal to -mu_i.
 *   - Chi-squared: Pearson's sum over sensors with mu_i > 0 of
 *     (s_i - mu_i)^2 / mu_i, divided by n_s - 3.
 *   - Random shift: normal, sigma given, Box-Muller of a Philox4x32-10 block.
 *
 * Every function is a direct transcription of a definition; no blocking,
 * fusion or reordering is done beyond what the definition states.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_RADIAL 1
#define OR_XY 2
#define OR_XYZ 3
#define OR_COMPOSITE 4 /* Sec. 6.1.1: an axial LRF plus an XY LRF */
#define OR_AXIAL_Z 5   /* Sec. 6.1.2: axial in the XY plane, varying along z */
#define OR_SLICED 6    /* Sec. 6.1.2: XY LRFs on z planes, linear in z between them */

#define OR_EVT_OK 0
#define OR_PI_SYM 3.14159265358979323846
#define OR_EVT_ZERO_SIGNAL 2
#define OR_EVT_BAD_SIGNAL 3
#define OR_EVT_OUT_OF_DOMAIN 4

#define OR_ETA_FLOOR 1e-30

/* Optional planted mistakes, used only by the test that shows the pins catch
 * them.  OR_MUTANT == 0 (the default build) is the oracle itself. */
#ifndef OR_MUTANT
#define OR_MUTANT 0
#endif

/* ------------------------------------------------------------------------ */
/* Uniform cubic B-splines (Cox-de Boor recursion)                           */
/* ------------------------------------------------------------------------ */

/* Knot t_j of the extended uniform knot vector, j = 0 .. n+6. */
static double or_knot(int n_int, double lo, double hi, int j)
{
    double h = (hi - lo) / (double)n_int;
    return lo + (double)(j - 3) * h;
}

/* Knot span m (3 <= m <= n+2) with t_m <= x < t_{m+1}; x == hi is put into
 * the last span.  Returns -1 when x lies outside [lo, hi]. */
static int or_span(int n_int, double lo, double hi, double x)
{
    if (!(x >= lo && x <= hi)) return -1;
    if (x == hi) return n_int + 2;
    /* first guess from the uniform spacing, then settle it by comparing
     * against the knots themselves */
    int m = 3 + (int)floor((x - lo) / ((hi - lo) / (double)n_int));
    if (m < 3) m = 3;
    if (m > n_int + 2) m = n_int + 2;
    while (m > 3 && x < or_knot(n_int, lo, hi, m)) --m;
    while (m < n_int + 2 && x >= or_knot(n_int, lo, hi, m + 1)) ++m;
    return m;
}

/* All n+3 cubic basis values B_{j,3}(x), j = 0..n+2, by the full Cox-de Boor
 * recursion B_{j,0} = [t_j <= x < t_{j+1}],
 * B_{j,k} = (x - t_j)/(t_{j+k} - t_j) B_{j,k-1}
 *         + (t_{j+k+1} - x)/(t_{j+k+1} - t_{j+1}) B_{j+1,k-1}.
 * Returns the span m, or -1 (all zeros) when x is outside [lo, hi]. */
int or_bspline_basis_all(int n_int, double lo, double hi, double x, double *B)
{
    int nk = n_int + 7;        /* knots */
    int nb0 = nk - 1;          /* degree-0 functions */
    double *N = (double *)calloc((size_t)nb0, sizeof(double));
    int m = or_span(n_int, lo, hi, x);
    for (int j = 0; j < n_int + 3; ++j) B[j] = 0.0;
    if (m < 0) { free(N); return -1; }
    N[m] = 1.0;
    for (int k = 1; k <= 3; ++k) {
        for (int j = 0; j + k < nb0; ++j) {
            double tj = or_knot(n_int, lo, hi, j);
            double tjk = or_knot(n_int, lo, hi, j + k);
            double tj1 = or_knot(n_int, lo, hi, j + 1);
            double tjk1 = or_knot(n_int, lo, hi, j + k + 1);
            double left = (x - tj) / (tjk - tj) * N[j];
#if OR_MUTANT == 2
            double right = (x - tjk1) / (tjk1 - tj1) * N[j + 1];
#else
            double right = (tjk1 - x) / (tjk1 - tj1) * N[j + 1];
#endif
            N[j] = left + right;
        }
    }
    for (int j = 0; j < n_int + 3; ++j) B[j] = N[j];
    free(N);
    return m;
}

/* The four basis functions that can be non-zero at x, B_{m-3..m,3}(x), by
 * the same recursion restricted to the triangle of non-zero terms (the
 * support of B_{j,3} is [t_j, t_{j+4})).  Returns the index m-3 of the first
 * one (0 .. n-1), or -1 when x is outside [lo, hi]. */
int or_bspline_basis4(int n_int, double lo, double hi, double x, double B[4])
{
    double full[4][4];
    int m = or_span(n_int, lo, hi, x);
    if (m < 0) return -1;
    /* full[k][r] holds B_{m-k+r, k}(x), r = 0..k */
    full[0][0] = 1.0;
    for (int k = 1; k <= 3; ++k) {
        for (int r = 0; r <= k; ++r) {
            int j = m - k + r;
            double v = 0.0;
            if (r >= 1) { /* B_{j,k-1} term: exists when j >= m-k+1 */
                double tj = or_knot(n_int, lo, hi, j);
#if OR_MUTANT == 9
                double tjk = or_knot(n_int, lo, hi, j + k + 1);
#else
                double tjk = or_knot(n_int, lo, hi, j + k);
#endif
                v += (x - tj) / (tjk - tj) * full[k - 1][r - 1];
            }
            if (r <= k - 1) { /* B_{j+1,k-1} term */
                double tj1 = or_knot(n_int, lo, hi, j + 1);
                double tjk1 = or_knot(n_int, lo, hi, j + k + 1);
                v += (tjk1 - x) / (tjk1 - tj1) * full[k - 1][r];
            }
            full[k][r] = v;
        }
    }
    for (int r = 0; r < 4; ++r) B[r] = full[3][r];
    return m - 3;
}

/* ------------------------------------------------------------------------ */
/* Light response functions (Sec. 6, 6.1, 6.2)                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int type;               /* OR_RADIAL .. OR_SLICED */
    int n_sensors;
    int n_int[3];           /* intervals per axis (radial: axis 0 = r; axial+z: r, z) */
    double lo[3], hi[3];    /* domain per axis (sliced: z planes span lo[2]..hi[2]) */
    int shared;             /* radial only: one coefficient set for all sensors */
    const double *coef;     /* [n_sets][n_coef], x fastest, then y, then z */
    const double *gain;     /* [n_sensors] relative gain on a radial LRF; NULL = 1 */
    const double *sensor_xy;/* [n_sensors][2] sensor centres (mm) */
    int n_int_r;            /* composite: intervals of the axial part on [0, hi_r] */
    double hi_r;
    int n_planes;           /* sliced: number of z planes (>= 2) */
    const int *group;       /* radial, not shared: nullable [n_sensors] coefficient set of each sensor (Sec. 6.2
                               groups); XY: the symmetry class of each sensor */
    const int *op;          /* XY with groups: [n_sensors] the symmetry operation of each sensor (or_sym_op) */
    double sym_c[2];        /* XY with groups: the centre of the operations */
} or_lrf;

/* Symmetry operation k of the plane about a centre (Sec. 6.2 groups by the
 * rotation and reflection symmetry of the array): the rotation by (k mod 12)
 * x 30 degrees, preceded for k >= 12 by the reflection y -> -y; M is the
 * 2 x 2 matrix, row-major. */
static void or_sym_op(int k, double M[4])
{
    double t = (double)(k % 12) * (OR_PI_SYM / 6.0), c = cos(t), s = sin(t);
    /* exact values at multiples of 90 degrees */
    if (k % 3 == 0) {
        int q = (k % 12) / 3;
        c = q == 0 ? 1.0 : (q == 2 ? -1.0 : 0.0);
        s = q == 1 ? 1.0 : (q == 3 ? -1.0 : 0.0);
    }
    double f = k >= 12 ? -1.0 : 1.0;
    M[0] = c;
    M[1] = -s * f;
    M[2] = s;
    M[3] = c * f;
}

/* (x, y) mapped into the frame of sensor i's class representative:
 * M^T ((x, y) - c) + c */
static void or_sym_point(const or_lrf *L, int i, double *x, double *y)
{
    double M[4], dx = *x - L->sym_c[0], dy = *y - L->sym_c[1];
    or_sym_op(L->op[i], M);
#if OR_MUTANT == 30
    *x = M[0] * dx + M[1] * dy + L->sym_c[0];
    *y = M[2] * dx + M[3] * dy + L->sym_c[1];
#else
    *x = M[0] * dx + M[2] * dy + L->sym_c[0];
    *y = M[1] * dx + M[3] * dy + L->sym_c[1];
#endif
}

/* the coefficient set of sensor i of a radial LRF: one for all (shared), its
 * group's (grouped) or its own */
static int or_set_of(const or_lrf *L, int i)
{
    if (L->shared) return 0;
#if OR_MUTANT == 29
    return i;
#else
    return L->group ? L->group[i] : i;
#endif
}

/* LRF types with a z coordinate, and with an XY box as domain */
static int or_is_3d(int type) { return type == OR_XYZ || type == OR_AXIAL_Z || type == OR_SLICED; }
static int or_has_box(int type) { return type == OR_XY || type == OR_XYZ || type == OR_COMPOSITE || type == OR_SLICED; }

static int or_n_coef(const or_lrf *L)
{
    if (L->type == OR_RADIAL) return L->n_int[0] + 3;
    if (L->type == OR_XY || L->type == OR_AXIAL_Z) return (L->n_int[0] + 3) * (L->n_int[1] + 3);
    if (L->type == OR_COMPOSITE) return (L->n_int_r + 3) + (L->n_int[0] + 3) * (L->n_int[1] + 3);
    if (L->type == OR_SLICED) return L->n_planes * (L->n_int[0] + 3) * (L->n_int[1] + 3);
    return (L->n_int[0] + 3) * (L->n_int[1] + 3) * (L->n_int[2] + 3);
}

/* A two-dimensional tensor spline (axis u fastest in c) at (u, v); *ok = 0
 * outside its box. */
static double or_spline2(int n0, double lo0, double hi0, int n1, double lo1, double hi1, const double *c, double u,
                         double v, int *ok)
{
    double B0[4], B1[4];
    int j0 = or_bspline_basis4(n0, lo0, hi0, u, B0);
    int j1 = or_bspline_basis4(n1, lo1, hi1, v, B1);
    *ok = j0 >= 0 && j1 >= 0;
    if (!*ok) return 0.0;
    double f = 0.0;
    for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a)
#if OR_MUTANT == 20
            f += c[(size_t)(j0 + a) * (n1 + 3) + (size_t)(j1 + b)] * B0[a] * B1[b];
#else
            f += c[(size_t)(j1 + b) * (n0 + 3) + (size_t)(j0 + a)] * B0[a] * B1[b];
#endif
    return f;
}

/* eta_i at (x, y, z) from the B-spline expansion.  *ok = 0 when the point
 * lies outside the LRF's domain for this sensor. */
static double or_lrf_eta(const or_lrf *L, int i, double x, double y, double z, int *ok)
{
    int nc = or_n_coef(L);
    *ok = 1;
    if (L->type == OR_COMPOSITE) {
        /* the axial part at the distance r, plus the XY part */
        const double *c = L->coef + (size_t)i * nc;
        double dx = x - L->sensor_xy[2 * i], dy = y - L->sensor_xy[2 * i + 1];
        double B[4];
        int j0 = or_bspline_basis4(L->n_int_r, 0.0, L->hi_r, sqrt(dx * dx + dy * dy), B);
        int okxy;
        double fxy = or_spline2(L->n_int[0], L->lo[0], L->hi[0], L->n_int[1], L->lo[1], L->hi[1],
                                c + L->n_int_r + 3, x, y, &okxy);
        if (j0 < 0 || !okxy) { *ok = 0; return 0.0; }
        double fa = 0.0;
        for (int a = 0; a < 4; ++a) fa += c[j0 + a] * B[a];
        return fa + fxy;
    }
    if (L->type == OR_AXIAL_Z) {
        /* one spline of (r, z), r the distance in the XY plane */
        double dx = x - L->sensor_xy[2 * i], dy = y - L->sensor_xy[2 * i + 1];
        return or_spline2(L->n_int[0], L->lo[0], L->hi[0], L->n_int[1], L->lo[1], L->hi[1],
                          L->coef + (size_t)i * nc, sqrt(dx * dx + dy * dy), z, ok);
    }
    if (L->type == OR_SLICED) {
        /* linear interpolation between the XY LRFs of the two closest planes */
        if (!(z >= L->lo[2] && z <= L->hi[2])) { *ok = 0; return 0.0; }
        int m = L->n_planes, ncxy = nc / m;
        double dz = (L->hi[2] - L->lo[2]) / (double)(m - 1), u = (z - L->lo[2]) / dz;
        int j = (int)floor(u);
        if (j > m - 2) j = m - 2;
        if (j < 0) j = 0;
        double w = u - (double)j;
        const double *c = L->coef + (size_t)i * nc;
        int ok0, ok1;
        double f0 = or_spline2(L->n_int[0], L->lo[0], L->hi[0], L->n_int[1], L->lo[1], L->hi[1],
                               c + (size_t)j * ncxy, x, y, &ok0);
        double f1 = or_spline2(L->n_int[0], L->lo[0], L->hi[0], L->n_int[1], L->lo[1], L->hi[1],
                               c + (size_t)(j + 1) * ncxy, x, y, &ok1);
        if (!ok0 || !ok1) { *ok = 0; return 0.0; }
#if OR_MUTANT == 19
        return w * f0 + (1.0 - w) * f1;
#else
        return (1.0 - w) * f0 + w * f1;
#endif
    }
    if (L->type == OR_RADIAL) {
        const double *c = L->coef + (size_t)or_set_of(L, i) * nc;
        double dx = x - L->sensor_xy[2 * i], dy = y - L->sensor_xy[2 * i + 1];
        double r = sqrt(dx * dx + dy * dy);
        double B[4];
        int j0 = or_bspline_basis4(L->n_int[0], L->lo[0], L->hi[0], r, B);
        if (j0 < 0) { *ok = 0; return 0.0; }
        double f = 0.0;
        for (int a = 0; a < 4; ++a) f += c[j0 + a] * B[a];
        double g = L->gain ? L->gain[i] : 1.0;
        return g * f;
    }
    const double *c = L->coef + (size_t)i * nc;
    double gs = 1.0;
    if (L->type == OR_XY && L->group) {
        /* symmetry class: the representative's LRF at the mapped point, times the gain */
        c = L->coef + (size_t)L->group[i] * nc;
        or_sym_point(L, i, &x, &y);
        gs = L->gain ? L->gain[i] : 1.0;
    }
    double Bx[4], By[4], Bz[4] = {1.0, 0.0, 0.0, 0.0};
    int jx = or_bspline_basis4(L->n_int[0], L->lo[0], L->hi[0], x, Bx);
    int jy = or_bspline_basis4(L->n_int[1], L->lo[1], L->hi[1], y, By);
    int jz = 0, nz = 1;
    if (L->type == OR_XYZ) {
        jz = or_bspline_basis4(L->n_int[2], L->lo[2], L->hi[2], z, Bz);
        nz = 4;
    }
    if (jx < 0 || jy < 0 || jz < 0) { *ok = 0; return 0.0; }
    int sx = L->n_int[0] + 3, sy = L->n_int[1] + 3;
    double f = 0.0;
    for (int cz = 0; cz < nz; ++cz)
        for (int b = 0; b < 4; ++b)
            for (int a = 0; a < 4; ++a) {
#if OR_MUTANT == 3
                size_t idx = ((size_t)(jz + cz) * sy + (size_t)(jx + a)) * sx + (size_t)(jy + b);
#else
                size_t idx = ((size_t)(jz + cz) * sy + (size_t)(jy + b)) * sx + (size_t)(jx + a);
#endif
                f += c[idx] * Bx[a] * By[b] * Bz[cz];
            }
    return gs * f;
}

/* Sensor classes by the rotation and reflection symmetry of the array (Sec.
 * 6.2): the centre is the mean sensor position; an operation of or_sym_op is
 * a symmetry when it maps every sensor onto a sensor (within tol); sensors
 * taken in index order open a class unless already reached, and every
 * symmetry (in table order) maps the class's first sensor onto the members
 * it reaches first, recording that operation.  Returns the number of
 * classes; group[i], op[i] and the centre c receive the result. */
int or_sensor_symmetry(int n, const double *sensor_xy, double tol, int *group, int *op, double *c)
{
    double cx = 0.0, cy = 0.0;
    for (int i = 0; i < n; ++i) {
        cx += sensor_xy[2 * i];
        cy += sensor_xy[2 * i + 1];
    }
    cx /= n;
    cy /= n;
    c[0] = cx;
    c[1] = cy;
    int valid[24], n_valid = 0;
    for (int k = 0; k < 24; ++k) {
        double M[4];
        or_sym_op(k, M);
        int ok = 1;
        for (int i = 0; i < n && ok; ++i) {
            double dx = sensor_xy[2 * i] - cx, dy = sensor_xy[2 * i + 1] - cy;
            double x = M[0] * dx + M[1] * dy + cx, y = M[2] * dx + M[3] * dy + cy;
            int hit = 0;
            for (int j = 0; j < n && !hit; ++j) hit = hypot(sensor_xy[2 * j] - x, sensor_xy[2 * j + 1] - y) <= tol;
            ok = hit;
        }
        if (ok) valid[n_valid++] = k;
    }
    for (int i = 0; i < n; ++i) group[i] = -1;
    int g = 0;
    for (int r = 0; r < n; ++r) {
        if (group[r] >= 0) continue;
        double dx = sensor_xy[2 * r] - cx, dy = sensor_xy[2 * r + 1] - cy;
        for (int v = 0; v < n_valid; ++v) {
            double M[4];
            or_sym_op(valid[v], M);
            double x = M[0] * dx + M[1] * dy + cx, y = M[2] * dx + M[3] * dy + cy;
            for (int j = 0; j < n; ++j)
                if (group[j] < 0 && hypot(sensor_xy[2 * j] - x, sensor_xy[2 * j + 1] - y) <= tol) {
                    group[j] = g;
                    op[j] = valid[v];
                    break;
                }
        }
        ++g;
    }
    return g;
}

/* Sensor groups by distance from the array's centre (Sec. 6.2): the centre
 * is the mean sensor position; sensors are taken in order of increasing
 * distance d (ties by index) and a new group starts when d exceeds the
 * distance of the current group's first sensor by more than tol.  group[i]
 * receives the group of sensor i (0 = the innermost); returns the number of
 * groups. */
int or_sensor_rings(int n, const double *sensor_xy, double tol, int *group)
{
    double cx = 0.0, cy = 0.0;
    for (int i = 0; i < n; ++i) {
        cx += sensor_xy[2 * i];
        cy += sensor_xy[2 * i + 1];
    }
    cx /= n;
    cy /= n;
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    int *order = (int *)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        d[i] = hypot(sensor_xy[2 * i] - cx, sensor_xy[2 * i + 1] - cy);
        order[i] = i;
    }
    /* insertion sort by (d, index) */
    for (int a = 1; a < n; ++a) {
        int v = order[a], b = a - 1;
        while (b >= 0 && (d[order[b]] > d[v] || (d[order[b]] == d[v] && order[b] > v))) {
            order[b + 1] = order[b];
            --b;
        }
        order[b + 1] = v;
    }
    int g = -1;
    double first = 0.0;
    for (int a = 0; a < n; ++a) {
        int i = order[a];
        if (g < 0 || d[i] - first > tol) {
            ++g;
            first = d[i];
        }
        group[i] = g;
    }
    free(d);
    free(order);
    return g + 1;
}

/* eta for every (point, sensor): out[p * n_sensors + i]; NaN outside. */
void or_lrf_eval(const or_lrf *L, long n_pts, const double *pts, int dim, double *out)
{
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n_pts; ++p) {
        double x = pts[p * dim], y = dim > 1 ? pts[p * dim + 1] : 0.0;
        double z = dim > 2 ? pts[p * dim + 2] : 0.0;
        for (int i = 0; i < L->n_sensors; ++i) {
            int ok;
            double v = or_lrf_eta(L, i, x, y, z, &ok);
            out[p * L->n_sensors + i] = ok ? v : NAN;
        }
    }
}

/* Value of one B-spline expansion (no sensor geometry) at d-dim points:
 * f(p) = sum c_{j..} B_j(p_x) B_k(p_y) [B_l(p_z)].  Used to check fits. */
void or_spline_eval(int dim, const int *n_int, const double *lo, const double *hi,
                    const double *coef, long n_pts, const double *pts, double *out)
{
    for (long p = 0; p < n_pts; ++p) {
        double B[3][4] = {{1, 0, 0, 0}, {1, 0, 0, 0}, {1, 0, 0, 0}};
        int j0[3] = {0, 0, 0}, nn[3] = {1, 1, 1}, st[3] = {1, 1, 1};
        int bad = 0;
        for (int a = 0; a < dim; ++a) {
            j0[a] = or_bspline_basis4(n_int[a], lo[a], hi[a], pts[p * dim + a], B[a]);
            if (j0[a] < 0) bad = 1;
            nn[a] = 4;
        }
        if (bad) { out[p] = NAN; continue; }
        st[0] = 1;
        st[1] = n_int[0] + 3;
        st[2] = (n_int[0] + 3) * (dim > 1 ? n_int[1] + 3 : 1);
        double f = 0.0;
        for (int c = 0; c < nn[2]; ++c)
            for (int b = 0; b < nn[1]; ++b)
                for (int a = 0; a < nn[0]; ++a)
                    f += coef[(size_t)(j0[0] + a) * st[0] + (size_t)(j0[1] + b) * st[1] +
                              (size_t)(j0[2] + c) * st[2]] * B[0][a] * B[1][b] * B[2][c];
        out[p] = f;
    }
}

/* ------------------------------------------------------------------------ */
/* Least-squares B-spline fit (Sec. 6: LRFs computed from (position, signal) */
/* datasets); normal equations + Cholesky, FP64.                             */
/* ------------------------------------------------------------------------ */

/* Cholesky A = L L^T in place (lower triangle).  Returns 0, or -1 when a
 * pivot is not positive. */
static int or_cholesky(int n, double *A)
{
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(d > 0.0)) return -1;
        double ljj = sqrt(d);
        A[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double v = A[(size_t)i * n + j];
#if OR_MUTANT == 8
            for (int k = 0; k < j; ++k) v -= A[(size_t)i * n + k] * A[(size_t)k * n + j];
#else
            for (int k = 0; k < j; ++k) v -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
#endif
            A[(size_t)i * n + j] = v / ljj;
        }
    }
    return 0;
}

/* Solve L L^T x = b in place. */
static void or_cholesky_solve(int n, const double *Lm, double *b)
{
    for (int i = 0; i < n; ++i) {
        double v = b[i];
        for (int k = 0; k < i; ++k) v -= Lm[(size_t)i * n + k] * b[k];
        b[i] = v / Lm[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double v = b[i];
        for (int k = i + 1; k < n; ++k) v -= Lm[(size_t)k * n + i] * b[k];
        b[i] = v / Lm[(size_t)i * n + i];
    }
}

/* Fit coefficients of a dim-dimensional tensor-product cubic B-spline to
 * n_out value sets sampled at the same n_pts points:
 *   minimise sum_p (f(p) - v[p][o])^2  for each o.
 * coef_out[o][n_coef].  Returns 0 (plain solve), 1 (ridge retry used) or
 * -1 (failure).  *ridge_used receives the lambda that was applied. */
int or_lrf_fit(int dim, const int *n_int, const double *lo, const double *hi,
               long n_pts, const double *pts, int n_out, const double *vals,
               double ridge, double *coef_out, double *ridge_used)
{
    int st[3] = {1, 1, 1}, nc = 1;
    for (int a = 0; a < dim; ++a) nc *= n_int[a] + 3;
    st[1] = n_int[0] + 3;
    st[2] = (n_int[0] + 3) * (dim > 1 ? n_int[1] + 3 : 1);
    double *A = (double *)calloc((size_t)nc * nc, sizeof(double));
    double *Bv = (double *)calloc((size_t)nc * n_out, sizeof(double));
    double *A0 = (double *)malloc((size_t)nc * nc * sizeof(double));
    if (!A || !Bv || !A0) { free(A); free(Bv); free(A0); return -1; }
    int nterm = 1;
    for (int a = 0; a < dim; ++a) nterm *= 4;
    int *idx = (int *)malloc(sizeof(int) * nterm);
    double *w = (double *)malloc(sizeof(double) * nterm);
    /* Assemble B^T B and B^T v from the non-zero basis products of each point. */
    for (long p = 0; p < n_pts; ++p) {
        double B[3][4] = {{1, 0, 0, 0}, {1, 0, 0, 0}, {1, 0, 0, 0}};
        int j0[3] = {0, 0, 0}, nn[3] = {1, 1, 1}, bad = 0;
        for (int a = 0; a < dim; ++a) {
            j0[a] = or_bspline_basis4(n_int[a], lo[a], hi[a], pts[p * dim + a], B[a]);
            if (j0[a] < 0) bad = 1;
            nn[a] = 4;
        }
        if (bad) continue; /* samples outside the domain carry no information */
        int t = 0;
        for (int c = 0; c < nn[2]; ++c)
            for (int b = 0; b < nn[1]; ++b)
                for (int a = 0; a < nn[0]; ++a) {
                    idx[t] = (j0[0] + a) * st[0] + (j0[1] + b) * st[1] + (j0[2] + c) * st[2];
                    w[t] = B[0][a] * B[1][b] * B[2][c];
                    ++t;
                }
        for (int u = 0; u < t; ++u) {
            for (int v = 0; v < t; ++v) A[(size_t)idx[u] * nc + idx[v]] += w[u] * w[v];
            for (int o = 0; o < n_out; ++o) Bv[(size_t)o * nc + idx[u]] += w[u] * vals[(size_t)p * n_out + o];
        }
    }
    free(idx);
    free(w);
    memcpy(A0, A, (size_t)nc * nc * sizeof(double));
    double lam = ridge;
    int rc = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        memcpy(A, A0, (size_t)nc * nc * sizeof(double));
        for (int j = 0; j < nc; ++j) A[(size_t)j * nc + j] += lam;
        if (or_cholesky(nc, A) == 0) break;
        if (attempt == 1) { rc = -1; break; }
        double tr = 0.0;
        for (int j = 0; j < nc; ++j) tr += A0[(size_t)j * nc + j];
        lam = 1e-10 * tr / (double)nc;
        rc = 1;
    }
    if (rc >= 0) {
        for (int o = 0; o < n_out; ++o) {
            memcpy(coef_out + (size_t)o * nc, Bv + (size_t)o * nc, sizeof(double) * nc);
            or_cholesky_solve(nc, A, coef_out + (size_t)o * nc);
        }
    }
    if (ridge_used) *ridge_used = lam;
    free(A);
    free(A0);
    free(Bv);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Centroid (Sec. 5.1.1)                                                     */
/* ------------------------------------------------------------------------ */

/* x = sum X_i s_i/g_i / sum s_i/g_i (and y).  Returns the denominator. */
static double or_cog1(int n_s, const double *s, const double *sensor_xy, const double *gain,
                      double *x, double *y)
{
    double num_x = 0.0, num_y = 0.0, den = 0.0;
    for (int i = 0; i < n_s; ++i) {
        double g = gain ? gain[i] : 1.0;
#if OR_MUTANT == 4
        double w = s[i];
        (void)g;
#else
        double w = s[i] / g;
#endif
        num_x += sensor_xy[2 * i] * w;
        num_y += sensor_xy[2 * i + 1] * w;
        den += w;
    }
    *x = num_x / den;
    *y = num_y / den;
    return den;
}

void or_cog(long n_e, int n_s, const double *sig, const double *sensor_xy, const double *gain,
            double *out_xy)
{
    for (long e = 0; e < n_e; ++e)
        or_cog1(n_s, sig + e * n_s, sensor_xy, gain, &out_xy[2 * e], &out_xy[2 * e + 1]);
}

/* ------------------------------------------------------------------------ */
/* Likelihood (Sec. 5.1.2, energy ratio of Sec. 5.1.2.2)                     */
/* ------------------------------------------------------------------------ */

/* Whether every LRF of the sensors with act[i] (all when act is NULL) is
 * defined at a node: within reach of each sensor for the axial parts
 * (radial, composite, axial+z), inside the XY box, inside the z range. */
static int or_valid_act(const or_lrf *L, const int *act, double x, double y, double z)
{
    if (L->type == OR_RADIAL || L->type == OR_COMPOSITE || L->type == OR_AXIAL_Z) {
        double rlo = L->type == OR_COMPOSITE ? 0.0 : L->lo[0];
        double rhi = L->type == OR_COMPOSITE ? L->hi_r : L->hi[0];
        for (int i = 0; i < L->n_sensors; ++i) {
            if (act && !act[i]) continue;
            double dx = x - L->sensor_xy[2 * i], dy = y - L->sensor_xy[2 * i + 1];
            double r = sqrt(dx * dx + dy * dy);
            if (!(r >= rlo && r <= rhi)) return 0;
        }
    }
    if (L->type == OR_XY && L->group) {
        /* symmetry classes: every sensor's mapped point inside the box */
        for (int i = 0; i < L->n_sensors; ++i) {
            if (act && !act[i]) continue;
            double u = x, v = y;
            or_sym_point(L, i, &u, &v);
            if (!(u >= L->lo[0] && u <= L->hi[0] && v >= L->lo[1] && v <= L->hi[1])) return 0;
        }
        return 1;
    }
    if (or_has_box(L->type) && !(x >= L->lo[0] && x <= L->hi[0] && y >= L->lo[1] && y <= L->hi[1])) return 0;
    if (L->type == OR_XYZ && !(z >= L->lo[2] && z <= L->hi[2])) return 0;
    if (L->type == OR_SLICED && !(z >= L->lo[2] && z <= L->hi[2])) return 0;
    if (L->type == OR_AXIAL_Z && !(z >= L->lo[1] && z <= L->hi[1])) return 0;
    return 1;
}

/* Whether a node is inside the LRF's domain. */
static int or_node_valid(const or_lrf *L, double x, double y, double z)
{
    return or_valid_act(L, NULL, x, y, z);
}

static double or_eta_floored(const or_lrf *L, int i, double x, double y, double z)
{
    int ok;
    double v = or_lrf_eta(L, i, x, y, z, &ok);
    return v > OR_ETA_FLOOR ? v : OR_ETA_FLOOR;
}

/* Profiled objective F = sum s_i ln eta_i - S ln H; -inf outside the domain. */
static double or_objective(const or_lrf *L, const double *s, double S, double x, double y, double z)
{
    if (!or_node_valid(L, x, y, z)) return -INFINITY;
    double acc = 0.0, H = 0.0;
    for (int i = 0; i < L->n_sensors; ++i) {
        double eta = or_eta_floored(L, i, x, y, z);
        if (s[i] != 0.0) acc += s[i] * log(eta);
        H += eta;
    }
#if OR_MUTANT == 1
    (void)S;
    return acc;
#else
    return acc - S * log(H);
#endif
}

/* ML energy E = S / H and the full Poisson log-likelihood at (x, y, z). */
static void or_energy_logl(const or_lrf *L, const double *s, double x, double y, double z,
                           double *E_out, double *logL_out)
{
    double S = 0.0, H = 0.0;
    for (int i = 0; i < L->n_sensors; ++i) {
        S += s[i];
        H += or_eta_floored(L, i, x, y, z);
    }
#if OR_MUTANT == 6
    double E = H / S;
#else
    double E = S / H;
#endif
    double ll = 0.0;
    for (int i = 0; i < L->n_sensors; ++i) {
        double mu = E * or_eta_floored(L, i, x, y, z);
#if OR_MUTANT == 7
        ll += (s[i] != 0.0 ? s[i] * log(mu) : 0.0) - mu - lgamma(s[i]);
#else
        ll += (s[i] != 0.0 ? s[i] * log(mu) : 0.0) - mu - lgamma(s[i] + 1.0);
#endif
    }
    *E_out = E;
    *logL_out = ll;
}

/* Full Poisson logL at an arbitrary energy, for the tests that check the
 * profiled energy is the maximiser. */
double or_logl_at_energy(const or_lrf *L, const double *s, double x, double y, double z, double E)
{
    double ll = 0.0;
    for (int i = 0; i < L->n_sensors; ++i) {
        double mu = E * or_eta_floored(L, i, x, y, z);
        ll += (s[i] != 0.0 ? s[i] * log(mu) : 0.0) - mu - lgamma(s[i] + 1.0);
    }
    return ll;
}

/* F at given points, one per event: out[e]. */
void or_objective_at(const or_lrf *L, long n_e, const double *sig, const double *xyz, double *out)
{
#pragma omp parallel for schedule(static)
    for (long e = 0; e < n_e; ++e) {
        const double *s = sig + e * L->n_sensors;
        double S = 0.0;
        for (int i = 0; i < L->n_sensors; ++i) S += s[i];
        out[e] = or_objective(L, s, S, xyz[3 * e], xyz[3 * e + 1], xyz[3 * e + 2]);
    }
}

/* E and full logL at given points, one per event. */
void or_energy_logl_at(const or_lrf *L, long n_e, const double *sig, const double *xyz,
                       double *E, double *logL)
{
#pragma omp parallel for schedule(static)
    for (long e = 0; e < n_e; ++e)
        or_energy_logl(L, sig + e * L->n_sensors, xyz[3 * e], xyz[3 * e + 1], xyz[3 * e + 2],
                       &E[e], &logL[e]);
}

/* ------------------------------------------------------------------------ */
/* Contracting grids (Sec. 5.1.2.2)                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n_xy;       /* nodes per axis in x and y (odd) */
    int n_z;        /* nodes along z (odd; 1 for 2D LRFs) */
    int iters;      /* number of grids */
    double shrink;  /* step factor between grids */
    double step_xy; /* first grid's node spacing in x and y */
    double step_z;  /* first grid's node spacing in z */
    double z0;      /* start z for XYZ LRFs */
} or_cgs_params;

/* Start position: the given one when start_xyz is not NULL, else the COG
 * clamped into the LRF's XY box (XY/XYZ) with z = z0.  Returns an event
 * status. */
static int or_start(const or_lrf *L, const or_cgs_params *P, const double *gain_cog,
                    const double *start_xyz, const double *s, double *cx, double *cy, double *cz,
                    double *S_out)
{
    double S = 0.0;
    for (int i = 0; i < L->n_sensors; ++i) {
        if (!isfinite(s[i]) || s[i] < 0.0) return OR_EVT_BAD_SIGNAL;
        S += s[i];
    }
    *S_out = S;
    if (!(S > 0.0)) return OR_EVT_ZERO_SIGNAL;
    if (start_xyz) {
        *cx = start_xyz[0];
        *cy = start_xyz[1];
        *cz = start_xyz[2];
        if (!or_node_valid(L, *cx, *cy, *cz)) return OR_EVT_OUT_OF_DOMAIN;
        return OR_EVT_OK;
    }
    or_cog1(L->n_sensors, s, L->sensor_xy, gain_cog, cx, cy);
    *cz = or_is_3d(L->type) ? P->z0 : 0.0;
    if (or_has_box(L->type)) {
        if (*cx < L->lo[0]) *cx = L->lo[0];
        if (*cx > L->hi[0]) *cx = L->hi[0];
        if (*cy < L->lo[1]) *cy = L->lo[1];
        if (*cy > L->hi[1]) *cy = L->hi[1];
    }
    if (!or_node_valid(L, *cx, *cy, *cz)) return OR_EVT_OUT_OF_DOMAIN;
    return OR_EVT_OK;
}

/* Node coordinates of flat index k on the grid centred at (cx, cy, cz). */
static void or_node(const or_cgs_params *P, double cx, double cy, double cz, double sxy, double sz,
                    int k, double *x, double *y, double *z)
{
    int n = P->n_xy, c = (P->n_xy - 1) / 2, cz_i = (P->n_z - 1) / 2;
    int ix = k % n, iy = (k / n) % n, iz = k / (n * n);
    *x = cx + (double)(ix - c) * sxy;
    *y = cy + (double)(iy - c) * sxy;
    *z = cz + (double)(iz - cz_i) * sz;
}

static void or_set_nan(double *xyz, double *E, double *logL)
{
    xyz[0] = xyz[1] = xyz[2] = NAN;
    *E = NAN;
    *logL = NAN;
}

/* Plain contracting-grid search for each event.  start_xyz[e][3] gives the
 * start positions (nullable: COG).  trace[e][it] receives the flat index of
 * the chosen node of grid it (nullable). */
void or_cgs(const or_lrf *L, const or_cgs_params *P, const double *gain_cog,
            const double *start_xyz, long n_e, const double *sig, double *xyz, double *E,
            double *logL, int *status, int *trace)
{
    int nodes = P->n_xy * P->n_xy * P->n_z;
#pragma omp parallel for schedule(dynamic, 16)
    for (long e = 0; e < n_e; ++e) {
        const double *s = sig + e * L->n_sensors;
        double cx, cy, cz, S;
        int st = or_start(L, P, gain_cog, start_xyz ? start_xyz + 3 * e : NULL, s, &cx, &cy, &cz,
                          &S);
        status[e] = st;
        if (st != OR_EVT_OK) {
            or_set_nan(&xyz[3 * e], &E[e], &logL[e]);
            if (trace) for (int it = 0; it < P->iters; ++it) trace[e * P->iters + it] = -1;
            continue;
        }
        double sxy = P->step_xy, sz = P->step_z;
        for (int it = 0; it < P->iters; ++it) {
            double best = -INFINITY;
            int best_k = -1;
            for (int k = 0; k < nodes; ++k) {
                double x, y, z;
                or_node(P, cx, cy, cz, sxy, sz, k, &x, &y, &z);
                double F = or_objective(L, s, S, x, y, z);
#if OR_MUTANT == 5
                if (F >= best) { best = F; best_k = k; }
#else
                if (F > best) { best = F; best_k = k; }
#endif
            }
            double x, y, z;
            or_node(P, cx, cy, cz, sxy, sz, best_k, &x, &y, &z);
            cx = x; cy = y; cz = z;
            if (trace) trace[e * P->iters + it] = best_k;
            sxy *= P->shrink;
            sz *= P->shrink;
        }
        xyz[3 * e] = cx;
        xyz[3 * e + 1] = cy;
        xyz[3 * e + 2] = cz;
        or_energy_logl(L, s, cx, cy, cz, &E[e], &logL[e]);
    }
}

/* Replay of another implementation's path (its chosen node per grid, in
 * trace_in) with the tie-certification rule: at every grid the chosen node
 * must score within tau = tau_rel * sum_i |s_i ln p_i(centre)| of the FP64
 * best node (p_i = eta_i / H), and it must lie in the domain.  The replay
 * continues from the chosen node.  Per event: n_tie = grids where the
 * choice was not the FP64 best but within tau; n_bad = grids where it was
 * outside tau or invalid; xyz/E/logL = FP64 values at the replayed end. */
void or_cgs_replay(const or_lrf *L, const or_cgs_params *P, const double *gain_cog,
                   const double *start_xyz, long n_e, const double *sig, const int *trace_in, double tau_rel, double *xyz, double *E,
                   double *logL, int *status, int *n_tie, int *n_bad)
{
    int nodes = P->n_xy * P->n_xy * P->n_z;
#pragma omp parallel for schedule(dynamic, 16)
    for (long e = 0; e < n_e; ++e) {
        const double *s = sig + e * L->n_sensors;
        double cx, cy, cz, S;
        int st = or_start(L, P, gain_cog, start_xyz ? start_xyz + 3 * e : NULL, s, &cx, &cy, &cz,
                          &S);
        status[e] = st;
        n_tie[e] = 0;
        n_bad[e] = 0;
        if (st != OR_EVT_OK) { or_set_nan(&xyz[3 * e], &E[e], &logL[e]); continue; }
        double sxy = P->step_xy, sz = P->step_z;
        for (int it = 0; it < P->iters; ++it) {
            double best = -INFINITY;
            int best_k = -1;
            for (int k = 0; k < nodes; ++k) {
                double x, y, z;
                or_node(P, cx, cy, cz, sxy, sz, k, &x, &y, &z);
                double F = or_objective(L, s, S, x, y, z);
                if (F > best) { best = F; best_k = k; }
            }
            int g = trace_in[e * P->iters + it];
            if (g < 0 || g >= nodes) { n_bad[e]++; g = best_k; }
            double gx, gy, gz;
            or_node(P, cx, cy, cz, sxy, sz, g, &gx, &gy, &gz);
            if (g != best_k) {
                double Fg = or_objective(L, s, S, gx, gy, gz);
                /* tau from the magnitude of the terms summed at the centre */
                double H = 0.0, mag = 0.0;
                for (int i = 0; i < L->n_sensors; ++i) H += or_eta_floored(L, i, cx, cy, cz);
                for (int i = 0; i < L->n_sensors; ++i)
                    mag += fabs(s[i] * log(or_eta_floored(L, i, cx, cy, cz) / H));
                double tau = tau_rel * mag;
                if (isfinite(Fg) && Fg >= best - tau) n_tie[e]++;
                else n_bad[e]++;
            }
            cx = gx; cy = gy; cz = gz;
            sxy *= P->shrink;
            sz *= P->shrink;
        }
        xyz[3 * e] = cx;
        xyz[3 * e + 1] = cy;
        xyz[3 * e + 2] = cz;
        or_energy_logl(L, s, cx, cy, cz, &E[e], &logL[e]);
    }
}

/* ------------------------------------------------------------------------ */
/* Search variants.  Sec. 5.1.2: the match is either maximum likelihood or   */
/* least squares, and sensors whose signal is below a threshold or that lie  */
/* farther than a given distance from the start position can be ignored;    */
/* Sec. 5.1.2.1 / 5.1.2.2: the start is the centroid or the position of the  */
/* sensor with the strongest signal; Sec. 5.3: passive sensors are ignored.  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int criterion;        /* 0: maximum likelihood, 1: least squares */
    int start;            /* 0: centroid, 1: sensor with the strongest signal */
    double min_signal;    /* > 0: sensors with s_i < min_signal are ignored */
    double max_distance;  /* > 0: sensors farther than this from the start are ignored */
    const int *passive;   /* nullable [n_sensors]: nonzero = passive */
} or_variant;

static int or_passive(const or_variant *V, int i) { return V->passive && V->passive[i]; }

/* A node is inside the domain when the LRF of every sensor in the match is
 * defined there (radial: within reach of each; XY / XYZ: inside the box). */
static int or_variant_valid(const or_lrf *L, const int *act, double x, double y, double z)
{
    return or_valid_act(L, act, x, y, z);
}

/* Start position, the sensors in the match (act) and their signal sum.
 * given (nullable): a start position to use instead of the variant's own. */
static int or_variant_start(const or_lrf *L, const or_cgs_params *P, const or_variant *V, const double *gain,
                            const double *s, const double *given, double *cx, double *cy, double *cz, double *S_out,
                            int *act)
{
    int n = L->n_sensors;
    double tot = 0.0;
    for (int i = 0; i < n; ++i) {
        act[i] = 0;
        if (or_passive(V, i)) continue;
        if (!isfinite(s[i]) || s[i] < 0.0) return OR_EVT_BAD_SIGNAL;
        tot += s[i];
    }
    *S_out = 0.0;
    if (!(tot > 0.0)) return OR_EVT_ZERO_SIGNAL;
    if (given) {
        *cx = given[0];
        *cy = given[1];
        *cz = given[2];
    } else if (V->start == 1) {
        int best = -1;
        double bv = -1.0;
        for (int i = 0; i < n; ++i) {
            if (or_passive(V, i)) continue;
            double v = s[i] / (gain ? gain[i] : 1.0);
#if OR_MUTANT == 17
            if (best < 0 || v < bv) {
#else
            if (v > bv) {
#endif
                bv = v;
                best = i;
            }
        }
        *cx = L->sensor_xy[2 * best];
        *cy = L->sensor_xy[2 * best + 1];
    } else {
        double nx = 0.0, ny = 0.0, den = 0.0;
        for (int i = 0; i < n; ++i) {
            if (or_passive(V, i)) continue;
            double w = s[i] / (gain ? gain[i] : 1.0);
            nx += L->sensor_xy[2 * i] * w;
            ny += L->sensor_xy[2 * i + 1] * w;
            den += w;
        }
        *cx = nx / den;
        *cy = ny / den;
    }
    if (!given) *cz = or_is_3d(L->type) ? P->z0 : 0.0;
    if (!given && or_has_box(L->type)) {
        if (*cx < L->lo[0]) *cx = L->lo[0];
        if (*cx > L->hi[0]) *cx = L->hi[0];
        if (*cy < L->lo[1]) *cy = L->lo[1];
        if (*cy > L->hi[1]) *cy = L->hi[1];
    }
    double S = 0.0;
    for (int i = 0; i < n; ++i) {
        if (or_passive(V, i)) continue;
        int a = 1;
        if (V->min_signal > 0.0 && s[i] < V->min_signal) a = 0;
        if (V->max_distance > 0.0) {
#if OR_MUTANT == 18
            double dx = L->sensor_xy[2 * i], dy = L->sensor_xy[2 * i + 1];
#else
            double dx = L->sensor_xy[2 * i] - *cx, dy = L->sensor_xy[2 * i + 1] - *cy;
#endif
            if (sqrt(dx * dx + dy * dy) > V->max_distance) a = 0;
        }
        act[i] = a;
        if (a) S += s[i];
    }
    *S_out = S;
    if (!(S > 0.0)) return OR_EVT_ZERO_SIGNAL;
    if (!or_variant_valid(L, act, *cx, *cy, *cz)) return OR_EVT_OUT_OF_DOMAIN;
    return OR_EVT_OK;
}

/* The match at a node, larger is better.  Maximum likelihood: F = sum_A s
 * ln eta - S ln H (the profiled objective over the sensors A in the match).
 * Least squares (reading: Poisson variances as weights): minus Pearson's
 * sum_A (s - E eta)^2 / (E eta) with E = S / H, the node's energy ratio. */
static double or_variant_score(const or_lrf *L, const or_variant *V, const int *act, const double *s, double S,
                               double x, double y, double z)
{
    if (!or_variant_valid(L, act, x, y, z)) return -INFINITY;
    double H = 0.0;
    for (int i = 0; i < L->n_sensors; ++i)
        if (act[i]) H += or_eta_floored(L, i, x, y, z);
    if (V->criterion == 0) {
        double acc = 0.0;
        for (int i = 0; i < L->n_sensors; ++i)
            if (act[i] && s[i] != 0.0) acc += s[i] * log(or_eta_floored(L, i, x, y, z));
        return acc - S * log(H);
    }
    double E = S / H, chi = 0.0;
    for (int i = 0; i < L->n_sensors; ++i) {
        if (!act[i]) continue;
        double mu = E * or_eta_floored(L, i, x, y, z), d = s[i] - mu;
#if OR_MUTANT == 16
        chi += d * d;
#else
        chi += d * d / mu;
#endif
    }
    return -chi;
}

/* E = S / H and the full Poisson log-likelihood over the sensors in the match. */
static void or_variant_energy_logl(const or_lrf *L, const int *act, const double *s, double S, double x, double y,
                                   double z, double *E_out, double *logL_out)
{
    double H = 0.0;
    for (int i = 0; i < L->n_sensors; ++i)
        if (act[i]) H += or_eta_floored(L, i, x, y, z);
    double E = S / H, ll = 0.0;
    for (int i = 0; i < L->n_sensors; ++i) {
        if (!act[i]) continue;
        double mu = E * or_eta_floored(L, i, x, y, z);
        ll += (s[i] != 0.0 ? s[i] * log(mu) : 0.0) - mu - lgamma(s[i] + 1.0);
    }
    *E_out = E;
    *logL_out = ll;
}

/* Magnitude of the terms summed at a node, for the tie tolerance of the
 * replay: sum_A |s ln p| (maximum likelihood, p = eta / H) or sum_A (s +
 * E eta) (least squares). */
static double or_variant_mag(const or_lrf *L, const or_variant *V, const int *act, const double *s, double S,
                             double x, double y, double z)
{
    double H = 0.0, mag = 0.0;
    for (int i = 0; i < L->n_sensors; ++i)
        if (act[i]) H += or_eta_floored(L, i, x, y, z);
    for (int i = 0; i < L->n_sensors; ++i) {
        if (!act[i]) continue;
        double eta = or_eta_floored(L, i, x, y, z);
        mag += V->criterion == 0 ? fabs(s[i] * log(eta / H)) : s[i] + S / H * eta;
    }
    return mag;
}

/* The contracting-grid search of or_cgs with the variant's criterion, start
 * and sensor selection; with trace_in (not NULL) the replay of another
 * implementation's path under the tie rule of or_cgs_replay (tau = tau_rel
 * times or_variant_mag at the grid's centre). */
static void or_cgs_variant_run(const or_lrf *L, const or_cgs_params *P, const or_variant *V, const double *gain,
                               long n_e, const double *sig, const int *trace_in, double tau_rel, double *xyz,
                               double *E, double *logL, int *status, int *trace, int *n_tie, int *n_bad)
{
    int nodes = P->n_xy * P->n_xy * P->n_z;
#pragma omp parallel for schedule(dynamic, 16)
    for (long e = 0; e < n_e; ++e) {
        const double *s = sig + e * L->n_sensors;
        int *act = (int *)malloc(sizeof(int) * (size_t)L->n_sensors);
        double cx, cy, cz, S;
        int st = or_variant_start(L, P, V, gain, s, NULL, &cx, &cy, &cz, &S, act);
        status[e] = st;
        if (n_tie) n_tie[e] = 0;
        if (n_bad) n_bad[e] = 0;
        if (st != OR_EVT_OK) {
            or_set_nan(&xyz[3 * e], &E[e], &logL[e]);
            if (trace) for (int it = 0; it < P->iters; ++it) trace[e * P->iters + it] = -1;
            free(act);
            continue;
        }
        double sxy = P->step_xy, sz = P->step_z;
        for (int it = 0; it < P->iters; ++it) {
            double best = -INFINITY;
            int best_k = -1;
            for (int k = 0; k < nodes; ++k) {
                double x, y, z;
                or_node(P, cx, cy, cz, sxy, sz, k, &x, &y, &z);
                double F = or_variant_score(L, V, act, s, S, x, y, z);
                if (F > best) { best = F; best_k = k; }
            }
            int g = best_k;
            if (trace_in) {
                g = trace_in[e * P->iters + it];
                if (g < 0 || g >= nodes) { n_bad[e]++; g = best_k; }
                if (g != best_k) {
                    double gx, gy, gz;
                    or_node(P, cx, cy, cz, sxy, sz, g, &gx, &gy, &gz);
                    double Fg = or_variant_score(L, V, act, s, S, gx, gy, gz);
                    double tau = tau_rel * or_variant_mag(L, V, act, s, S, cx, cy, cz);
                    if (isfinite(Fg) && Fg >= best - tau) n_tie[e]++;
                    else n_bad[e]++;
                }
            }
            double x, y, z;
            or_node(P, cx, cy, cz, sxy, sz, g, &x, &y, &z);
            cx = x; cy = y; cz = z;
            if (trace) trace[e * P->iters + it] = g;
            sxy *= P->shrink;
            sz *= P->shrink;
        }
        xyz[3 * e] = cx;
        xyz[3 * e + 1] = cy;
        xyz[3 * e + 2] = cz;
        or_variant_energy_logl(L, act, s, S, cx, cy, cz, &E[e], &logL[e]);
        free(act);
    }
}

void or_cgs_variant(const or_lrf *L, const or_cgs_params *P, const or_variant *V, const double *gain, long n_e,
                    const double *sig, double *xyz, double *E, double *logL, int *status, int *trace)
{
    or_cgs_variant_run(L, P, V, gain, n_e, sig, NULL, 0.0, xyz, E, logL, status, trace, NULL, NULL);
}

void or_cgs_variant_replay(const or_lrf *L, const or_cgs_params *P, const or_variant *V, const double *gain,
                           long n_e, const double *sig, const int *trace_in, double tau_rel, double *xyz, double *E,
                           double *logL, int *status, int *n_tie, int *n_bad)
{
    or_cgs_variant_run(L, P, V, gain, n_e, sig, trace_in, tau_rel, xyz, E, logL, status, NULL, n_tie, n_bad);
}

/* ------------------------------------------------------------------------ */
/* Continuous minimisation (Sec. 5.1.2.1: the match, maximum likelihood or   */
/* least squares, minimised over the two or three coordinates by a gradient  */
/* method from the centroid or strongest-sensor start; the paper uses        */
/* Minuit2's Migrad).  Here: damped Fisher scoring (Levenberg-Marquardt)     */
/* with the energy profiled out, E = S / H at every position.                */
/* ------------------------------------------------------------------------ */

/* The four non-zero cubic basis functions at x and their derivatives,
 * dB_{j,3}/dx = 3 [B_{j,2}(x) / (t_{j+3} - t_j) - B_{j+1,2}(x) / (t_{j+4} -
 * t_{j+1})] (the derivative of a B-spline as a difference of lower-degree
 * ones), from the Cox-de Boor triangle of degrees 0..3.  Returns the index
 * of the first one, or -1 outside [lo, hi]. */
int or_bspline_dbasis4(int n_int, double lo, double hi, double x, double B[4], double dB[4])
{
    int m = or_span(n_int, lo, hi, x);
    if (m < 0) return -1;
    double N[4][4]; /* N[k][r] = B_{m-k+r, k}(x) */
    N[0][0] = 1.0;
    for (int k = 1; k <= 3; ++k) {
        for (int r = 0; r <= k; ++r) {
            int j = m - k + r;
            double v = 0.0;
            if (r >= 1)
                v += (x - or_knot(n_int, lo, hi, j)) / (or_knot(n_int, lo, hi, j + k) - or_knot(n_int, lo, hi, j)) *
                     N[k - 1][r - 1];
            if (r <= k - 1)
                v += (or_knot(n_int, lo, hi, j + k + 1) - x) /
                     (or_knot(n_int, lo, hi, j + k + 1) - or_knot(n_int, lo, hi, j + 1)) * N[k - 1][r];
            N[k][r] = v;
        }
    }
    for (int r = 0; r < 4; ++r) {
        int j = m - 3 + r;
        double a = r >= 1 ? N[2][r - 1] / (or_knot(n_int, lo, hi, j + 3) - or_knot(n_int, lo, hi, j)) : 0.0;
        double b = r <= 2 ? N[2][r] / (or_knot(n_int, lo, hi, j + 4) - or_knot(n_int, lo, hi, j + 1)) : 0.0;
        B[r] = N[3][r];
#if OR_MUTANT == 21
        dB[r] = 3.0 * (a + b);
#else
        dB[r] = 3.0 * (a - b);
#endif
    }
    return m - 3;
}

/* or_spline2 with its partial derivatives along u and v. */
static double or_spline2_grad(int n0, double lo0, double hi0, int n1, double lo1, double hi1, const double *c,
                              double u, double v, int *ok, double *du, double *dv)
{
    double B0[4], B1[4], D0[4], D1[4];
    int j0 = or_bspline_dbasis4(n0, lo0, hi0, u, B0, D0);
    int j1 = or_bspline_dbasis4(n1, lo1, hi1, v, B1, D1);
    *ok = j0 >= 0 && j1 >= 0;
    *du = *dv = 0.0;
    if (!*ok) return 0.0;
    double f = 0.0;
    for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a) {
            double cc = c[(size_t)(j1 + b) * (n0 + 3) + (size_t)(j0 + a)];
            f += cc * B0[a] * B1[b];
            *du += cc * D0[a] * B1[b];
            *dv += cc * B0[a] * D1[b];
        }
    return f;
}

/* An axial part's derivative along x and y: df/dr times (dx, dy) / r
 * (taken as 0 at r = 0, where the direction is undefined). */
static void or_axial_dir(double dfdr, double dx, double dy, double r, double *gx, double *gy)
{
    *gx = r > 0.0 ? dfdr * dx / r : 0.0;
    *gy = r > 0.0 ? dfdr * dy / r : 0.0;
}

/* eta_i at (x, y, z) as or_lrf_eta, and its gradient g = (d/dx, d/dy,
 * d/dz) (d/dz = 0 for 2D LRFs). */
static double or_lrf_eta_grad(const or_lrf *L, int i, double x, double y, double z, int *ok, double g[3])
{
    int nc = or_n_coef(L);
    double dx = x - L->sensor_xy[2 * i], dy = y - L->sensor_xy[2 * i + 1];
    double r = sqrt(dx * dx + dy * dy);
    g[0] = g[1] = g[2] = 0.0;
    *ok = 1;
    if (L->type == OR_RADIAL || L->type == OR_COMPOSITE) {
        const double *c = L->coef + (size_t)(L->type == OR_RADIAL ? or_set_of(L, i) : i) * nc;
        int n = L->type == OR_RADIAL ? L->n_int[0] : L->n_int_r;
        double lo = L->type == OR_RADIAL ? L->lo[0] : 0.0, hi = L->type == OR_RADIAL ? L->hi[0] : L->hi_r;
        double B[4], D[4];
        int j0 = or_bspline_dbasis4(n, lo, hi, r, B, D);
        if (j0 < 0) { *ok = 0; return 0.0; }
        double f = 0.0, fr = 0.0;
        for (int a = 0; a < 4; ++a) {
            f += c[j0 + a] * B[a];
            fr += c[j0 + a] * D[a];
        }
        if (L->type == OR_RADIAL) {
            double gn = L->gain ? L->gain[i] : 1.0;
            or_axial_dir(gn * fr, dx, dy, r, &g[0], &g[1]);
            return gn * f;
        }
        int okxy;
        double fx, fy;
        double fxy = or_spline2_grad(L->n_int[0], L->lo[0], L->hi[0], L->n_int[1], L->lo[1], L->hi[1],
                                     c + L->n_int_r + 3, x, y, &okxy, &fx, &fy);
        if (!okxy) { *ok = 0; g[0] = g[1] = 0.0; return 0.0; }
        or_axial_dir(fr, dx, dy, r, &g[0], &g[1]);
        g[0] += fx;
        g[1] += fy;
        return f + fxy;
    }
    if (L->type == OR_AXIAL_Z) {
        double fr, fz;
        double f = or_spline2_grad(L->n_int[0], L->lo[0], L->hi[0], L->n_int[1], L->lo[1], L->hi[1],
                                   L->coef + (size_t)i * nc, r, z, ok, &fr, &fz);
        if (!*ok) return 0.0;
        or_axial_dir(fr, dx, dy, r, &g[0], &g[1]);
        g[2] = fz;
        return f;
    }
    if (L->type == OR_SLICED) {
        if (!(z >= L->lo[2] && z <= L->hi[2])) { *ok = 0; return 0.0; }
        int m = L->n_planes, ncxy = nc / m;
        double dz = (L->hi[2] - L->lo[2]) / (double)(m - 1), u = (z - L->lo[2]) / dz;
        int j = (int)floor(u);
        if (j > m - 2) j = m - 2;
        if (j < 0) j = 0;
        double w = u - (double)j;
        const double *c = L->coef + (size_t)i * nc;
        int ok0, ok1;
        double f0x, f0y, f1x, f1y;
        double f0 = or_spline2_grad(L->n_int[0], L->lo[0], L->hi[0], L->n_int[1], L->lo[1], L->hi[1],
                                    c + (size_t)j * ncxy, x, y, &ok0, &f0x, &f0y);
        double f1 = or_spline2_grad(L->n_int[0], L->lo[0], L->hi[0], L->n_int[1], L->lo[1], L->hi[1],
                                    c + (size_t)(j + 1) * ncxy, x, y, &ok1, &f1x, &f1y);
        if (!ok0 || !ok1) { *ok = 0; return 0.0; }
        g[0] = (1.0 - w) * f0x + w * f1x;
        g[1] = (1.0 - w) * f0y + w * f1y;
        g[2] = (f1 - f0) / dz;
        return (1.0 - w) * f0 + w * f1;
    }
    const double *c = L->coef + (size_t)i * nc;
    double gs = 1.0, M[4] = {1.0, 0.0, 0.0, 1.0};
    if (L->type == OR_XY && L->group) {
        c = L->coef + (size_t)L->group[i] * nc;
        or_sym_point(L, i, &x, &y);
        or_sym_op(L->op[i], M);
        gs = L->gain ? L->gain[i] : 1.0;
    }
    double Bx[4], By[4], Bz[4] = {1.0, 0.0, 0.0, 0.0}, Dx[4], Dy[4], Dz[4] = {0.0, 0.0, 0.0, 0.0};
    int jx = or_bspline_dbasis4(L->n_int[0], L->lo[0], L->hi[0], x, Bx, Dx);
    int jy = or_bspline_dbasis4(L->n_int[1], L->lo[1], L->hi[1], y, By, Dy);
    int jz = 0, nz = 1;
    if (L->type == OR_XYZ) {
        jz = or_bspline_dbasis4(L->n_int[2], L->lo[2], L->hi[2], z, Bz, Dz);
        nz = 4;
    }
    if (jx < 0 || jy < 0 || jz < 0) { *ok = 0; return 0.0; }
    int sx = L->n_int[0] + 3, sy = L->n_int[1] + 3;
    double f = 0.0;
    for (int cz = 0; cz < nz; ++cz)
        for (int b = 0; b < 4; ++b)
            for (int a = 0; a < 4; ++a) {
                double cc = c[((size_t)(jz + cz) * sy + (size_t)(jy + b)) * sx + (size_t)(jx + a)];
                f += cc * Bx[a] * By[b] * Bz[cz];
                g[0] += cc * Dx[a] * By[b] * Bz[cz];
                g[1] += cc * Bx[a] * Dy[b] * Bz[cz];
                g[2] += cc * Bx[a] * By[b] * Dz[cz];
            }
    /* the gradient of F(M^T (p - c) + c) is M grad F */
    double gx = M[0] * g[0] + M[1] * g[1], gy = M[2] * g[0] + M[3] * g[1];
    g[0] = gs * gx;
    g[1] = gs * gy;
    g[2] *= gs;
    return gs * f;
}

/* Gradients of every sensor's LRF at the points: out[(p n_s + i) 3 + k]; NaN
 * where the LRF is undefined. */
void or_lrf_grad(const or_lrf *L, long n_pts, const double *pts, int dim, double *out)
{
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n_pts; ++p) {
        double x = pts[p * dim], y = dim > 1 ? pts[p * dim + 1] : 0.0;
        double z = dim > 2 ? pts[p * dim + 2] : 0.0;
        for (int i = 0; i < L->n_sensors; ++i) {
            int ok;
            double g[3];
            or_lrf_eta_grad(L, i, x, y, z, &ok, g);
            for (int k = 0; k < 3; ++k) out[(p * L->n_sensors + i) * 3 + k] = ok ? g[k] : NAN;
        }
    }
}

typedef struct {
    int max_iter;   /* trial steps (accepted or not) */
    double tol;     /* converged when an accepted step is shorter than tol (mm) */
    double lambda0; /* initial damping */
    int fit_z;      /* 3D LRFs: z is a free coordinate too */
} or_min_params;

#define OR_LAMBDA_MIN 1e-12
#define OR_LAMBDA_MAX 1e8

/* The match's value C (larger is better: F for maximum likelihood, minus
 * Pearson's chi^2 for least squares) at p over the sensors in act, with the
 * energy profiled (E = S / H, eta floored as everywhere).  With g and J (not
 * NULL) also, over the first d coordinates:
 *   J = E sum_A (grad eta_i - eta_i grad H / H)(...)^T / eta_i, the Fisher
 *       information of the position with E profiled out (grad mu_i = E (grad
 *       eta_i - eta_i grad H / H) for mu_i = E eta_i);
 *   g = grad F = sum_A (s_i - E eta_i) grad eta_i / eta_i (maximum
 *       likelihood), or -grad chi^2 / 2 = -(1/2) sum_A (1 - s_i^2 / mu_i^2)
 *       grad mu_i (least squares, d chi^2 / d mu_i = 1 - s_i^2 / mu_i^2),
 *   so that the scoring step solves J delta = g in both cases (chi^2's
 *   Gauss-Newton curvature is 2 J). */
static double or_min_value(const or_lrf *L, int crit, const int *act, const double *s, double S, const double p[3],
                           int d, double g[3], double J[9])
{
    int n = L->n_sensors;
    double H = 0.0, dH[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n; ++i) {
        if (!act[i]) continue;
        int ok;
        double gi[3];
        double eta = or_lrf_eta_grad(L, i, p[0], p[1], p[2], &ok, gi);
        if (!(eta > OR_ETA_FLOOR)) { eta = OR_ETA_FLOOR; gi[0] = gi[1] = gi[2] = 0.0; }
        H += eta;
        for (int k = 0; k < 3; ++k) dH[k] += gi[k];
    }
    double E = S / H, C = 0.0;
    if (g) {
        for (int k = 0; k < 3; ++k) g[k] = 0.0;
        for (int k = 0; k < 9; ++k) J[k] = 0.0;
    }
    for (int i = 0; i < n; ++i) {
        if (!act[i]) continue;
        int ok;
        double gi[3];
        double eta = or_lrf_eta_grad(L, i, p[0], p[1], p[2], &ok, gi);
        if (!(eta > OR_ETA_FLOOR)) { eta = OR_ETA_FLOOR; gi[0] = gi[1] = gi[2] = 0.0; }
        double mu = E * eta;
        if (crit == 0) C += s[i] != 0.0 ? s[i] * log(eta) : 0.0;
        else C -= (s[i] - mu) * (s[i] - mu) / mu;
        if (!g) continue;
        double dmu[3];
        for (int k = 0; k < 3; ++k) dmu[k] = E * (gi[k] - eta * dH[k] / H);
        for (int k = 0; k < d; ++k) {
#if OR_MUTANT == 22
            if (crit == 0) g[k] += s[i] * gi[k] / eta;
#else
            if (crit == 0) g[k] += (s[i] - mu) * gi[k] / eta;
#endif
#if OR_MUTANT == 23
            else g[k] -= 0.5 * (1.0 + s[i] * s[i] / (mu * mu)) * dmu[k];
#else
            else g[k] -= 0.5 * (1.0 - s[i] * s[i] / (mu * mu)) * dmu[k];
#endif
            for (int l = 0; l < d; ++l) J[k * 3 + l] += dmu[k] * dmu[l] / mu;
        }
    }
    if (crit == 0) C -= S * log(H);
    return C;
}

/* Solve (J + lambda D) delta = g for d = 2 or 3, D = diag(J) with each entry
 * floored at 1e-12 of the largest; Cramer's rule.  Coordinates in the mask
 * `fixed` (bit k) are held: their rows and columns become those of the
 * identity and their right-hand side 0, so delta_k = 0 and the others solve
 * the reduced system.  Returns 0 when the system is singular. */
static int or_min_solve(const double J[9], double lambda, const double g_in[3], int d, int fixed, double delta[3])
{
    double dmax = 0.0;
    for (int k = 0; k < d; ++k) dmax = J[k * 4] > dmax ? J[k * 4] : dmax;
    if (!(dmax > 0.0)) return 0;
    double A[9], g[3] = {g_in[0], g_in[1], g_in[2]};
    for (int k = 0; k < 9; ++k) A[k] = J[k];
    for (int k = 0; k < d; ++k) {
        double dk = J[k * 4] > 1e-12 * dmax ? J[k * 4] : 1e-12 * dmax;
        A[k * 4] += lambda * dk;
    }
    for (int k = 0; k < d; ++k) {
        if (!(fixed >> k & 1)) continue;
        for (int l = 0; l < 3; ++l) A[k * 3 + l] = A[l * 3 + k] = 0.0;
        A[k * 4] = 1.0;
        g[k] = 0.0;
    }
    delta[0] = delta[1] = delta[2] = 0.0;
    if (d == 2) {
        double det = A[0] * A[4] - A[1] * A[3];
        if (!(fabs(det) > 0.0)) return 0;
        delta[0] = (g[0] * A[4] - A[1] * g[1]) / det;
        delta[1] = (A[0] * g[1] - g[0] * A[3]) / det;
        return 1;
    }
    double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                 A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (!(fabs(det) > 0.0)) return 0;
    for (int c = 0; c < 3; ++c) {
        double M[9];
        for (int k = 0; k < 9; ++k) M[k] = A[k];
        for (int r = 0; r < 3; ++r) M[r * 3 + c] = g[r];
        delta[c] = (M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                    M[2] * (M[3] * M[7] - M[4] * M[6])) / det;
    }
    return 1;
}

/* The box bounds of coordinate k (x and y: the XY box of XY, XYZ,
 * composite and sliced LRFs; z: the z range of XYZ, sliced and axial+z
 * ones); 0 when the coordinate has none. */
static int or_min_bounds(const or_lrf *L, int k, double *lo, double *hi)
{
    if (k < 2) {
        if (!or_has_box(L->type)) return 0;
        *lo = L->lo[k];
        *hi = L->hi[k];
        return 1;
    }
    if (!or_is_3d(L->type)) return 0;
    int kz = L->type == OR_AXIAL_Z ? 1 : 2;
    *lo = L->lo[kz];
    *hi = L->hi[kz];
    return 1;
}

/* A trial position moved onto the domain's box. */
static void or_min_clamp(const or_lrf *L, double q[3])
{
    for (int k = 0; k < 3; ++k) {
        double lo, hi;
        if (or_min_bounds(L, k, &lo, &hi)) q[k] = q[k] < lo ? lo : (q[k] > hi ? hi : q[k]);
    }
}

/* The coordinates (bit k) that lie on a bound of the box while the step
 * delta points out of it: the active constraints, held in the next solve. */
static int or_min_active(const or_lrf *L, const double p[3], const double delta[3], int d)
{
    int fixed = 0;
    for (int k = 0; k < d; ++k) {
        double lo, hi;
        if (!or_min_bounds(L, k, &lo, &hi)) continue;
        if ((p[k] == lo && delta[k] < 0.0) || (p[k] == hi && delta[k] > 0.0)) fixed |= 1 << k;
    }
    return fixed;
}

/* The minimisation of one event from p (already inside the domain):
 *   each trial solves (J + lambda D) delta = g at p, again with the
 *   coordinates held that lie on a bound of the domain's box while delta
 *   points out of it (or_min_active; a projected step), and moves to q = p +
 *   delta moved onto the box (or_min_clamp).  q is accepted when
 *   every LRF in the match is defined there and the match improves: when
 *   |C(q) - C(p)| > tau = 2^-18 S (beyond a bound on the single-precision
 *   rounding of the difference, used by both implementations) by its sign,
 *   else by the sign of (g(p) + g(q)) . (q - p), the trapezoid rule for the
 *   change along the step (exact for a quadratic match, and computed from
 *   gradients, which keep their precision near the optimum).  An accepted
 *   trial sets lambda = max(lambda / 10, 1e-12), or, when the slope along
 *   the step changed sign (a0 = g(p) . (q - p) > 0 > a1 = g(q) . (q - p):
 *   the step overshot the optimum along its line, which a quadratic places
 *   at t* = a0 / (a0 - a1) of it), the larger 1 / t* - 1 (the damping that
 *   shortens a step by t* when D = J), and ends the minimisation when
 *   |q - p| < tol; a rejected trial multiplies lambda by 10 and ends it
 *   above 1e8.  At most max_iter trials.
 * Returns the trials used, negative when max_iter ran out first. */
static int or_min_run(const or_lrf *L, int crit, const or_min_params *M, const int *act, const double *s, double S,
                      double p[3])
{
    int d = or_is_3d(L->type) && M->fit_z ? 3 : 2;
    double tau = ldexp(S, -18);
    double lambda = M->lambda0, g[3], J[9];
    double C = or_min_value(L, crit, act, s, S, p, d, g, J);
    for (int it = 1; it <= M->max_iter; ++it) {
        double delta[3] = {0.0, 0.0, 0.0};
        int okd = or_min_solve(J, lambda, g, d, 0, delta);
        int fixed = okd ? or_min_active(L, p, delta, d) : 0;
        if (fixed) okd = or_min_solve(J, lambda, g, d, fixed, delta);
        double q[3] = {p[0] + delta[0], p[1] + delta[1], p[2] + delta[2]};
        or_min_clamp(L, q);
        int acc = okd && isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) && or_valid_act(L, act, q[0], q[1], q[2]);
        double gq[3], Jq[9], Cq = 0.0;
        if (acc) {
            Cq = or_min_value(L, crit, act, s, S, q, d, gq, Jq);
            double dC = Cq - C;
            if (fabs(dC) > tau) {
                acc = dC > 0.0;
            } else {
                double t = 0.0;
                for (int k = 0; k < 3; ++k) t += (g[k] + gq[k]) * (q[k] - p[k]);
#if OR_MUTANT == 24
                acc = 1;
#else
                acc = t >= 0.0;
#endif
            }
        }
        if (acc) {
            double step = sqrt((q[0] - p[0]) * (q[0] - p[0]) + (q[1] - p[1]) * (q[1] - p[1]) +
                               (q[2] - p[2]) * (q[2] - p[2]));
            double a0 = 0.0, a1 = 0.0, next = lambda * 0.1 > OR_LAMBDA_MIN ? lambda * 0.1 : OR_LAMBDA_MIN;
            for (int k = 0; k < 3; ++k) {
                a0 += g[k] * (q[k] - p[k]);
                a1 += gq[k] * (q[k] - p[k]);
            }
            if (a0 > 0.0 && a1 < 0.0) {
                double ts = a0 / (a0 - a1);
                if (1.0 / ts - 1.0 > next) next = 1.0 / ts - 1.0;
            }
            for (int k = 0; k < 3; ++k) {
                p[k] = q[k];
                g[k] = gq[k];
            }
            for (int k = 0; k < 9; ++k) J[k] = Jq[k];
            C = Cq;
            lambda = next;
            if (step < M->tol) return it;
        } else {
            lambda *= 10.0;
            if (lambda > OR_LAMBDA_MAX) return it;
        }
    }
    return -M->max_iter;
}

/* Minimisation of n_e events: the start and the sensors in the match as
 * for the search variants (start_xyz, when not NULL, gives the start of
 * every event instead), then or_min_run; E = S / H and the full Poisson
 * logL over the match at the result; n_iter: the trials of or_min_run. */
void or_minimize(const or_lrf *L, const or_cgs_params *P, const or_variant *V, const or_min_params *M,
                 const double *gain, long n_e, const double *sig, const double *start_xyz, double *xyz, double *E,
                 double *logL, int *status, int *n_iter)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (long e = 0; e < n_e; ++e) {
        const double *s = sig + e * L->n_sensors;
        int *act = (int *)malloc(sizeof(int) * (size_t)L->n_sensors);
        double p[3], S;
        int st = or_variant_start(L, P, V, gain, s, start_xyz ? start_xyz + 3 * e : NULL, &p[0], &p[1], &p[2], &S,
                                  act);
        status[e] = st;
        n_iter[e] = 0;
        if (st != OR_EVT_OK) {
            or_set_nan(&xyz[3 * e], &E[e], &logL[e]);
            free(act);
            continue;
        }
        n_iter[e] = or_min_run(L, V->criterion, M, act, s, S, p);
        xyz[3 * e] = p[0];
        xyz[3 * e + 1] = p[1];
        xyz[3 * e + 2] = p[2];
        or_variant_energy_logl(L, act, s, S, p[0], p[1], p[2], &E[e], &logL[e]);
        free(act);
    }
}

/* Exhaustive search: the best node of a regular nx x ny grid over
 * [x_lo, x_hi] x [y_lo, y_hi] at height z (ties to the lowest index). */
void or_brute_force(const or_lrf *L, long n_e, const double *sig, double x_lo, double x_hi,
                    int nx, double y_lo, double y_hi, int ny, double z, double *out_xy,
                    double *out_F)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (long e = 0; e < n_e; ++e) {
        const double *s = sig + e * L->n_sensors;
        double S = 0.0;
        for (int i = 0; i < L->n_sensors; ++i) S += s[i];
        double best = -INFINITY, bx = NAN, by = NAN;
        for (int k = 0; k < ny; ++k)
            for (int j = 0; j < nx; ++j) {
                double x = x_lo + (x_hi - x_lo) * (double)j / (double)(nx - 1);
                double y = y_lo + (y_hi - y_lo) * (double)k / (double)(ny - 1);
                double F = or_objective(L, s, S, x, y, z);
                if (F > best) { best = F; bx = x; by = y; }
            }
        out_xy[2 * e] = bx;
        out_xy[2 * e + 1] = by;
        out_F[e] = best;
    }
}

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Run the following calls on n threads (timing the oracle single-threaded
 * and on all cores); no effect without OpenMP. */
void or_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Learned proposal: multilayer perceptron (the ANN role of Sec. 5.1.3)      */
/* ------------------------------------------------------------------------ */
/* u = s / sum(s); z1 = W1 u + b1; h1 = GELU(z1); z2 = W2 h1 + b2;
 * h2 = GELU(z2); o = W3 h2 + b3.  GELU(x) = x Phi(x) = 0.5 x (1 + erf(x/sqrt 2)).
 * Weights are row-major [out][in].  Training loss: mean squared error over
 * the batch and the n_out outputs. */

typedef struct {
    int n_in, n_hid, n_out;
    const double *W1, *b1, *W2, *b2, *W3, *b3;
} or_mlp;

static double or_gelu(double x)
{
#if OR_MUTANT == 10
    return 0.5 * x * (1.0 + erf(x));
#else
    return 0.5 * x * (1.0 + erf(x / sqrt(2.0)));
#endif
}

/* d GELU / dx = Phi(x) + x phi(x) */
static double or_gelu_grad(double x)
{
    const double inv_sqrt_2pi = 0.3989422804014327;
    return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * inv_sqrt_2pi * exp(-0.5 * x * x);
}

double or_gelu_value(double x) { return or_gelu(x); }

/* Forward pass of one event (input already normalised); act (nullable)
 * receives z1, h1, z2, h2 (4 * n_hid values). */
static void or_mlp_forward1(const or_mlp *M, const double *u, double *o, double *act)
{
    int H = M->n_hid;
    double *z1 = (double *)malloc(sizeof(double) * 4 * H);
    double *h1 = z1 + H, *z2 = z1 + 2 * H, *h2 = z1 + 3 * H;
    for (int j = 0; j < H; ++j) {
        double v = M->b1[j];
        for (int i = 0; i < M->n_in; ++i) v += M->W1[(size_t)j * M->n_in + i] * u[i];
        z1[j] = v;
        h1[j] = or_gelu(v);
    }
    for (int j = 0; j < H; ++j) {
        double v = M->b2[j];
        for (int i = 0; i < H; ++i) v += M->W2[(size_t)j * H + i] * h1[i];
        z2[j] = v;
        h2[j] = or_gelu(v);
    }
    for (int k = 0; k < M->n_out; ++k) {
        double v = M->b3[k];
        for (int i = 0; i < H; ++i) v += M->W3[(size_t)k * H + i] * h2[i];
        o[k] = v;
    }
    if (act) memcpy(act, z1, sizeof(double) * 4 * H);
    free(z1);
}

/* u = s / sum(s) for every event, then the forward pass: out[n][n_out]. */
void or_mlp_forward(const or_mlp *M, long n, const double *sig, double *out)
{
#pragma omp parallel for schedule(static)
    for (long e = 0; e < n; ++e) {
        double *u = (double *)malloc(sizeof(double) * M->n_in);
        double S = 0.0;
        for (int i = 0; i < M->n_in; ++i) S += sig[e * M->n_in + i];
        for (int i = 0; i < M->n_in; ++i) u[i] = S > 0.0 ? sig[e * M->n_in + i] / S : 0.0;
        or_mlp_forward1(M, u, out + e * M->n_out, NULL);
        free(u);
    }
}

/* Mean squared error L = 1/(n n_out) sum (o - t)^2 over a batch of signals,
 * and its gradient by back-propagation, accumulated in the order of the
 * parameters: gW1, gb1, gW2, gb2, gW3, gb3 (same shapes).  Returns L. */
double or_mlp_loss_grad(const or_mlp *M, long n, const double *sig, const double *target, double *gW1,
                        double *gb1, double *gW2, double *gb2, double *gW3, double *gb3)
{
    int H = M->n_hid, I = M->n_in, O = M->n_out;
    memset(gW1, 0, sizeof(double) * H * I);
    memset(gb1, 0, sizeof(double) * H);
    memset(gW2, 0, sizeof(double) * H * H);
    memset(gb2, 0, sizeof(double) * H);
    memset(gW3, 0, sizeof(double) * O * H);
    memset(gb3, 0, sizeof(double) * O);
    double *u = (double *)malloc(sizeof(double) * I);
    double *act = (double *)malloc(sizeof(double) * 4 * H);
    double *o = (double *)malloc(sizeof(double) * O);
    double *dz1 = (double *)malloc(sizeof(double) * H), *dz2 = (double *)malloc(sizeof(double) * H);
    double loss = 0.0, scale = 1.0 / ((double)n * O);
    for (long e = 0; e < n; ++e) {
        double S = 0.0;
        for (int i = 0; i < I; ++i) S += sig[e * I + i];
        for (int i = 0; i < I; ++i) u[i] = S > 0.0 ? sig[e * I + i] / S : 0.0;
        or_mlp_forward1(M, u, o, act);
        double *z1 = act, *h1 = act + H, *z2 = act + 2 * H, *h2 = act + 3 * H;
        /* dL/do = 2 (o - t) / (n O) */
        double dout[16];
        for (int k = 0; k < O; ++k) {
            double d = o[k] - target[e * O + k];
            loss += d * d * scale;
#if OR_MUTANT == 11
            dout[k] = d * scale;
#else
            dout[k] = 2.0 * d * scale;
#endif
        }
        for (int k = 0; k < O; ++k) {
            gb3[k] += dout[k];
            for (int i = 0; i < H; ++i) gW3[(size_t)k * H + i] += dout[k] * h2[i];
        }
        for (int i = 0; i < H; ++i) {
            double v = 0.0;
            for (int k = 0; k < O; ++k) v += M->W3[(size_t)k * H + i] * dout[k];
            dz2[i] = v * or_gelu_grad(z2[i]);
        }
        for (int j = 0; j < H; ++j) {
            gb2[j] += dz2[j];
            for (int i = 0; i < H; ++i) gW2[(size_t)j * H + i] += dz2[j] * h1[i];
        }
        for (int i = 0; i < H; ++i) {
            double v = 0.0;
            for (int j = 0; j < H; ++j) v += M->W2[(size_t)j * H + i] * dz2[j];
            dz1[i] = v * or_gelu_grad(z1[i]);
        }
        for (int j = 0; j < H; ++j) {
            gb1[j] += dz1[j];
            for (int i = 0; i < I; ++i) gW1[(size_t)j * I + i] += dz1[j] * u[i];
        }
    }
    free(u);
    free(act);
    free(o);
    free(dz1);
    free(dz2);
    return loss;
}

/* One Adam step (Kingma & Ba, Algorithm 1) on n parameters, step t >= 1:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr mhat / (sqrt(vhat) + eps)
 * with mhat = m / (1 - b1^t), vhat = v / (1 - b2^t). */
void or_adam_step(long n, double *p, const double *g, double *m, double *v, int t, double lr, double b1, double b2,
                  double eps)
{
    double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (long i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* Poisson deviance D = 2 sum_i [ s_i ln(s_i / mu_i) - (s_i - mu_i) ] at the
 * given positions (s_i = 0 terms: 2 mu_i) -- twice the gap to the saturated
 * likelihood, used to flag events for the fallback search. */
void or_deviance_at(const or_lrf *L, long n_e, const double *sig, const double *xyz, double *D)
{
#pragma omp parallel for schedule(static)
    for (long e = 0; e < n_e; ++e) {
        const double *s = sig + e * L->n_sensors;
        double E, ll;
        or_energy_logl(L, s, xyz[3 * e], xyz[3 * e + 1], xyz[3 * e + 2], &E, &ll);
        double sat = 0.0;
        for (int i = 0; i < L->n_sensors; ++i)
            if (s[i] > 0.0) sat += s[i] * log(s[i]) - s[i] - lgamma(s[i] + 1.0);
        D[e] = 2.0 * (sat - ll);
    }
}

/* ------------------------------------------------------------------------ */
/* Event simulation from an LRF set (Poisson photo-electron counts,          */
/* Sec. 4.2.5 signals; the photon transport of Sec. 4.2.3 is replaced by     */
/* the LRF mean response)                                                    */
/* ------------------------------------------------------------------------ */
#include <stdint.h>

/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror and Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two
 * 32x32->64-bit multiplications with the published multipliers and Weyl key
 * increments. */
static void or_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

void or_philox_block(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t *out)
{
    uint32_t ctr[4] = {c0, c1, c2, c3}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox(ctr, key, out);
}

/* uniform in (0, 1) from the top 24 bits */
static double or_u01(uint32_t x) { return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0); }

typedef struct {
    uint32_t key[2], ctr[4], buf[4];
    int pos;
} or_stream;

static void or_stream_init(or_stream *s, uint64_t seed, long e, uint32_t lane)
{
    s->key[0] = (uint32_t)seed;
    s->key[1] = (uint32_t)(seed >> 32);
    s->ctr[0] = (uint32_t)e;
    s->ctr[1] = (uint32_t)((uint64_t)e >> 32);
    s->ctr[2] = lane;
    s->ctr[3] = 0;
    s->pos = 4;
}

static double or_next_u(or_stream *s)
{
    if (s->pos == 4) {
        or_philox(s->ctr, s->key, s->buf);
        s->ctr[3]++;
        s->pos = 0;
    }
    return or_u01(s->buf[s->pos++]);
}

/* ------------------------------------------------------------------------ */
/* Optical photon transport in a stack of horizontal slabs (Sec. 4.2.3     */
/* photon tracing, 4.2.4 detection, 4.2.6 pre-rejection; Sec. 3.5 custom    */
/* interface properties).  Photons are emitted isotropically from a point; */
/* each tracing cycle finds the next interface, draws absorption and        */
/* Rayleigh ranges, and at an interface applies the custom properties, then */
/* Fresnel reflection (unpolarised) or Snell refraction.  Sensors are       */
/* square windows on the bottom boundary.                                   */
/* ------------------------------------------------------------------------ */

#define OR_OPT_MAX_LAYERS 8
#define OR_PI 3.14159265358979323846
#define OR_OPT_TAG 0x0F7105u

typedef struct {
    int n_layers;
    double z[OR_OPT_MAX_LAYERS + 1];    /* boundaries, increasing */
    double n[OR_OPT_MAX_LAYERS];        /* refractive index per layer */
    double abs_len[OR_OPT_MAX_LAYERS];  /* absorption length, 0 = none */
    double ray_len[OR_OPT_MAX_LAYERS];  /* Rayleigh mean free path, 0 = none */
    double n_below, n_above;            /* media outside the stack */
    double half_x, half_y;              /* lateral extent of the stack */
    double p_abs[OR_OPT_MAX_LAYERS + 1], p_spec[OR_OPT_MAX_LAYERS + 1], p_diff[OR_OPT_MAX_LAYERS + 1];
    int n_sensors;
    const double *sensor_xy;            /* [n_sensors][2] window centres on z[0] */
    double sensor_size;                 /* side of the square windows */
    double n_sensor;                    /* window index */
    const double *qe;                   /* [n_sensors] */
    int n_ang;                          /* angular response samples (0: none) */
    const double *ang;                  /* [n_ang] at theta_j = j (pi/2) / (n_ang - 1) */
    int max_cycles;
    int pre_reject;
} or_optics;

/* outcome codes of a photon (>= 0: the detecting sensor) */
#define OR_PH_ABSORBED -1
#define OR_PH_ESCAPED -2
#define OR_PH_MAX_CYCLES -3
#define OR_PH_UNDETECTED -4 /* entered a sensor, failed the detection test */
#define OR_PH_REJECTED -5   /* discarded before tracing (pre-rejection) */

/* Fresnel reflection coefficient for unpolarised light, the mean of the s
 * and p coefficients, from medium n1 into n2 at incidence cosine ci; 1
 * beyond the critical angle. */
double or_fresnel(double n1, double n2, double ci)
{
    double si2 = 1.0 - ci * ci;
    double st2 = (n1 / n2) * (n1 / n2) * si2;
    if (st2 >= 1.0) return 1.0;
    double ct = sqrt(1.0 - st2);
#if OR_MUTANT == 25
    double rs = (n1 * ci - n2 * ct) / (n1 * ct + n2 * ci);
#else
    double rs = (n1 * ci - n2 * ct) / (n1 * ci + n2 * ct);
#endif
    double rp = (n1 * ct - n2 * ci) / (n1 * ct + n2 * ci);
    return 0.5 * (rs * rs + rp * rp);
}

/* cos(theta) drawn from the Rayleigh phase function, density (3/8)(1 +
 * mu^2) on [-1, 1]: the CDF (mu^3 + 3 mu + 4) / 8 = u inverted by Cardano's
 * formula for the depressed cubic mu^3 + 3 mu + (4 - 8u) = 0. */
double or_rayleigh_mu(double u)
{
    double q = 4.0 * u - 2.0, r = sqrt(q * q + 1.0);
    return cbrt(q + r) + cbrt(q - r);
}

/* a unit direction at angle acos(mu) from d and azimuth phi about it */
static void or_turn(double d[3], double mu, double phi)
{
    double s = sqrt(fmax(0.0, 1.0 - mu * mu)), cp = cos(phi), sp = sin(phi);
    double nx, ny, nz;
    if (fabs(d[2]) > 0.99999) {
        double sg = d[2] > 0.0 ? 1.0 : -1.0;
        nx = s * cp;
        ny = s * sp;
        nz = sg * mu;
    } else {
        double a = sqrt(1.0 - d[2] * d[2]);
        nx = mu * d[0] + s * (d[0] * d[2] * cp - d[1] * sp) / a;
        ny = mu * d[1] + s * (d[1] * d[2] * cp + d[0] * sp) / a;
        nz = mu * d[2] - s * a * cp;
    }
    d[0] = nx;
    d[1] = ny;
    d[2] = nz;
}

/* or_turn on a copy of d (exported for the pins) */
void or_turn_dir(const double d_in[3], double mu, double phi, double out[3])
{
    for (int c = 0; c < 3; ++c) out[c] = d_in[c];
    or_turn(out, mu, phi);
}

/* relative angular response at incidence cosine ci (linear in the angle) */
static double or_ang_resp(const or_optics *O, double ci)
{
    if (O->n_ang < 2) return 1.0;
    double th = acos(fmin(1.0, fmax(0.0, ci))) / (0.5 * OR_PI) * (double)(O->n_ang - 1);
    int j = (int)floor(th);
    if (j >= O->n_ang - 1) return O->ang[O->n_ang - 1];
    double w = th - (double)j;
    return (1.0 - w) * O->ang[j] + w * O->ang[j + 1];
}

/* the sensor whose window contains (x, y) on the bottom boundary, or -1 */
static int or_sensor_at(const or_optics *O, double x, double y)
{
    double h = 0.5 * O->sensor_size;
    for (int i = 0; i < O->n_sensors; ++i) {
#if OR_MUTANT == 26
        if (fabs(x - O->sensor_xy[2 * i]) <= O->sensor_size && fabs(y - O->sensor_xy[2 * i + 1]) <= O->sensor_size)
#else
        if (fabs(x - O->sensor_xy[2 * i]) <= h && fabs(y - O->sensor_xy[2 * i + 1]) <= h)
#endif
            return i;
    }
    return -1;
}

/* the largest detection probability of any sensor (pre-rejection) */
static double or_pmax(const or_optics *O)
{
    double a = 0.0, q = 0.0;
    for (int i = 0; i < O->n_sensors; ++i) q = O->qe[i] > q ? O->qe[i] : q;
    if (O->n_ang < 2) a = 1.0;
    for (int j = 0; j < O->n_ang; ++j) a = O->ang[j] > a ? O->ang[j] : a;
    return q * a;
}

/* One photon of source src_index from (x, y, z), photon index ph. */
static int or_trace_photon(const or_optics *O, uint64_t seed, long src_index, long ph, double x, double y, double z)
{
    or_stream st;
    or_stream_init(&st, seed, (long)(((uint64_t)src_index << 32) | (uint64_t)ph), OR_OPT_TAG);
    double u_det = -1.0;
    if (O->pre_reject) {
        u_det = or_next_u(&st);
#if OR_MUTANT == 27
        if (u_det < or_pmax(O)) return OR_PH_REJECTED;
#else
        if (!(u_det < or_pmax(O))) return OR_PH_REJECTED;
#endif
    }
    /* layer of the source: z[k] <= z < z[k+1] (the top boundary belongs to the top layer) */
    int k = 0;
    while (k < O->n_layers - 1 && z >= O->z[k + 1]) ++k;
    double r[3] = {x, y, z}, d[3];
    {
        double mu = 2.0 * or_next_u(&st) - 1.0, phi = 2.0 * OR_PI * or_next_u(&st);
        double s = sqrt(fmax(0.0, 1.0 - mu * mu));
        d[0] = s * cos(phi);
        d[1] = s * sin(phi);
        d[2] = mu;
    }
    for (int cyc = 0; cyc < O->max_cycles; ++cyc) {
        /* distance to the next interface: the layer's boundaries, the lateral walls */
        double tz = INFINITY, tw = INFINITY;
        int b = -1;
        if (d[2] > 0.0) { tz = (O->z[k + 1] - r[2]) / d[2]; b = k + 1; }
        else if (d[2] < 0.0) { tz = (O->z[k] - r[2]) / d[2]; b = k; }
        if (d[0] != 0.0) tw = ((d[0] > 0.0 ? O->half_x : -O->half_x) - r[0]) / d[0];
        if (d[1] != 0.0) {
            double ty = ((d[1] > 0.0 ? O->half_y : -O->half_y) - r[1]) / d[1];
            tw = ty < tw ? ty : tw;
        }
        /* random ranges of absorption and Rayleigh scattering */
        double ua = or_next_u(&st), ur = or_next_u(&st);
#if OR_MUTANT == 28
        double sa = O->abs_len[k] > 0.0 ? O->abs_len[k] * ua : INFINITY;
#else
        double sa = O->abs_len[k] > 0.0 ? -O->abs_len[k] * log(ua) : INFINITY;
#endif
        double sr = O->ray_len[k] > 0.0 ? -O->ray_len[k] * log(ur) : INFINITY;
        double t = tz < tw ? tz : tw, s = sa < sr ? sa : sr;
        if (s < t) {
            for (int c = 0; c < 3; ++c) r[c] += s * d[c];
            if (sa <= sr) return OR_PH_ABSORBED;
            double mu = or_rayleigh_mu(or_next_u(&st)), phi = 2.0 * OR_PI * or_next_u(&st);
            or_turn(d, mu, phi);
            continue;
        }
        if (tw <= tz) return OR_PH_ESCAPED; /* through a lateral wall */
        for (int c = 0; c < 3; ++c) r[c] += tz * d[c];
        r[2] = O->z[b]; /* on the boundary */
        double ci = fabs(d[2]);
        int sens = b == 0 ? or_sensor_at(O, r[0], r[1]) : -1;
        if (sens >= 0) {
            /* into the sensor's window (Fresnel), then the detection test */
            if (or_next_u(&st) < or_fresnel(O->n[k], O->n_sensor, ci)) {
                d[2] = -d[2];
                continue;
            }
            double pd = O->qe[sens] * or_ang_resp(O, ci);
            if (u_det < 0.0) u_det = or_next_u(&st);
            return u_det < pd ? sens : OR_PH_UNDETECTED;
        }
        double pa = O->p_abs[b], ps = O->p_spec[b], pf = O->p_diff[b];
        if (pa + ps + pf > 0.0) {
            double u = or_next_u(&st);
            if (u < pa) return OR_PH_ABSORBED;
            if (u < pa + ps) {
                d[2] = -d[2];
                continue;
            }
            if (u < pa + ps + pf) {
                /* Lambertian: cosine-weighted about the normal into layer k */
                double mu = sqrt(or_next_u(&st)), phi = 2.0 * OR_PI * or_next_u(&st);
                double sn = sqrt(fmax(0.0, 1.0 - mu * mu));
                d[0] = sn * cos(phi);
                d[1] = sn * sin(phi);
                d[2] = b == k + 1 ? -mu : mu;
                continue;
            }
        }
        /* Fresnel reflection or Snell refraction into the next medium */
        double n1 = O->n[k];
        double n2 = b == k + 1 ? (b == O->n_layers ? O->n_above : O->n[k + 1]) : (b == 0 ? O->n_below : O->n[k - 1]);
        if (or_next_u(&st) < or_fresnel(n1, n2, ci)) {
            d[2] = -d[2];
            continue;
        }
        if (b == 0 || b == O->n_layers) return OR_PH_ESCAPED; /* out of the stack */
        double eta = n1 / n2, ct = sqrt(fmax(0.0, 1.0 - eta * eta * (1.0 - ci * ci)));
        d[0] *= eta;
        d[1] *= eta;
        d[2] = d[2] > 0.0 ? ct : -ct;
        k = b == k + 1 ? k + 1 : k - 1;
    }
    return OR_PH_MAX_CYCLES;
}

/* Photons of n_src point sources, n_ph each: detected counts per sensor
 * counts[src][sensor] and, when outcome is not NULL, every photon's
 * outcome[src][photon]. */
void or_trace_photons(const or_optics *O, long n_src, const double *src_xyz, long n_ph, uint64_t seed, int *counts,
                      int *outcome)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (long q = 0; q < n_src; ++q) {
        int *c = counts + q * O->n_sensors;
        for (int i = 0; i < O->n_sensors; ++i) c[i] = 0;
        for (long p = 0; p < n_ph; ++p) {
            int o = or_trace_photon(O, seed, q, p, src_xyz[3 * q], src_xyz[3 * q + 1], src_xyz[3 * q + 2]);
            if (o >= 0) c[o]++;
            if (outcome) outcome[q * n_ph + p] = o;
        }
    }
}

/* Poisson(lam): inversion of the CDF for lam < 10; Hormann's transformed
 * rejection with squeeze (PTRS, Insurance: Mathematics and Economics 12,
 * 1993) otherwise. */
static long or_poisson(double lam, or_stream *s)
{
    if (!(lam > 0.0)) return 0;
    if (lam < 10.0) {
        double u = or_next_u(s), p = exp(-lam), F = p;
        long k = 0;
        while (u > F && k < 1000) {
            ++k;
            p *= lam / (double)k;
            F += p;
        }
        return k;
    }
    double slam = sqrt(lam), loglam = log(lam);
    double b = 0.931 + 2.53 * slam, a = -0.059 + 0.02483 * b;
    double inv_alpha = 1.1239 + 1.1328 / (b - 3.4), vr = 0.9277 - 3.6224 / (b - 2.0);
    for (int it = 0; it < 1000; ++it) {
        double U = or_next_u(s) - 0.5, V = or_next_u(s);
        double us = 0.5 - fabs(U);
        long k = (long)floor((2.0 * a / us + b) * U + lam + 0.43);
        if (us >= 0.07 && V <= vr) return k;
        if (k < 0 || (us < 0.013 && V > us)) continue;
        if (log(V) + log(inv_alpha) - log(a / (us * us) + b) <= -lam + (double)k * loglam - lgamma((double)k + 1.0))
            return k;
    }
    return (long)lam;
}

typedef struct {
    int region;     /* 0 disk, 1 square */
    double extent;  /* radius or half-width */
    double cx, cy;
    double z_lo, z_hi;
    double e0, e_spread;
    double spe_sigma;
} or_sim_params;

/* Events first_event .. first_event+n-1: source position and energy from
 * stream (e, 0xFFFFFFFF), counts of sensor i from stream (e, i). */
void or_simulate(const or_lrf *L, const or_sim_params *P, uint64_t seed, long first_event, long n, double *sig,
                 double *truth)
{
#pragma omp parallel for schedule(static)
    for (long r = 0; r < n; ++r) {
        long e = first_event + r;
        uint32_t ev[4];
        or_philox_block(seed, (uint32_t)e, (uint32_t)((uint64_t)e >> 32), 0xFFFFFFFFu, 0u, ev);
        double u0 = or_u01(ev[0]), u1 = or_u01(ev[1]), u2 = or_u01(ev[2]), u3 = or_u01(ev[3]);
        double x, y;
        if (P->region == 0) {
#if OR_MUTANT == 12
            double rad = P->extent * u0, th = 6.283185307179586 * u1;
#else
            double rad = P->extent * sqrt(u0), th = 6.283185307179586 * u1;
#endif
            x = P->cx + rad * cos(th);
            y = P->cy + rad * sin(th);
        } else {
            x = P->cx + P->extent * (2.0 * u0 - 1.0);
            y = P->cy + P->extent * (2.0 * u1 - 1.0);
        }
        double E = P->e0 * (1.0 + P->e_spread * (2.0 * u2 - 1.0));
        double z = P->z_lo + (P->z_hi - P->z_lo) * u3;
        if (!or_is_3d(L->type)) z = 0.0;
        if (truth) {
            truth[4 * r] = x;
            truth[4 * r + 1] = y;
            truth[4 * r + 2] = z;
            truth[4 * r + 3] = E;
        }
        for (int i = 0; i < L->n_sensors; ++i) {
            int ok;
            double eta = or_lrf_eta(L, i, x, y, z, &ok);
            double lam = ok && eta > 0.0 ? E * eta : 0.0;
            or_stream st;
            or_stream_init(&st, seed, e, (uint32_t)i);
            double cnt = (double)or_poisson(lam, &st);
            if (P->spe_sigma > 0.0 && cnt > 0.0) {
                double a = or_next_u(&st), b = or_next_u(&st);
                double zn = sqrt(-2.0 * log(a)) * cos(6.283185307179586 * b);
                cnt = cnt + P->spe_sigma * sqrt(cnt) * zn;
                if (cnt < 0.0) cnt = 0.0;
            }
            sig[r * L->n_sensors + i] = cnt;
        }
    }
}

/* Poisson draws of one stream (for the distribution pins). */
void or_poisson_draws(double lam, uint64_t seed, long n, double *out)
{
    for (long e = 0; e < n; ++e) {
        or_stream st;
        or_stream_init(&st, seed, e, 0u);
        out[e] = (double)or_poisson(lam, &st);
    }
}

/* ------------------------------------------------------------------------ */
/* Global-grid log-response table of the precision form                     */
/* ------------------------------------------------------------------------ */
/* T[g][i] = ln p_i(g) - m_i with p_i = eta_i / sum_j eta_j at the centres of
 * the nx x ny cells of the XY box and m_i = mean_g ln p_i(g). */
void or_logtable(const or_lrf *L, int nx, int ny, double *T, double *m)
{
    long G = (long)nx * ny;
    int n = L->n_sensors;
#pragma omp parallel for schedule(static)
    for (long g = 0; g < G; ++g) {
        double x = L->lo[0] + ((double)(g % nx) + 0.5) * (L->hi[0] - L->lo[0]) / nx;
        double y = L->lo[1] + ((double)(g / nx) + 0.5) * (L->hi[1] - L->lo[1]) / ny;
        double H = 0.0;
        for (int i = 0; i < n; ++i) H += or_eta_floored(L, i, x, y, 0.0);
        for (int i = 0; i < n; ++i) T[g * n + i] = log(or_eta_floored(L, i, x, y, 0.0) / H);
    }
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (long g = 0; g < G; ++g) acc += T[g * n + i];
        m[i] = acc / (double)G;
        for (long g = 0; g < G; ++g) T[g * n + i] -= m[i];
    }
}

/* ------------------------------------------------------------------------ */
/* Event filters (Sec. 5.2) and the steps of iterative LRF reconstruction    */
/* (Sec. 8: reconstruct a flood dataset, discard badly reconstructed events, */
/* refit the LRFs from the reconstructed positions, repeat; Sec. 6.3: refit  */
/* the relative gains of a group with its LRF profile fixed)                 */
/* ------------------------------------------------------------------------ */

/* Chi-squared of a reconstruction, one of the quantities Sec. 5.2 filters
 * on.  Reading: Pearson's statistic of the signals against the mean counts
 * mu_i = E eta_i(x, y, z) at the reconstructed point, over the sensors with
 * mu_i > 0, divided by the degrees of freedom n_s - 3 (x, y and E fitted;
 * 1 when n_s <= 3).  NaN when the position or E is not finite. */
void or_chi2_at(const or_lrf *L, long n_e, const double *sig, const double *xyz, const double *E, double *chi2)
{
    int n = L->n_sensors;
    double dof = n > 3 ? (double)(n - 3) : 1.0;
#pragma omp parallel for schedule(static)
    for (long e = 0; e < n_e; ++e) {
        double x = xyz[3 * e], y = xyz[3 * e + 1], z = xyz[3 * e + 2], En = E[e];
        if (!isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(En)) {
            chi2[e] = NAN;
            continue;
        }
        double acc = 0.0;
        for (int i = 0; i < n; ++i) {
            int ok;
            double mu = En * or_lrf_eta(L, i, x, y, z, &ok);
            if (!ok || !(mu > 0.0)) continue;
            double d = sig[e * n + i] - mu;
#if OR_MUTANT == 13
            acc += d * d;
#else
            acc += d * d / mu;
#endif
        }
        chi2[e] = acc / dof;
    }
}

/* The cuts of Sec. 5.2 used by the iterative procedure; a cut whose upper
 * bound is not above its lower bound (or whose maximum is <= 0) is off. */
typedef struct {
    double chi2_max;       /* chi2 <= chi2_max */
    double e_lo, e_hi;     /* e_lo <= E <= e_hi */
    double sum_lo, sum_hi; /* sum_lo <= sum of signals <= sum_hi */
    double r_max, cx, cy;  /* (x - cx)^2 + (y - cy)^2 <= r_max^2 */
} or_filter;

/* keep[e] = 1 when event e was reconstructed (status OK, finite position,
 * energy and chi2) and passes every active cut. */
void or_event_filter(long n_e, const int *status, const double *xyz, const double *E, const double *chi2,
                     const double *sum, const or_filter *F, int *keep)
{
    for (long e = 0; e < n_e; ++e) {
        double x = xyz[3 * e], y = xyz[3 * e + 1], z = xyz[3 * e + 2];
        int k = status[e] == OR_EVT_OK && isfinite(x) && isfinite(y) && isfinite(z) && isfinite(E[e]) &&
                isfinite(chi2[e]);
        if (k && F->chi2_max > 0.0) k = chi2[e] <= F->chi2_max;
        if (k && F->e_hi > F->e_lo) k = E[e] >= F->e_lo && E[e] <= F->e_hi;
        if (k && F->sum_hi > F->sum_lo) k = sum[e] >= F->sum_lo && sum[e] <= F->sum_hi;
        if (k && F->r_max > 0.0) {
            double dx = x - F->cx, dy = y - F->cy;
            k = dx * dx + dy * dy <= F->r_max * F->r_max;
        }
        keep[e] = k;
    }
}

/* Random shift of reconstructed positions before a refit (Sec. 8: a small
 * random shift helps the first iterations).  Reading: a normal pair of
 * standard deviation sigma per event, by the Box-Muller transform of the
 * first two uniforms of the Philox block at counter (e_lo, e_hi, 0xFFFFFFFE,
 * cycle) under key `seed`; e is the event's index in the flood dataset. */
void or_shift_xy(uint64_t seed, int cycle, long n, const long *event, double sigma, double *dxy)
{
    for (long k = 0; k < n; ++k) {
        uint64_t e = (uint64_t)event[k];
        uint32_t w[4];
        or_philox_block(seed, (uint32_t)e, (uint32_t)(e >> 32), 0xFFFFFFFEu, (uint32_t)cycle, w);
        double ua = or_u01(w[0]), ub = or_u01(w[1]);
        double rho = sqrt(-2.0 * log(ua)), th = 6.283185307179586 * ub;
        dxy[2 * k] = sigma * rho * cos(th);
#if OR_MUTANT == 14
        dxy[2 * k + 1] = sigma * rho * cos(th);
#else
        dxy[2 * k + 1] = sigma * rho * sin(th);
#endif
    }
}

/* Relative gains of one group with its profile f fixed (Sec. 6.3): g_i
 * minimises sum_e (v_ei - g_i f(r_ei))^2 over the samples of sensor i with
 * r_ei inside the profile's domain, so g_i = sum f v / sum f^2.
 * r, v: [n_e][n_s]; coef: the profile's n_int + 3 coefficients.  A sensor
 * without samples (sum f^2 = 0) gets g_i = NaN. */
void or_gain_refit(int n_int, double lo, double hi, const double *coef, long n_e, int n_s, const double *r,
                   const double *v, double *g)
{
    for (int i = 0; i < n_s; ++i) {
        double fv = 0.0, ff = 0.0;
        for (long e = 0; e < n_e; ++e) {
            double B[4];
            int j0 = or_bspline_basis4(n_int, lo, hi, r[e * n_s + i], B);
            if (j0 < 0) continue;
            double f = 0.0;
            for (int a = 0; a < 4; ++a) f += coef[j0 + a] * B[a];
#if OR_MUTANT == 15
            fv += f * v[e * n_s + i];
            ff += f;
#else
            fv += f * v[e * n_s + i];
            ff += f * f;
#endif
        }
        g[i] = ff > 0.0 ? fv / ff : NAN;
    }
}
