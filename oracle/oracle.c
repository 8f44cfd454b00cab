/*
 * FP64 single-threaded CPU oracle for the mass-spring cloth step of
 * "Real-Time Cloth Simulation Using WebGPU" (arXiv 2507.11794).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain statement of what
 * the GPU path must compute; it is used by the test-suite, by the smoke check
 * and by the benchmark's CPU-baseline leg, and by nothing else.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Precision: double throughout, except the broad-phase cell formula, which
 * is defined in float32 (round-to-nearest, no FMA contraction: this file is
 * compiled with -ffp-contract=off) so that integer candidate sets can be
 * compared bit for bit with the GPU on identical float32 inputs.
 *
 * One substep (global index k, time t_k = k*dt_s) follows the paper's frame
 * (Section 3, Methodology):
 *   1. spring forces, spring-centric exactly as Algorithm 1: for every spring
 *      (node1=a, node2=b) dir = normalize(p_b - p_a),
 *      F = (ks*(|p_b - p_a| - L0) + kd*(v_b.dir - v_a.dir)) * dir,
 *      Force[a] += F, Force[b] -= F, springs taken in canonical order;
 *   2. "the Euler method" with spring force, gravity and external force
 *      (Section 3), read as symplectic Euler: v += dt_s*(F/m + g + w),
 *      x* = x + dt_s*v; pinned nodes move kinematically at the prescribed pin
 *      velocity u (x += dt_s*u, v = u; u = 0: fixed pins, the paper's hanging
 *      cloth; u != 0: its pulling scene);
 *   3. collision of the segment x -> x* of every free node with the static
 *      surface triangles by the extended Moller-Trumbore test (Section 3,
 *      "Extended Moller-Trumbore Process"), candidates from a uniform grid
 *      (or all triangles in brute-force mode);
 *   4. response (Section 3 and Algorithm 2): with K > 0 hits the node moves
 *      from its previous position along the averaged response direction,
 *      x = S + (1/K) * sum_k max(t_k - delta, 0) * r, and v = -0.5 * v;
 *      otherwise x = x*.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OC_PI 3.14159265358979323846

typedef struct {
    int32_t nx, ny;
    double origin[3], du[3], dv[3];  /* rest position X0(r,c) = origin + c*du + r*dv */
    double mass;                     /* per node */
    double ks[3], kd[3];             /* per spring type: structural, shear, bend */
    const double *ks_spring;         /* NULL or one value per spring, canonical order */
    const double *kd_spring;
    const uint8_t *pinned;           /* NULL or N bytes (nonzero = pinned) */
    double gravity[3];
    double dt_s;                     /* substep */
    double delta;                    /* contact offset along the path */
    double eps;                      /* epsilon of the extended MT test (|a| < eps: parallel) */
    double t_min;                    /* lower bound of the hit distance: t_min < t < |d| */
    double restitution;              /* velocity factor on contact (Alg. 2: -0.5) */
    double wind_amp, wind_dir[3], wind_udir[3], wind_freq, wind_kappa, wind_phase;
    double pin_vel[3];               /* pinned nodes move kinematically: x += dt_s*u, v = u */
} OcCloth;

typedef struct {
    float h, inv;          /* cell size and its float reciprocal */
    float origin[3];
    int32_t dims[3];
    int64_t ncells;
    int64_t nentries;
    int32_t *cell_start;   /* ncells + 1 */
    int32_t *tri_ids;      /* nentries, ascending within each cell */
} OcGrid;

typedef struct {
    const float *verts;    /* V x 3 */
    int32_t nverts;
    const int32_t *tris;   /* T x 3 */
    int32_t ntris;
} OcMesh;

/* Canonical spring directions (drow, dcol) and their types. */
static const int oc_dir_r[6] = {0, 1, 1, 1, 0, 2};
static const int oc_dir_c[6] = {1, 0, 1, -1, 2, 0};
static const int oc_dir_t[6] = {0, 0, 1, 1, 2, 2};

/* ------------------------------------------------------------------ springs */

/* Enumerate springs in canonical order: nodes row-major, each emitting the
 * six directions above when the other end is inside the grid.  Writes up to
 * `cap` entries and returns the total count. */
int64_t oc_springs(int32_t nx, int32_t ny, int32_t *a, int32_t *b, int32_t *type, int64_t cap)
{
    int64_t s = 0;
    for (int32_t r = 0; r < ny; r++)
        for (int32_t c = 0; c < nx; c++)
            for (int d = 0; d < 6; d++) {
                int32_t r2 = r + oc_dir_r[d], c2 = c + oc_dir_c[d];
                if (r2 < 0 || r2 >= ny || c2 < 0 || c2 >= nx) continue;
                if (s < cap) {
                    if (a) a[s] = r * nx + c;
                    if (b) b[s] = r2 * nx + c2;
                    if (type) type[s] = oc_dir_t[d];
                }
                s++;
            }
    return s;
}

static void oc_rest(const OcCloth *cl, int32_t node, double X0[3])
{
    int32_t r = node / cl->nx, c = node % cl->nx;
    for (int k = 0; k < 3; k++) X0[k] = cl->origin[k] + c * cl->du[k] + r * cl->dv[k];
}

/* Spring forces only (Algorithm 1), accumulated into F (3N, zeroed here). */
void oc_spring_forces(const OcCloth *cl, const double *x, const double *v, double *F)
{
    const int64_t N = (int64_t)cl->nx * cl->ny;
    memset(F, 0, sizeof(double) * 3 * N);
    int64_t s = 0;
    for (int32_t r = 0; r < cl->ny; r++)
        for (int32_t c = 0; c < cl->nx; c++)
            for (int d = 0; d < 6; d++) {
                int32_t r2 = r + oc_dir_r[d], c2 = c + oc_dir_c[d];
                if (r2 < 0 || r2 >= cl->ny || c2 < 0 || c2 >= cl->nx) continue;
                int32_t n1 = r * cl->nx + c, n2 = r2 * cl->nx + c2;
                int t = oc_dir_t[d];
                double ks = cl->ks_spring ? cl->ks_spring[s] : cl->ks[t];
                double kd = cl->kd_spring ? cl->kd_spring[s] : cl->kd[t];
                s++;
                /* rest length from the flat (un-jittered) grid */
                double X1[3], X2[3], L0 = 0.0;
                oc_rest(cl, n1, X1);
                oc_rest(cl, n2, X2);
                for (int k = 0; k < 3; k++) L0 += (X2[k] - X1[k]) * (X2[k] - X1[k]);
                L0 = sqrt(L0);
                double d3[3], len = 0.0;
                for (int k = 0; k < 3; k++) {
                    d3[k] = x[3 * n2 + k] - x[3 * n1 + k];
                    len += d3[k] * d3[k];
                }
                len = sqrt(len);
                if (len < 1e-12) continue; /* normalize() undefined: no contribution */
                double dir[3], v2d = 0.0, v1d = 0.0;
                for (int k = 0; k < 3; k++) {
                    dir[k] = d3[k] / len;
                    v2d += v[3 * n2 + k] * dir[k];
                    v1d += v[3 * n1 + k] * dir[k];
                }
                double spring = ks * (len - L0);
                double damp = kd * (v2d - v1d);
                for (int k = 0; k < 3; k++) {
                    double f = (spring + damp) * dir[k];
                    F[3 * n1 + k] += f;
                    F[3 * n2 + k] -= f;
                }
            }
}

/* External acceleration at node i, time t: gravity + wind
 * w(X0,t) = amp * dir * sin(2*pi*freq*t + kappa*(udir . X0) + phase). */
static void oc_external(const OcCloth *cl, int32_t i, double t, double a[3])
{
    double X0[3];
    oc_rest(cl, i, X0);
    double ph = 2.0 * OC_PI * cl->wind_freq * t + cl->wind_phase;
    ph += cl->wind_kappa * (cl->wind_udir[0] * X0[0] + cl->wind_udir[1] * X0[1] + cl->wind_udir[2] * X0[2]);
    double w = cl->wind_amp * sin(ph);
    for (int k = 0; k < 3; k++) a[k] = cl->gravity[k] + w * cl->wind_dir[k];
}

/* Full acceleration a_i = F_i/m + g + w(X0_i, t) for every node. */
void oc_accel(const OcCloth *cl, const double *x, const double *v, double t, double *A)
{
    const int64_t N = (int64_t)cl->nx * cl->ny;
    oc_spring_forces(cl, x, v, A);
    for (int64_t i = 0; i < N; i++) {
        double e[3];
        oc_external(cl, (int32_t)i, t, e);
        for (int k = 0; k < 3; k++) A[3 * i + k] = A[3 * i + k] / cl->mass + e[k];
    }
}

/* -------------------------------------------------------------- MT test */

/* Extended Moller-Trumbore segment-triangle test, in the paper's steps.
 * Returns 1 and writes t (distance from S along r) on a hit.  The paper
 * bounds t by the same epsilon as the parallel test (eps < t < |d|); the
 * lower bound is a separate argument here (t_min = eps is the literal text,
 * t_min = 0 the default reading of the cloth step). */
int oc_mt(const double S[3], const double E[3], const double V0[3], const double V1[3],
          const double V2[3], double eps, double t_min, double *t_out)
{
    double d[3], L = 0.0;
    for (int k = 0; k < 3; k++) { d[k] = E[k] - S[k]; L += d[k] * d[k]; }
    L = sqrt(L);
    if (L < eps) return 0; /* zero-length edge: nothing to intersect */
    double r[3], e1[3], e2[3], s[3];
    for (int k = 0; k < 3; k++) {
        r[k] = d[k] / L;
        e1[k] = V1[k] - V0[k];
        e2[k] = V2[k] - V0[k];
        s[k] = S[k] - V0[k];
    }
    double h[3] = {r[1] * e2[2] - r[2] * e2[1], r[2] * e2[0] - r[0] * e2[2], r[0] * e2[1] - r[1] * e2[0]};
    double a = e1[0] * h[0] + e1[1] * h[1] + e1[2] * h[2];
    if (fabs(a) < eps) return 0;
    double f = 1.0 / a;
    double u = f * (s[0] * h[0] + s[1] * h[1] + s[2] * h[2]);
    if (u < 0.0 || u > 1.0) return 0;
    double q[3] = {s[1] * e1[2] - s[2] * e1[1], s[2] * e1[0] - s[0] * e1[2], s[0] * e1[1] - s[1] * e1[0]};
    double vv = f * (r[0] * q[0] + r[1] * q[1] + r[2] * q[2]);
    double t = f * (e2[0] * q[0] + e2[1] * q[1] + e2[2] * q[2]);
    if (vv < 0.0 || u + vv > 1.0) return 0;
    if (!(t > t_min && t < L)) return 0;
    *t_out = t;
    return 1;
}

/* ---------------------------------------------------------- uniform grid */

/* Cell coordinate of one float coordinate: floor((x - o) * inv) evaluated in
 * float32 with round-to-nearest and no contraction, clamped to [0, dim-1]
 * (NaN maps to 0). */
static int32_t oc_cell_coord(float x, float o, float inv, int32_t dim)
{
    float dlt = x - o;
    float sc = dlt * inv;
    float fl = floorf(sc);
    if (!(fl >= 0.0f)) fl = 0.0f;
    if (fl > (float)(dim - 1)) fl = (float)(dim - 1);
    return (int32_t)fl;
}

/* Grid parameters: h = (float)(2 * mean over triangles of the longest side of
 * the triangle's AABB), the sum taken in double in triangle order;
 * origin = (float)(meshmin - 1.5h); dims = floor((max - min)/h) + 4 per axis
 * (so the outermost layer of cells holds no triangle, with half a cell of
 * slack for float rounding);
 * while the cell count exceeds 2^24 the cell size doubles.  A mesh whose
 * triangles all have zero extent gets h = 1. */
int oc_grid_params(const float *verts, const int32_t *tris, int32_t nt, float *h_out,
                   float origin[3], int32_t dims[3], float *inv_out)
{
    if (nt <= 0) return -1;
    double sum = 0.0;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int32_t t = 0; t < nt; t++) {
        float lo[3], hi[3];
        for (int k = 0; k < 3; k++) { lo[k] = INFINITY; hi[k] = -INFINITY; }
        for (int j = 0; j < 3; j++) {
            const float *p = verts + 3 * (int64_t)tris[3 * (int64_t)t + j];
            for (int k = 0; k < 3; k++) {
                if (p[k] < lo[k]) lo[k] = p[k];
                if (p[k] > hi[k]) hi[k] = p[k];
            }
        }
        double side = 0.0;
        for (int k = 0; k < 3; k++) {
            double e = (double)hi[k] - (double)lo[k];
            if (e > side) side = e;
            if (lo[k] < mn[k]) mn[k] = lo[k];
            if (hi[k] > mx[k]) mx[k] = hi[k];
        }
        sum += side;
    }
    float h = (float)(2.0 * (sum / (double)nt));
    if (!(h > 0.0f)) h = 1.0f;
    for (;;) {
        int64_t cells = 1;
        for (int k = 0; k < 3; k++) {
            origin[k] = (float)((double)mn[k] - 1.5 * (double)h);
            dims[k] = (int32_t)floor(((double)mx[k] - (double)mn[k]) / (double)h) + 4;
            cells *= dims[k];
        }
        if (cells <= (int64_t)1 << 24) break;
        h = h * 2.0f;
    }
    *h_out = h;
    *inv_out = (float)(1.0 / (double)h);
    return 0;
}

static void oc_tri_cells(const OcGrid *g, const float *verts, const int32_t *tri, int32_t lo[3], int32_t hi[3])
{
    for (int k = 0; k < 3; k++) {
        float a = verts[3 * (int64_t)tri[0] + k], b = verts[3 * (int64_t)tri[1] + k],
              c = verts[3 * (int64_t)tri[2] + k];
        float mn = a < b ? a : b, mx = a > b ? a : b;
        mn = c < mn ? c : mn;
        mx = c > mx ? c : mx;
        lo[k] = oc_cell_coord(mn, g->origin[k], g->inv, g->dims[k]);
        hi[k] = oc_cell_coord(mx, g->origin[k], g->inv, g->dims[k]);
    }
}

/* Counting sort of (cell, triangle) pairs: every triangle is listed in every
 * cell of its float AABB's cell range; filling in triangle order leaves each
 * cell's list ascending. */
int oc_grid_build(const float *verts, int32_t nv, const int32_t *tris, int32_t nt, OcGrid *g)
{
    memset(g, 0, sizeof(*g));
    for (int64_t i = 0; i < 3 * (int64_t)nt; i++)
        if (tris[i] < 0 || tris[i] >= nv) return -2;
    if (oc_grid_params(verts, tris, nt, &g->h, g->origin, g->dims, &g->inv)) return -1;
    g->ncells = (int64_t)g->dims[0] * g->dims[1] * g->dims[2];
    int64_t *cnt = calloc((size_t)g->ncells + 1, sizeof(int64_t));
    g->cell_start = malloc(sizeof(int32_t) * ((size_t)g->ncells + 1));
    if (!cnt || !g->cell_start) return -3;
    for (int32_t t = 0; t < nt; t++) {
        int32_t lo[3], hi[3];
        oc_tri_cells(g, verts, tris + 3 * (int64_t)t, lo, hi);
        for (int32_t z = lo[2]; z <= hi[2]; z++)
            for (int32_t y = lo[1]; y <= hi[1]; y++)
                for (int32_t x = lo[0]; x <= hi[0]; x++)
                    cnt[((int64_t)z * g->dims[1] + y) * g->dims[0] + x]++;
    }
    int64_t run = 0;
    for (int64_t c = 0; c < g->ncells; c++) {
        g->cell_start[c] = (int32_t)run;
        run += cnt[c];
        cnt[c] = g->cell_start[c];
    }
    g->cell_start[g->ncells] = (int32_t)run;
    g->nentries = run;
    g->tri_ids = malloc(sizeof(int32_t) * (size_t)(run > 0 ? run : 1));
    if (!g->tri_ids) return -3;
    for (int32_t t = 0; t < nt; t++) {
        int32_t lo[3], hi[3];
        oc_tri_cells(g, verts, tris + 3 * (int64_t)t, lo, hi);
        for (int32_t z = lo[2]; z <= hi[2]; z++)
            for (int32_t y = lo[1]; y <= hi[1]; y++)
                for (int32_t x = lo[0]; x <= hi[0]; x++)
                    g->tri_ids[cnt[((int64_t)z * g->dims[1] + y) * g->dims[0] + x]++] = t;
    }
    free(cnt);
    return 0;
}

void oc_grid_free(OcGrid *g)
{
    free(g->cell_start);
    free(g->tri_ids);
    memset(g, 0, sizeof(*g));
}

static int oc_cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Union of the triangle lists of the cell box [lo, hi], ascending, unique.
 * Returns the count; *buf is grown as needed. */
static int64_t oc_gather_cells(const OcGrid *g, const int32_t lo[3], const int32_t hi[3],
                               int32_t **buf, int64_t *cap)
{
    int64_t n = 0;
    for (int32_t z = lo[2]; z <= hi[2]; z++)
        for (int32_t y = lo[1]; y <= hi[1]; y++)
            for (int32_t x = lo[0]; x <= hi[0]; x++) {
                int64_t c = ((int64_t)z * g->dims[1] + y) * g->dims[0] + x;
                for (int32_t e = g->cell_start[c]; e < g->cell_start[c + 1]; e++) {
                    if (n == *cap) {
                        *cap = *cap ? 2 * *cap : 64;
                        *buf = realloc(*buf, sizeof(int32_t) * (size_t)*cap);
                    }
                    (*buf)[n++] = g->tri_ids[e];
                }
            }
    if (n > 1) {
        qsort(*buf, (size_t)n, sizeof(int32_t), oc_cmp_i32);
        int64_t m = 1;
        for (int64_t i = 1; i < n; i++)
            if ((*buf)[i] != (*buf)[m - 1]) (*buf)[m++] = (*buf)[i];
        n = m;
    }
    return n;
}

/* Candidate set of the float32 segment S->E: the cells of its float AABB by
 * the float32 cell formula (the definition the GPU grid must match bit for
 * bit).  Writes up to `cap` ids, returns the full count. */
int64_t oc_candidates_f32(const OcGrid *g, const float S[3], const float E[3], int32_t *out, int64_t cap)
{
    int32_t lo[3], hi[3];
    for (int k = 0; k < 3; k++) {
        float mn = S[k] < E[k] ? S[k] : E[k];
        float mx = S[k] > E[k] ? S[k] : E[k];
        lo[k] = oc_cell_coord(mn, g->origin[k], g->inv, g->dims[k]);
        hi[k] = oc_cell_coord(mx, g->origin[k], g->inv, g->dims[k]);
    }
    int32_t *buf = NULL;
    int64_t bcap = 0;
    int64_t n = oc_gather_cells(g, lo, hi, &buf, &bcap);
    for (int64_t i = 0; i < n && i < cap; i++) out[i] = buf[i];
    free(buf);
    return n;
}

/* Conservative cell range of a double segment, padded by 1e-6 m, so the
 * oracle's own broad phase never drops a triangle that all-pairs testing of
 * its double trajectory would hit. */
static void oc_cells_f64(const OcGrid *g, const double S[3], const double E[3], int32_t lo[3], int32_t hi[3])
{
    const double pad = 1e-6;
    for (int k = 0; k < 3; k++) {
        double mn = (S[k] < E[k] ? S[k] : E[k]) - pad;
        double mx = (S[k] > E[k] ? S[k] : E[k]) + pad;
        double inv = 1.0 / (double)g->h;
        double a = floor((mn - (double)g->origin[k]) * inv);
        double b = floor((mx - (double)g->origin[k]) * inv);
        if (!(a >= 0.0)) a = 0.0;
        if (a > g->dims[k] - 1) a = g->dims[k] - 1;
        if (!(b >= 0.0)) b = 0.0;
        if (b > g->dims[k] - 1) b = g->dims[k] - 1;
        lo[k] = (int32_t)a;
        hi[k] = (int32_t)b;
    }
}

/* ------------------------------------------------------------------ step */

/* Candidate triangles of the free node's path S -> E (grid, or all of them
 * when grid is NULL), into *buf; returns their count. */
static int64_t oc_candidates(const OcMesh *mesh, const OcGrid *grid, const double S[3], const double E[3],
                             int32_t **buf, int64_t *bcap)
{
    if (grid) {
        int32_t lo[3], hi[3];
        oc_cells_f64(grid, S, E, lo, hi);
        return oc_gather_cells(grid, lo, hi, buf, bcap);
    }
    const int64_t nc = mesh->ntris;
    if (*bcap < nc) {
        *bcap = nc;
        *buf = realloc(*buf, sizeof(int32_t) * (size_t)*bcap);
    }
    for (int64_t j = 0; j < nc; j++) (*buf)[j] = (int32_t)j;
    return nc;
}

/* Hits of the path S -> E (extended MT, candidates in ascending id):
 * returns K, *acc = sum max(t_k - delta, 0).  With g1/g2 non-NULL also the
 * sums over the active hits (t_k > delta) of n/a and t n/a, n = e1 x e2,
 * a = e1.(r x e2): the derivatives dt/dS = n/a and dt/dr = t n/a of the
 * distance to the triangle's plane along r. */
static int32_t oc_hits(const OcCloth *cl, const OcMesh *mesh, const OcGrid *grid, const double S[3],
                       const double E[3], int32_t **buf, int64_t *bcap, double *acc, double g1[3], double g2[3],
                       uint64_t *sig)
{
    int32_t K = 0;
    *acc = 0.0;
    if (g1) g1[0] = g1[1] = g1[2] = g2[0] = g2[1] = g2[2] = 0.0;
    if (!mesh || mesh->ntris <= 0) return 0;
    const int64_t nc = oc_candidates(mesh, grid, S, E, buf, bcap);
    double d[3], L = 0.0, r[3];
    for (int k = 0; k < 3; k++) { d[k] = E[k] - S[k]; L += d[k] * d[k]; }
    L = sqrt(L);
    for (int k = 0; k < 3; k++) r[k] = L > 0.0 ? d[k] / L : 0.0;
    for (int64_t j = 0; j < nc; j++) {
        const int32_t tid = (*buf)[j];
        const int32_t *tr = mesh->tris + 3 * (int64_t)tid;
        double V[3][3];
        for (int q = 0; q < 3; q++)
            for (int k = 0; k < 3; k++) V[q][k] = (double)mesh->verts[3 * (int64_t)tr[q] + k];
        double th;
        if (!oc_mt(S, E, V[0], V[1], V[2], cl->eps, cl->t_min, &th)) continue;
        K++;
        /* the signature records the hit and which side of the max(t - delta, 0)
           kink it lies on */
        if (sig) *sig = (*sig ^ ((uint64_t)(tid + 1) * 2u + (th - cl->delta > 0.0))) * 0x100000001b3ull;
        if (th - cl->delta > 0.0) {
            *acc += th - cl->delta;
            if (g1) {
                double e1[3], e2[3];
                for (int k = 0; k < 3; k++) { e1[k] = V[1][k] - V[0][k]; e2[k] = V[2][k] - V[0][k]; }
                double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                               e1[0] * e2[1] - e1[1] * e2[0]};
                double a = -(n[0] * r[0] + n[1] * r[1] + n[2] * r[2]);
                for (int k = 0; k < 3; k++) {
                    g1[k] += n[k] / a;
                    g2[k] += th * n[k] / a;
                }
            }
        }
    }
    return K;
}

/* Advance nsub substeps starting at global substep index k0.  x, v: 3N
 * doubles (node-major xyz), updated in place.  mesh may be NULL (no
 * collision).  grid NULL with a mesh means brute force over all triangles.
 * Optional outputs: hits (N ints) = hit count K of every node in the last
 * substep; xh, vh, vph (nsub*3N doubles) = position and velocity at the
 * start of every substep and the velocity after integration; sig = a hash of
 * every (substep, node, hit triangle) -- equal signatures mean equal contact
 * sets.  Returns 0, or -3 on allocation failure. */
int oc_step_ex(const OcCloth *cl, const OcMesh *mesh, const OcGrid *grid, double *x, double *v, int64_t k0,
               int32_t nsub, int32_t *hits, double *xh, double *vh, double *vph, uint64_t *sig)
{
    const int64_t N = (int64_t)cl->nx * cl->ny;
    double *A = malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    int32_t *buf = NULL;
    int64_t bcap = 0;
    if (!A) return -3;
    for (int32_t s = 0; s < nsub; s++) {
        double t = (double)(k0 + s) * cl->dt_s;
        if (xh) memcpy(xh + (int64_t)s * 3 * N, x, sizeof(double) * 3 * (size_t)N);
        if (vh) memcpy(vh + (int64_t)s * 3 * N, v, sizeof(double) * 3 * (size_t)N);
        oc_accel(cl, x, v, t, A);
        for (int64_t i = 0; i < N; i++) {
            int pinned = cl->pinned && cl->pinned[i];
            if (hits) hits[i] = 0;
            if (pinned) {
                /* kinematic pin: prescribed velocity, no force, no collision */
                for (int k = 0; k < 3; k++) {
                    v[3 * i + k] = cl->pin_vel[k];
                    x[3 * i + k] += cl->dt_s * cl->pin_vel[k];
                    if (vph) vph[((int64_t)s * N + i) * 3 + k] = cl->pin_vel[k];
                }
                continue;
            }
            double S[3], E[3];
            for (int k = 0; k < 3; k++) {
                v[3 * i + k] += cl->dt_s * A[3 * i + k];
                S[k] = x[3 * i + k];
                E[k] = S[k] + cl->dt_s * v[3 * i + k];
                if (vph) vph[((int64_t)s * N + i) * 3 + k] = v[3 * i + k];
            }
            if (sig) *sig = (*sig ^ (uint64_t)(s * N + i + 1)) * 0x100000001b3ull;
            double acc;
            const int32_t K = oc_hits(cl, mesh, grid, S, E, &buf, &bcap, &acc, NULL, NULL, sig);
            if (K > 0) {
                double L = 0.0, d[3];
                for (int k = 0; k < 3; k++) { d[k] = E[k] - S[k]; L += d[k] * d[k]; }
                L = sqrt(L);
                double m = acc / (double)K;
                for (int k = 0; k < 3; k++) {
                    x[3 * i + k] = S[k] + m * (d[k] / L);
                    v[3 * i + k] *= cl->restitution;
                }
            } else {
                for (int k = 0; k < 3; k++) x[3 * i + k] = E[k];
            }
            if (hits) hits[i] = K;
        }
    }
    free(A);
    free(buf);
    return 0;
}

int oc_step(const OcCloth *cl, const OcMesh *mesh, const OcGrid *grid, double *x, double *v, int64_t k0,
            int32_t nsub, int32_t *hits)
{
    return oc_step_ex(cl, mesh, grid, x, v, k0, nsub, hits, NULL, NULL, NULL, NULL);
}

/* ------------------------------------------------------------- adjoint */

/* Reverse mode of nsub substeps from (x0, v0) at global substep k0, the
 * contact set of every substep frozen at the one the forward pass finds.
 * In: lx, lv = dL/dx, dL/dv at the end (3N each); out: the same arrays hold
 * dL/dx0, dL/dv0, and gks, gkd (S entries, canonical spring order) receive
 * += dL/dks_s, dL/dkd_s.  Per substep, backwards:
 *   response  x' = S + m(S, r) r, m = mean over hits of max(t_k - delta, 0),
 *             r = vs / |vs|, v' = c vs on contact; x' = S + dt vs, v' = vs
 *             otherwise (pinned: x' = x, v' = 0);
 *   Euler     vs = v + dt (F(x, v)/m + g + w);
 *   springs   F as in Algorithm 1, differentiated in x, v, ks, kd.
 * Returns 0, or -3 on allocation failure. */
int oc_adjoint(const OcCloth *cl, const OcMesh *mesh, const OcGrid *grid, const double *x0, const double *v0,
               int64_t k0, int32_t nsub, double *lx, double *lv, double *gks, double *gkd)
{
    const int64_t N = (int64_t)cl->nx * cl->ny;
    const size_t per = 3 * (size_t)N;
    double *xh = malloc(sizeof(double) * per * (size_t)nsub);
    double *vh = malloc(sizeof(double) * per * (size_t)nsub);
    double *vph = malloc(sizeof(double) * per * (size_t)nsub);
    double *x = malloc(sizeof(double) * per), *v = malloc(sizeof(double) * per);
    double *lF = malloc(sizeof(double) * per), *nlx = malloc(sizeof(double) * per), *nlv = malloc(sizeof(double) * per);
    int32_t *buf = NULL;
    int64_t bcap = 0;
    if (!xh || !vh || !vph || !x || !v || !lF || !nlx || !nlv) {
        free(xh); free(vh); free(vph); free(x); free(v); free(lF); free(nlx); free(nlv);
        return -3;
    }
    memcpy(x, x0, sizeof(double) * per);
    memcpy(v, v0, sizeof(double) * per);
    oc_step_ex(cl, mesh, grid, x, v, k0, nsub, NULL, xh, vh, vph, NULL);
    const double dt = cl->dt_s, c = cl->restitution;
    for (int32_t s = nsub - 1; s >= 0; s--) {
        const double *X = xh + (size_t)s * per, *VV = vh + (size_t)s * per, *VP = vph + (size_t)s * per;
        /* response and integration, node by node */
        for (int64_t i = 0; i < N; i++) {
            double *ox = nlx + 3 * i, *ov = nlv + 3 * i, *of = lF + 3 * i;
            const double *lxi = lx + 3 * i, *lvi = lv + 3 * i;
            if (cl->pinned && cl->pinned[i]) {
                for (int k = 0; k < 3; k++) { ox[k] = lxi[k]; ov[k] = 0.0; of[k] = 0.0; }
                continue;
            }
            double S[3], E[3], lvp[3];
            for (int k = 0; k < 3; k++) { S[k] = X[3 * i + k]; E[k] = S[k] + dt * VP[3 * i + k]; }
            double acc, g1[3], g2[3];
            const int32_t K = oc_hits(cl, mesh, grid, S, E, &buf, &bcap, &acc, g1, g2, NULL);
            if (K > 0) {
                double nv = sqrt(VP[3 * i] * VP[3 * i] + VP[3 * i + 1] * VP[3 * i + 1] + VP[3 * i + 2] * VP[3 * i + 2]);
                double r[3], lr[3];
                for (int k = 0; k < 3; k++) r[k] = VP[3 * i + k] / nv;
                const double m = acc / (double)K;
                const double rl = r[0] * lxi[0] + r[1] * lxi[1] + r[2] * lxi[2];
                for (int k = 0; k < 3; k++) {
                    ox[k] = lxi[k] + (g1[k] / (double)K) * rl;            /* dx'/dS */
                    lr[k] = m * lxi[k] + (g2[k] / (double)K) * rl;        /* dx'/dr */
                }
                const double rlr = r[0] * lr[0] + r[1] * lr[1] + r[2] * lr[2];
                for (int k = 0; k < 3; k++) lvp[k] = (lr[k] - r[k] * rlr) / nv + c * lvi[k];
            } else {
                for (int k = 0; k < 3; k++) { ox[k] = lxi[k]; lvp[k] = dt * lxi[k] + lvi[k]; }
            }
            for (int k = 0; k < 3; k++) { ov[k] = lvp[k]; of[k] = dt / cl->mass * lvp[k]; }
        }
        /* springs (Algorithm 1's order), differentiated */
        int64_t sp = 0;
        for (int32_t r = 0; r < cl->ny; r++)
            for (int32_t cc = 0; cc < cl->nx; cc++)
                for (int d = 0; d < 6; d++) {
                    int32_t r2 = r + oc_dir_r[d], c2 = cc + oc_dir_c[d];
                    if (r2 < 0 || r2 >= cl->ny || c2 < 0 || c2 >= cl->nx) continue;
                    const int32_t a = r * cl->nx + cc, b = r2 * cl->nx + c2;
                    const int t = oc_dir_t[d];
                    const double ks = cl->ks_spring ? cl->ks_spring[sp] : cl->ks[t];
                    const double kd = cl->kd_spring ? cl->kd_spring[sp] : cl->kd[t];
                    double X1[3], X2[3], L0 = 0.0, dd[3], len = 0.0;
                    oc_rest(cl, a, X1);
                    oc_rest(cl, b, X2);
                    for (int k = 0; k < 3; k++) L0 += (X2[k] - X1[k]) * (X2[k] - X1[k]);
                    L0 = sqrt(L0);
                    for (int k = 0; k < 3; k++) { dd[k] = X[3 * b + k] - X[3 * a + k]; len += dd[k] * dd[k]; }
                    len = sqrt(len);
                    if (len < 1e-12) { sp++; continue; }
                    double u[3], dv[3], mu[3], ud = 0.0, um = 0.0;
                    for (int k = 0; k < 3; k++) {
                        u[k] = dd[k] / len;
                        dv[k] = VV[3 * b + k] - VV[3 * a + k];
                        mu[k] = lF[3 * a + k] - lF[3 * b + k];
                        ud += u[k] * dv[k];
                        um += u[k] * mu[k];
                    }
                    const double phi = ks * (len - L0) + kd * ud;
                    if (gks) gks[sp] += um * (len - L0);
                    if (gkd) gkd[sp] += um * ud;
                    for (int k = 0; k < 3; k++) {
                        const double gd = phi / len * (mu[k] - u[k] * um) +
                                          um * (ks * u[k] + kd / len * (dv[k] - u[k] * ud));
                        const double gv = kd * u[k] * um;
                        nlx[3 * b + k] += gd;
                        nlx[3 * a + k] -= gd;
                        nlv[3 * b + k] += gv;
                        nlv[3 * a + k] -= gv;
                    }
                    sp++;
                }
        memcpy(lx, nlx, sizeof(double) * per);
        memcpy(lv, nlv, sizeof(double) * per);
    }
    free(xh); free(vh); free(vph); free(x); free(v); free(lF); free(nlx); free(nlv); free(buf);
    return 0;
}

/* ------------------------------------- edge-triangle narrow phase (f1) */

/* The paper's own narrow phase (Section 3): triangle-triangle collision
 * between the cloth at its updated positions and the surface model, by the
 * extended Moller-Trumbore test of the cloth triangles' edges against the
 * surface triangles; the nodes "affected by the collision between triangles"
 * move along "the average value of the direction" (Algorithm 2:
 * pos = prevPos + responseDirection, vel = -0.5 vel).  The paper gives no
 * formula for the direction; the reading here, parallel to the point-path
 * reading of the default narrow phase:
 *   - the cloth triangles are the grid's quads split along their
 *     (r,c)-(r+1,c+1) diagonal; the tested edges are the triangulation's
 *     edges (r,c)-(r,c+1), (r,c)-(r+1,c), (r,c)-(r+1,c+1) at the updated
 *     positions x*;
 *   - a hit of edge e at the point P affects every vertex of the (one or
 *     two) cloth triangles that contain e;
 *   - an affected free node i gets the direction from its previous position
 *     towards P, stopping delta short: max(|P - x_i| - delta, 0) (P - x_i)/|P - x_i|
 *     (zero when P = x_i); the directions of all its hits are averaged.
 * Free nodes with no hit end at x*; pinned nodes neither move nor receive. */

/* Affected nodes of edge kind q (0: (r,c)-(r,c+1), 1: (r,c)-(r+1,c),
 * 2: (r,c)-(r+1,c+1)) owned by node (r,c): up to 4 node indices into out;
 * returns their number (0 when the edge does not exist). */
int32_t oc_edge_affected(int32_t nx, int32_t ny, int32_t r, int32_t c, int32_t q, int32_t out[4])
{
    int32_t n = 0;
#define OC_NODE(rr, cc) ((int32_t)(rr) * nx + (int32_t)(cc))
    if (q == 0) {
        if (c + 1 >= nx) return 0;
        out[n++] = OC_NODE(r, c);
        out[n++] = OC_NODE(r, c + 1);
        if (r + 1 < ny) out[n++] = OC_NODE(r + 1, c + 1); /* second triangle of quad (r, c) */
        if (r >= 1) out[n++] = OC_NODE(r - 1, c);         /* first triangle of quad (r-1, c) */
    } else if (q == 1) {
        if (r + 1 >= ny) return 0;
        out[n++] = OC_NODE(r, c);
        out[n++] = OC_NODE(r + 1, c);
        if (c + 1 < nx) out[n++] = OC_NODE(r + 1, c + 1); /* first triangle of quad (r, c) */
        if (c >= 1) out[n++] = OC_NODE(r, c - 1);         /* second triangle of quad (r, c-1) */
    } else {
        if (r + 1 >= ny || c + 1 >= nx) return 0;
        out[n++] = OC_NODE(r, c);
        out[n++] = OC_NODE(r + 1, c + 1);
        out[n++] = OC_NODE(r + 1, c); /* both triangles of quad (r, c) */
        out[n++] = OC_NODE(r, c + 1);
    }
#undef OC_NODE
    return n;
}

/* nsub substeps with the edge-triangle narrow phase; arguments as oc_step.
 * hits (optional, N ints): number of hits each node received in the last
 * substep.  Returns 0, or -3 on allocation failure. */
int oc_step_edges(const OcCloth *cl, const OcMesh *mesh, const OcGrid *grid, double *x, double *v, int64_t k0,
                  int32_t nsub, int32_t *hits)
{
    const int64_t N = (int64_t)cl->nx * cl->ny;
    double *A = malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    double *E = malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    double *acc = malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    int32_t *cnt = malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    int32_t *buf = NULL;
    int64_t bcap = 0;
    int rc = 0;
    if (!A || !E || !acc || !cnt) {
        rc = -3;
        goto done;
    }
    for (int32_t s = 0; s < nsub; s++) {
        const double t = (double)(k0 + s) * cl->dt_s;
        oc_accel(cl, x, v, t, A);
        for (int64_t i = 0; i < N; i++) {
            const int pinned = cl->pinned && cl->pinned[i];
            for (int k = 0; k < 3; k++) {
                if (pinned) {
                    v[3 * i + k] = cl->pin_vel[k];
                    E[3 * i + k] = x[3 * i + k] + cl->dt_s * cl->pin_vel[k];
                } else {
                    v[3 * i + k] += cl->dt_s * A[3 * i + k];
                    E[3 * i + k] = x[3 * i + k] + cl->dt_s * v[3 * i + k];
                }
                acc[3 * i + k] = 0.0;
            }
            cnt[i] = 0;
        }
        if (mesh && mesh->ntris > 0) {
            for (int32_t r = 0; r < cl->ny; r++)
                for (int32_t c = 0; c < cl->nx; c++)
                    for (int32_t q = 0; q < 3; q++) {
                        int32_t aff[4];
                        const int32_t na = oc_edge_affected(cl->nx, cl->ny, r, c, q, aff);
                        if (na == 0) continue;
                        const int32_t a = r * cl->nx + c;
                        const int32_t b = q == 0 ? a + 1 : (q == 1 ? a + cl->nx : a + cl->nx + 1);
                        const double *Sa = E + 3 * (int64_t)a, *Eb = E + 3 * (int64_t)b;
                        double d[3], L = 0.0;
                        for (int k = 0; k < 3; k++) { d[k] = Eb[k] - Sa[k]; L += d[k] * d[k]; }
                        L = sqrt(L);
                        const int64_t nc = oc_candidates(mesh, grid, Sa, Eb, &buf, &bcap);
                        for (int64_t j = 0; j < nc; j++) {
                            const int32_t *tr = mesh->tris + 3 * (int64_t)buf[j];
                            double V[3][3];
                            for (int p = 0; p < 3; p++)
                                for (int k = 0; k < 3; k++) V[p][k] = (double)mesh->verts[3 * (int64_t)tr[p] + k];
                            double th;
                            if (!oc_mt(Sa, Eb, V[0], V[1], V[2], cl->eps, cl->t_min, &th)) continue;
                            double P[3];
                            for (int k = 0; k < 3; k++) P[k] = Sa[k] + th * (d[k] / L);
                            for (int32_t m = 0; m < na; m++) {
                                const int32_t i = aff[m];
                                if (cl->pinned && cl->pinned[i]) continue;
                                double w[3], lw = 0.0;
                                for (int k = 0; k < 3; k++) { w[k] = P[k] - x[3 * (int64_t)i + k]; lw += w[k] * w[k]; }
                                lw = sqrt(lw);
                                const double sc = lw > 0.0 ? (lw - cl->delta > 0.0 ? lw - cl->delta : 0.0) / lw : 0.0;
                                for (int k = 0; k < 3; k++) acc[3 * (int64_t)i + k] += sc * w[k];
                                cnt[i]++;
                            }
                        }
                    }
        }
        for (int64_t i = 0; i < N; i++) {
            if (cnt[i] > 0) {
                for (int k = 0; k < 3; k++) {
                    x[3 * i + k] += acc[3 * i + k] / (double)cnt[i];
                    v[3 * i + k] *= cl->restitution;
                }
            } else {
                for (int k = 0; k < 3; k++) x[3 * i + k] = E[3 * i + k];
            }
            if (hits) hits[i] = cnt[i];
        }
    }
done:
    free(A);
    free(E);
    free(acc);
    free(cnt);
    free(buf);
    return rc;
}
