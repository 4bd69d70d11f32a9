/*
 * md_oracle.c -- plain FP64 CPU oracle for the molecular-dynamics hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests/, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no source with the CUDA path.
 *
 * Every function is the plain definition written out, in FP64, with no
 * blocking, fusion or reordering:
 *   - periodic space: minimum-image displacement and wrapping   (Sec. 3.2.1)
 *   - neighbor sets {(i,j): i != j, r_ij < r_list}              (Sec. 3.2.3)
 *     built either by brute force over all pairs or from a cell list
 *   - pair energy U = 1/2 sum_{i != j} u(r_ij), F = -grad U     (Sec. 3.2.2, 3.3.2)
 *     for Lennard-Jones and soft spheres
 *   - Stillinger-Weber 2-body + 3-body energy and forces        (Sec. 3.3.2)
 *   - velocity-Verlet NVE, gradient-descent and FIRE minimisation,
 *     BAOAB Langevin NVT, Nose-Hoover chain NVT                  (Sec. 3.3.1)
 *   - reverse-mode derivative of the final energy of a gradient-descent
 *     minimisation with respect to the small-disk diameter D     (Sec. 4.2, App. A)
 *   - the flocking energy model of boids and its forward-Euler steps (Sec. 4.3)
 *   - Philox4x32-10 counter-based generator (Salmon et al., SC'11), the
 *     published definition, used for Langevin noise.
 *
 * Readings where the paper is silent (functional forms, constants, cutoff
 * comparisons) are stated at each function.
 *
 * Positions are double[N*3] (z = 0 in 2-D); the box is double[3].
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no -ffast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ----------------------------------------------------------------------- */
/* Periodic space (Sec. 3.2.1): the box is [0,L_x) x [0,L_y) (x [0,L_z)) with
 * r ~ r + n L.  The displacement is r_a - r_b taken to the nearest image. */
/* ----------------------------------------------------------------------- */
static void min_image64(int dim, const double *L, const double *a, const double *b, double *d)
{
    for (int k = 0; k < 3; ++k) d[k] = 0.0;
    for (int k = 0; k < dim; ++k) {
        double t = a[k] - b[k];
        d[k] = t - L[k] * nearbyint(t / L[k]);
    }
}

/* Image integers n of the minimum-image displacement d = a - b - n L. */
static void image_index64(int dim, const double *L, const double *a, const double *b, double *n)
{
    for (int k = 0; k < 3; ++k) n[k] = 0.0;
    for (int k = 0; k < dim; ++k) n[k] = nearbyint((a[k] - b[k]) / L[k]);
}

static double wrap64(double x, double L)
{
    double y = x - L * floor(x / L);
    if (y >= L) y -= L;
    if (y < 0.0) y = 0.0;
    return y;
}

/* Squared distance evaluated in FP32, used wherever a floating-point
 * comparison decides membership of a pair (the neighbor list and the LJ
 * cutoff).  Reading: the decision is taken in the precision the kernels use,
 * on FP32 coordinates and the FP32 box, with
 *     t = a - b;  d = t - L * rint(t * Linv);  r2 = (dx*dx + dy*dy) + dz*dz
 * each operation rounded separately (no fused multiply-add). Linv is 1/L
 * evaluated in FP64 and rounded to FP32. */
static float r2_f32(int dim, const float *Lf, const float *Linvf, const float *a, const float *b)
{
    float r2 = 0.0f;
    for (int k = 0; k < dim; ++k) {
        float t = a[k] - b[k];
        float n = rintf(t * Linvf[k]);
        float m = Lf[k] * n;
        float d = t - m;
        float dd = d * d;
        r2 = (k == 0) ? dd : (r2 + dd);
    }
    return r2;
}

/* ----------------------------------------------------------------------- */
/* Neighbor sets (Sec. 3.2.3): all j != i with r_ij < r_cut, as sorted CSR
 * rows.  Candidates come either from every particle (brute force) or from
 * a cell list whose cells have side >= r_cut; with fewer than three cells
 * along an axis, the periodic stencil offsets are deduplicated so each cell
 * is visited once.                                                        */
/* ----------------------------------------------------------------------- */
typedef struct {
    int n[3];
    int ncell;
    int *start;   /* [ncell+1] */
    int *atoms;   /* [N] ascending index inside each cell */
} cells_t;

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

static void cells_build(cells_t *c, int N, int dim, const double *r, const double *L, double side_min)
{
    for (int k = 0; k < 3; ++k) {
        c->n[k] = 1;
        if (k < dim) {
            int n = (int)floor(L[k] / side_min);
            c->n[k] = n < 1 ? 1 : n;
        }
    }
    c->ncell = c->n[0] * c->n[1] * c->n[2];
    int *cell_of = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    c->start = (int *)calloc((size_t)c->ncell + 1, sizeof(int));
    c->atoms = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    for (int i = 0; i < N; ++i) {
        int ci[3] = {0, 0, 0};
        for (int k = 0; k < dim; ++k) {
            double x = wrap64(r[3 * i + k], L[k]);
            int q = (int)floor(x / L[k] * c->n[k]);
            if (q >= c->n[k]) q = c->n[k] - 1;
            if (q < 0) q = 0;
            ci[k] = q;
        }
        cell_of[i] = (ci[2] * c->n[1] + ci[1]) * c->n[0] + ci[0];
        c->start[cell_of[i] + 1]++;
    }
    for (int q = 0; q < c->ncell; ++q) c->start[q + 1] += c->start[q];
    int *fill = (int *)calloc((size_t)c->ncell, sizeof(int));
    for (int i = 0; i < N; ++i) {      /* ascending i: stable */
        int q = cell_of[i];
        c->atoms[c->start[q] + fill[q]++] = i;
    }
    free(fill);
    free(cell_of);
}

static void cells_free(cells_t *c)
{
    free(c->start);
    free(c->atoms);
}

/* Distinct neighbor-cell indices along one axis: {(q-1) mod n, q, (q+1) mod n}. */
static int axis_stencil(int q, int n, int *out)
{
    int m = 0;
    for (int d = -1; d <= 1; ++d) {
        int v = ((q + d) % n + n) % n;
        int dup = 0;
        for (int s = 0; s < m; ++s) dup |= (out[s] == v);
        if (!dup) out[m++] = v;
    }
    return m;
}

/* Candidate list for particle i: every particle in the (deduplicated)
 * stencil of cells around i's cell, or all particles when c == NULL. */
static int candidates(const cells_t *c, int N, int dim, const double *r, const double *L, int i, int *buf)
{
    if (!c) {
        for (int j = 0; j < N; ++j) buf[j] = j;
        return N;
    }
    int ci[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
        double x = wrap64(r[3 * i + k], L[k]);
        int q = (int)floor(x / L[k] * c->n[k]);
        if (q >= c->n[k]) q = c->n[k] - 1;
        if (q < 0) q = 0;
        ci[k] = q;
    }
    int sx[3], sy[3], sz[3];
    int mx = axis_stencil(ci[0], c->n[0], sx);
    int my = axis_stencil(ci[1], c->n[1], sy);
    int mz = axis_stencil(ci[2], c->n[2], sz);
    int m = 0;
    for (int a = 0; a < mz; ++a)
        for (int b = 0; b < my; ++b)
            for (int e = 0; e < mx; ++e) {
                int q = (sz[a] * c->n[1] + sy[b]) * c->n[0] + sx[e];
                for (int s = c->start[q]; s < c->start[q + 1]; ++s) buf[m++] = c->atoms[s];
            }
    return m;
}

typedef struct {
    int N;
    long *start;  /* [N+1] */
    int *idx;
} csr_t;

static void csr_free(csr_t *g)
{
    free(g->start);
    free(g->idx);
}

/* mode 0: FP64 test d(r_i, r_j) < rcut;  mode 1: FP32 test r2_f32 < rc2_f32
 * with rc2_f32 = fl32(fl32(rcut) * fl32(rcut)).  use_cells: 0 brute force. */
static int pair_in(int mode, int dim, const double *L, const float *Lf, const float *Linvf,
                   const double *r, const float *rf, int i, int j, double rcut2, float rc2f)
{
    if (mode == 1) return r2_f32(dim, Lf, Linvf, rf + 3 * i, rf + 3 * j) < rc2f;
    double d[3];
    min_image64(dim, L, r + 3 * i, r + 3 * j, d);
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < rcut2;
}

static csr_t neighbors(int N, int dim, const double *r, const double *L, double rcut, int mode, int use_cells)
{
    csr_t g;
    g.N = N;
    g.start = (long *)calloc((size_t)N + 1, sizeof(long));
    float Lf[3], Linvf[3];
    for (int k = 0; k < 3; ++k) {
        Lf[k] = (float)L[k];
        Linvf[k] = (float)(1.0 / L[k]);
    }
    float *rf = (float *)malloc(sizeof(float) * 3 * (size_t)(N > 0 ? N : 1));
    for (int i = 0; i < 3 * N; ++i) rf[i] = (float)r[i];
    float rcf = (float)rcut;
    float rc2f = rcf * rcf;
    double rcut2 = rcut * rcut;
    cells_t c;
    cells_t *cp = NULL;
    if (use_cells) {
        /* margin so a pair accepted by the FP32 test is never outside the stencil */
        cells_build(&c, N, dim, r, L, rcut * (1.0 + 1e-4));
        cp = &c;
    }
    int *cnt = (int *)calloc((size_t)N + 1, sizeof(int));
#pragma omp parallel
    {
        int *buf = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < N; ++i) {
            int m = candidates(cp, N, dim, r, L, i, buf);
            int k = 0;
            for (int s = 0; s < m; ++s) {
                int j = buf[s];
                if (j != i && pair_in(mode, dim, L, Lf, Linvf, r, rf, i, j, rcut2, rc2f)) ++k;
            }
            cnt[i] = k;
        }
        free(buf);
    }
    for (int i = 0; i < N; ++i) g.start[i + 1] = g.start[i] + cnt[i];
    g.idx = (int *)malloc(sizeof(int) * (size_t)(g.start[N] > 0 ? g.start[N] : 1));
#pragma omp parallel
    {
        int *buf = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < N; ++i) {
            int m = candidates(cp, N, dim, r, L, i, buf);
            long k = g.start[i];
            for (int s = 0; s < m; ++s) {
                int j = buf[s];
                if (j != i && pair_in(mode, dim, L, Lf, Linvf, r, rf, i, j, rcut2, rc2f)) g.idx[k++] = j;
            }
            qsort(g.idx + g.start[i], (size_t)(k - g.start[i]), sizeof(int), cmp_int);
        }
        free(buf);
    }
    free(cnt);
    free(rf);
    if (cp) cells_free(cp);
    return g;
}

/* Exported: neighbor list as padded rows [N][cap] (sorted ascending, padded
 * with N) and counts [N]; a row longer than cap is truncated but its count
 * is the true count.  mode/use_cells as above.  Returns the total pair count. */
long or_neighbor_list(int N, int dim, const double *r, const double *L, double r_list, int mode,
                      int use_cells, int cap, int *cnt, int *nbr)
{
    csr_t g = neighbors(N, dim, r, L, r_list, mode, use_cells);
    for (int i = 0; i < N; ++i) {
        int c = (int)(g.start[i + 1] - g.start[i]);
        cnt[i] = c;
        for (int s = 0; s < cap; ++s) nbr[(long)i * cap + s] = (s < c) ? g.idx[g.start[i] + s] : N;
    }
    long tot = g.start[N];
    csr_free(&g);
    return tot;
}

/* ----------------------------------------------------------------------- */
/* Lennard-Jones (Sec. 3.3.2; form not printed in the paper).  Reading:
 *   u(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6] - u(r_c)   for r < r_c
 * with the energy shift applied when shifted != 0 and forces not shifted.
 * The r < r_c decision is the FP32 test above.  U = 1/2 sum_{i!=j} u(r_ij)
 * (Sec. 3.2.2), e_i = 1/2 sum_j u(r_ij), F_i = -dU/dr_i.                */
/* ----------------------------------------------------------------------- */
static double lj_u(double r, double eps, double sigma)
{
    double s6 = pow(sigma / r, 6.0);
    return 4.0 * eps * (s6 * s6 - s6);
}

/* du/dr */
static double lj_du(double r, double eps, double sigma)
{
    double s6 = pow(sigma / r, 6.0);
    return 4.0 * eps * (-12.0 * s6 * s6 + 6.0 * s6) / r;
}

double or_lj_pair(double r, double eps, double sigma, double *du)
{
    if (du) *du = lj_du(r, eps, sigma);
    return lj_u(r, eps, sigma);
}

double or_lj(int N, const double *r, const double *L, double eps, double sigma, double rc, int shifted,
             int use_cells, double *f, double *e)
{
    csr_t g = neighbors(N, 3, r, L, rc, 1, use_cells);
    double uc = shifted ? lj_u(rc, eps, sigma) : 0.0;
    double U = 0.0;
#pragma omp parallel for reduction(+ : U) schedule(dynamic, 64)
    for (int i = 0; i < N; ++i) {
        double fi[3] = {0, 0, 0}, ei = 0.0;
        for (long s = g.start[i]; s < g.start[i + 1]; ++s) {
            int j = g.idx[s];
            double d[3];
            min_image64(3, L, r + 3 * i, r + 3 * j, d);
            double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            ei += 0.5 * (lj_u(rr, eps, sigma) - uc);
            double du = lj_du(rr, eps, sigma);
            for (int k = 0; k < 3; ++k) fi[k] -= du * d[k] / rr;
        }
        if (f)
            for (int k = 0; k < 3; ++k) f[3 * i + k] = fi[k];
        if (e) e[i] = ei;
        U += ei;
    }
    csr_free(&g);
    return U;
}

/* ----------------------------------------------------------------------- */
/* Soft spheres (Sec. 3.3.2, O'Hern et al. 2003; form not printed).  Reading:
 *   u(r) = (eps/alpha) (1 - r/sigma_ij)^alpha  for r < sigma_ij, else 0,
 *   sigma_ij = (d_i + d_j)/2 (the mixing of App. A's species_sigma).   */
/* ----------------------------------------------------------------------- */
double or_soft(int N, int dim, const double *r, const double *diam, const double *L, double eps,
               double alpha, double *f, double *e)
{
    double dmax = 0.0;
    for (int i = 0; i < N; ++i) dmax = diam[i] > dmax ? diam[i] : dmax;
    csr_t g = neighbors(N, dim, r, L, dmax, 0, 1);
    double U = 0.0;
#pragma omp parallel for reduction(+ : U) schedule(dynamic, 64)
    for (int i = 0; i < N; ++i) {
        double fi[3] = {0, 0, 0}, ei = 0.0;
        for (long s = g.start[i]; s < g.start[i + 1]; ++s) {
            int j = g.idx[s];
            double d[3];
            min_image64(dim, L, r + 3 * i, r + 3 * j, d);
            double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double sg = 0.5 * (diam[i] + diam[j]);
            if (rr >= sg) continue;
            double x = 1.0 - rr / sg;
            ei += 0.5 * eps / alpha * pow(x, alpha);
            double du = -eps / sg * pow(x, alpha - 1.0);
            for (int k = 0; k < dim; ++k) fi[k] -= du * d[k] / rr;
        }
        if (f)
            for (int k = 0; k < 3; ++k) f[3 * i + k] = fi[k];
        if (e) e[i] = ei;
        U += ei;
    }
    csr_free(&g);
    return U;
}

/* ----------------------------------------------------------------------- */
/* Stillinger-Weber (Sec. 3.3.2; form from Stillinger & Weber 1985):
 *   E = sum_{i<j} phi2(r_ij) + sum_i sum_{j<k in N(i)} phi3(r_ij, r_ik, theta_jik)
 *   phi2(r) = A eps [B (sigma/r)^p - (sigma/r)^q] exp(sigma / (r - a sigma))
 *   phi3    = lambda eps (cos theta_jik - cos0)^2
 *             exp(gamma sigma/(r_ij - a sigma)) exp(gamma sigma/(r_ik - a sigma))
 * all for r < a sigma.  P = {eps, sigma, a, lambda, gamma, A, B, p, q, cos0}.
 * e_i = 1/2 sum_j phi2(r_ij) + sum_{j<k} phi3(i; j, k).               */
/* ----------------------------------------------------------------------- */
static double sw_phi2(const double *P, double r, double *dphi)
{
    double eps = P[0], sg = P[1], a = P[2], A = P[5], B = P[6], p = P[7], q = P[8];
    double rc = a * sg;
    if (r >= rc) {
        *dphi = 0.0;
        return 0.0;
    }
    double bra = B * pow(sg / r, p) - pow(sg / r, q);
    double dbra = -p * B * pow(sg / r, p) / r + q * pow(sg / r, q) / r;
    double ex = exp(sg / (r - rc));
    double dex = ex * (-sg / ((r - rc) * (r - rc)));
    *dphi = A * eps * (dbra * ex + bra * dex);
    return A * eps * bra * ex;
}

static double sw_g(const double *P, double r, double *dg)
{
    double sg = P[1], a = P[2], gm = P[4];
    double rc = a * sg;
    if (r >= rc) {
        *dg = 0.0;
        return 0.0;
    }
    double v = exp(gm * sg / (r - rc));
    *dg = v * (-gm * sg / ((r - rc) * (r - rc)));
    return v;
}

double or_sw_phi2(const double *P, double r, double *dphi) { return sw_phi2(P, r, dphi); }

double or_sw(int N, const double *r, const double *L, const double *P, double *f, double *e)
{
    double rc = P[2] * P[1];
    csr_t g = neighbors(N, 3, r, L, rc, 0, 1);
    double *F = (double *)calloc((size_t)3 * N + 1, sizeof(double));
    double *E = (double *)calloc((size_t)N + 1, sizeof(double));
    double lam = P[3], eps = P[0], c0 = P[9];
    for (int i = 0; i < N; ++i) {
        long b = g.start[i], n = g.start[i + 1] - g.start[i];
        /* two-body: each ordered pair contributes half of phi2 to e_i and the
         * full derivative to F_i (the j-side is added when visiting j). */
        for (long s = 0; s < n; ++s) {
            int j = g.idx[b + s];
            double d[3];
            min_image64(3, L, r + 3 * i, r + 3 * j, d);          /* r_i - r_j */
            double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double dphi;
            double ph = sw_phi2(P, rr, &dphi);
            E[i] += 0.5 * ph;
            for (int k = 0; k < 3; ++k) F[3 * i + k] -= dphi * d[k] / rr;
        }
        /* three-body, centre i, legs j < k */
        for (long s = 0; s < n; ++s)
            for (long t = s + 1; t < n; ++t) {
                int j = g.idx[b + s], k = g.idx[b + t];
                double u[3], w[3];
                min_image64(3, L, r + 3 * j, r + 3 * i, u);      /* r_j - r_i */
                min_image64(3, L, r + 3 * k, r + 3 * i, w);      /* r_k - r_i */
                double ru = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                double rw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
                double c = (u[0] * w[0] + u[1] * w[1] + u[2] * w[2]) / (ru * rw);
                double dgu, dgw;
                double gu = sw_g(P, ru, &dgu), gw = sw_g(P, rw, &dgw);
                double h = lam * eps * (c - c0) * (c - c0) * gu * gw;
                E[i] += h;
                double dh_dc = 2.0 * lam * eps * (c - c0) * gu * gw;
                double dh_dru = lam * eps * (c - c0) * (c - c0) * dgu * gw;
                double dh_drw = lam * eps * (c - c0) * (c - c0) * gu * dgw;
                for (int q = 0; q < 3; ++q) {
                    double dc_du = w[q] / (ru * rw) - c * u[q] / (ru * ru);
                    double dc_dw = u[q] / (ru * rw) - c * w[q] / (rw * rw);
                    double gu_q = dh_dc * dc_du + dh_dru * u[q] / ru;   /* dh/dr_j */
                    double gw_q = dh_dc * dc_dw + dh_drw * w[q] / rw;   /* dh/dr_k */
                    F[3 * j + q] -= gu_q;
                    F[3 * k + q] -= gw_q;
                    F[3 * i + q] += gu_q + gw_q;
                }
            }
    }
    double U = 0.0;
    for (int i = 0; i < N; ++i) {
        U += E[i];
        if (e) e[i] = E[i];
        if (f)
            for (int k = 0; k < 3; ++k) f[3 * i + k] = F[3 * i + k];
    }
    free(F);
    free(E);
    csr_free(&g);
    return U;
}

/* ----------------------------------------------------------------------- */
/* Dynamics (Sec. 3.3.1).                                                   */
/* ----------------------------------------------------------------------- */
enum { OR_LJ = 0, OR_SOFT = 1, OR_SW = 2 };

/* Potential parameters: LJ {eps, sigma, r_c, shifted}; SOFT {eps, alpha}
 * (+ diam); SW the 10 values above. */
static double energy_forces(int pot, int N, int dim, const double *r, const double *diam, const double *L,
                            const double *pp, double *f)
{
    if (pot == OR_LJ) return or_lj(N, r, L, pp[0], pp[1], pp[2], (int)pp[3], 1, f, NULL);
    if (pot == OR_SOFT) return or_soft(N, dim, r, diam, L, pp[0], pp[1], f, NULL);
    return or_sw(N, r, L, pp, f, NULL);
}

static double kinetic(int N, int dim, const double *v, double mass)
{
    double K = 0.0;
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < dim; ++k) K += 0.5 * mass * v[3 * i + k] * v[3 * i + k];
    return K;
}

/* Velocity-Verlet NVE (Sec. 3.3.1 "constant energy (NVE) simulation").
 * mass is in energy*time^2/length^2, so a = F / mass.  Positions are
 * wrapped into the box after every drift.  PE/KE series have nsteps+1
 * entries, entry 0 being the initial state. */
void or_nve(int N, int dim, double *r, double *v, const double *diam, const double *L, int pot,
            const double *pp, double mass, double dt, int nsteps, double *PE, double *KE)
{
    double *f = (double *)calloc((size_t)3 * N + 1, sizeof(double));
    double U = energy_forces(pot, N, dim, r, diam, L, pp, f);
    if (PE) PE[0] = U;
    if (KE) KE[0] = kinetic(N, dim, v, mass);
    for (int s = 1; s <= nsteps; ++s) {
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < dim; ++k) {
                v[3 * i + k] += 0.5 * dt * f[3 * i + k] / mass;
                r[3 * i + k] = wrap64(r[3 * i + k] + dt * v[3 * i + k], L[k]);
            }
        U = energy_forces(pot, N, dim, r, diam, L, pp, f);
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < dim; ++k) v[3 * i + k] += 0.5 * dt * f[3 * i + k] / mass;
        if (PE) PE[s] = U;
        if (KE) KE[s] = kinetic(N, dim, v, mass);
    }
    free(f);
}

/* Gradient descent (Sec. 3.3.1): r <- r + eta F(r), positions unwrapped.
 * E series has nsteps+1 entries (energy before each step, then final). */
void or_gd(int N, int dim, double *r, const double *diam, const double *L, int pot, const double *pp,
           double eta, int nsteps, double *Eser)
{
    double *f = (double *)calloc((size_t)3 * N + 1, sizeof(double));
    for (int s = 0; s < nsteps; ++s) {
        double U = energy_forces(pot, N, dim, r, diam, L, pp, f);
        if (Eser) Eser[s] = U;
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < dim; ++k) r[3 * i + k] += eta * f[3 * i + k];
    }
    double U = energy_forces(pot, N, dim, r, diam, L, pp, f);
    if (Eser) Eser[nsteps] = U;
    free(f);
}

/* Flocking energy model (Sec. 4.3 and its appendix): boids with positions
 * R_i in a periodic square and headings theta_i, N(theta) = (cos, sin).
 * rho(r; Rc) = (1 - r/Rc)^a / a for r < Rc (a = 2), else 0.  With R_ij the
 * nearest-image displacement R_i - R_j and each unordered pair once:
 *   E_align  = sum_{i<j} J_al rho(r_ij; R_al) (1 - N_i.N_j)^2
 *              (no gradient through the displacement: it turns the boids)
 *   E_avoid  = sum_{i<j} J_av rho(r_ij; R_av)
 *   E_coh    = sum_i J_co/2 (1 - u_i.N_i)^2,  u_i the unit vector towards
 *              the mean of R_j - R_i over the boids j within R_co (no term
 *              without neighbours; no gradient through the displacements)
 *   E_obst   = sum_i sum_o J_ob rho(|R_o - R_i|; D_o) (1 + N_i.w_io)^2,
 *              w_io the unit vector from boid i to obstacle o (disk of
 *              radius D_o), smallest when the boid faces away
 * Predators p (position, heading), a two-player game: the boids add
 *   E_flee   = sum_i sum_p J_fl rho(|R_p - R_i|; R_fl) (1 + N_i.w_ip)^2
 * (the obstacle form, gradient in the boid's variables), and the predators
 * minimise
 *   E_chase  = sum_p J_ch/2 (1 - u_p.N_p)^2, u_p towards the mean offset of
 *              the boids within R_ch (the cohesion form), plus E_obst of
 *              the predators (gradient in the predator's variables).
 * Forward Euler for both: R += dt (v N - dE/dR), theta -= dt dE/dtheta,
 * positions wrapped; speeds v (boids) and v_p (predators).  Sprints (the
 * paper lets predators sprint now and then without saying how): in step s
 * (counted from 0 in each run) the predators swim at v_p * f_sp when
 * P_sp > 0 and s mod P_sp < n_sp.
 * prm = {J_al, R_al, J_av, R_av, J_co, R_co, J_ob, a, v, J_fl, R_fl, J_ch,
 *        R_ch, v_p, P_sp, n_sp, f_sp};  obs: n_obs x 3 (x, y, D);
 *        pred: n_p x 3 (x, y, theta).
 * Brute force over all pairs. */
static double nearest1(double t, double L) { return t - L * nearbyint(t / L); }
static double rho_cut(double r, double Rc, double a) { return r < Rc ? pow(1.0 - r / Rc, a) / a : 0.0; }
static double rho_cut_d(double r, double Rc, double a) { return r < Rc ? -pow(1.0 - r / Rc, a - 1.0) / Rc : 0.0; }

/* The obstacle form J rho(r; D) (1 + N.w)^2 of an agent at (x, y) with
 * heading th against a disk at (ox, oy) of radius D; adds its energy and its
 * gradient in the agent's variables. */
static double disk_term(double x, double y, double th, double ox, double oy, double D, double J, double a,
                        const double *L, double *gx, double *gy, double *gth)
{
    const double dx = nearest1(ox - x, L[0]), dy = nearest1(oy - y, L[1]);
    const double r = sqrt(dx * dx + dy * dy);
    if (!(r > 0.0 && r < D)) return 0.0;
    const double wx = dx / r, wy = dy / r;
    const double nx = cos(th), ny = sin(th);
    const double nw = nx * wx + ny * wy, q = 1.0 + nw;
    const double rh = rho_cut(r, D, a), rhd = rho_cut_d(r, D, a);
    *gth += 2.0 * J * rh * q * (-sin(th) * wx + cos(th) * wy);
    /* r depends on the agent as dr/dR = -w; w as dw/dR = -(I - w w^T)/r */
    *gx += J * (rhd * (-wx) * q * q + rh * 2.0 * q * (-(nx - nw * wx) / r));
    *gy += J * (rhd * (-wy) * q * q + rh * 2.0 * q * (-(ny - nw * wy) / r));
    return J * rh * q * q;
}

/* The cohesion form J/2 (1 - u.N)^2 from the summed offsets (cx, cy) of n
 * agents; adds its heading gradient. */
static double heading_term(double cx, double cy, int n, double th, double J, double *gth)
{
    if (n <= 0) return 0.0;
    cx /= n;
    cy /= n;
    const double m = sqrt(cx * cx + cy * cy);
    if (!(m > 0.0)) return 0.0;
    const double ux = cx / m, uy = cy / m;
    const double un = ux * cos(th) + uy * sin(th);
    const double up = -ux * sin(th) + uy * cos(th);   /* u . dN/dtheta */
    *gth += -J * (1.0 - un) * up;
    return 0.5 * J * (1.0 - un) * (1.0 - un);
}

double or_flock_grad(int N, const double *R, const double *th, const double *L, const double *prm, int n_obs,
                     const double *obs, int n_p, const double *pred, double *gR, double *gth, double *gP,
                     double *parts)
{
    const double Jal = prm[0], Ral = prm[1], Jav = prm[2], Rav = prm[3], Jco = prm[4], Rco = prm[5], Job = prm[6],
                 a = prm[7], Jfl = prm[9], Rfl = prm[10], Jch = prm[11], Rch = prm[12];
    double Eal = 0.0, Eav = 0.0, Eco = 0.0, Eob = 0.0, Efl = 0.0, Ech = 0.0;
    for (int i = 0; i < 2 * N; ++i) gR[i] = 0.0;
    for (int i = 0; i < N; ++i) gth[i] = 0.0;
    for (int i = 0; i < 3 * n_p; ++i) gP[i] = 0.0;
    for (int i = 0; i < N; ++i) {
        double cx = 0.0, cy = 0.0;
        int nco = 0;
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            double d[2];
            for (int k = 0; k < 2; ++k) d[k] = nearest1(R[2 * i + k] - R[2 * j + k], L[k]);
            const double r = sqrt(d[0] * d[0] + d[1] * d[1]);
            const double c = cos(th[i] - th[j]);
            /* alignment: d/dtheta_i of rho (1 - c)^2 = 2 rho (1 - c) sin(theta_i - theta_j) */
            const double ral = rho_cut(r, Ral, a);
            if (j > i) Eal += Jal * ral * (1.0 - c) * (1.0 - c);
            gth[i] += 2.0 * Jal * ral * (1.0 - c) * sin(th[i] - th[j]);
            if (j > i) Eav += Jav * rho_cut(r, Rav, a);
            if (r > 0.0 && r < Rav) {
                const double g = Jav * rho_cut_d(r, Rav, a) / r;
                gR[2 * i] += g * d[0];
                gR[2 * i + 1] += g * d[1];
            }
            if (r < Rco) {
                cx -= d[0];
                cy -= d[1];
                nco += 1;
            }
        }
        Eco += heading_term(cx, cy, nco, th[i], Jco, &gth[i]);
        for (int o = 0; o < n_obs; ++o)
            Eob += disk_term(R[2 * i], R[2 * i + 1], th[i], obs[3 * o], obs[3 * o + 1], obs[3 * o + 2], Job, a, L,
                             &gR[2 * i], &gR[2 * i + 1], &gth[i]);
        for (int p = 0; p < n_p; ++p)
            Efl += disk_term(R[2 * i], R[2 * i + 1], th[i], pred[3 * p], pred[3 * p + 1], Rfl, Jfl, a, L, &gR[2 * i],
                             &gR[2 * i + 1], &gth[i]);
    }
    for (int p = 0; p < n_p; ++p) {
        double cx = 0.0, cy = 0.0;
        int n = 0;
        for (int i = 0; i < N; ++i) {
            const double dx = nearest1(R[2 * i] - pred[3 * p], L[0]), dy = nearest1(R[2 * i + 1] - pred[3 * p + 1], L[1]);
            if (sqrt(dx * dx + dy * dy) < Rch) {
                cx += dx;
                cy += dy;
                n += 1;
            }
        }
        Ech += heading_term(cx, cy, n, pred[3 * p + 2], Jch, &gP[3 * p + 2]);
        for (int o = 0; o < n_obs; ++o)
            Eob += disk_term(pred[3 * p], pred[3 * p + 1], pred[3 * p + 2], obs[3 * o], obs[3 * o + 1], obs[3 * o + 2],
                             Job, a, L, &gP[3 * p], &gP[3 * p + 1], &gP[3 * p + 2]);
    }
    if (parts) {
        parts[0] = Eal;
        parts[1] = Eav;
        parts[2] = Eco;
        parts[3] = Eob;
        parts[4] = Efl;
        parts[5] = Ech;
    }
    return Eal + Eav + Eco + Eob + Efl + Ech;
}

void or_flock_run(int N, double *R, double *th, const double *L, const double *prm, int n_obs, const double *obs,
                  int n_p, double *pred, double dt, int nsteps, double *Eser)
{
    double *gR = (double *)calloc((size_t)2 * N + 1, sizeof(double));
    double *gth = (double *)calloc((size_t)N + 1, sizeof(double));
    double *gP = (double *)calloc((size_t)3 * n_p + 1, sizeof(double));
    const double v = prm[8];
    const long P_sp = (long)prm[14], n_sp = (long)prm[15];
    for (int s = 0; s < nsteps; ++s) {
        const double vp = (P_sp > 0 && s % P_sp < n_sp) ? prm[13] * prm[16] : prm[13];
        const double E = or_flock_grad(N, R, th, L, prm, n_obs, obs, n_p, pred, gR, gth, gP, NULL);
        if (Eser) Eser[s] = E;
        for (int i = 0; i < N; ++i) {
            R[2 * i] = wrap64(R[2 * i] + dt * (v * cos(th[i]) - gR[2 * i]), L[0]);
            R[2 * i + 1] = wrap64(R[2 * i + 1] + dt * (v * sin(th[i]) - gR[2 * i + 1]), L[1]);
            th[i] -= dt * gth[i];
        }
        for (int p = 0; p < n_p; ++p) {
            const double tp = pred[3 * p + 2];
            pred[3 * p] = wrap64(pred[3 * p] + dt * (vp * cos(tp) - gP[3 * p]), L[0]);
            pred[3 * p + 1] = wrap64(pred[3 * p + 1] + dt * (vp * sin(tp) - gP[3 * p + 1]), L[1]);
            pred[3 * p + 2] = tp - dt * gP[3 * p + 2];
        }
    }
    if (Eser) Eser[nsteps] = or_flock_grad(N, R, th, L, prm, n_obs, obs, n_p, pred, gR, gth, gP, NULL);
    free(gP);
    free(gth);
    free(gR);
}

/* Nose-Hoover chain NVT (Sec. 3.3.1 lists Nose-Hoover constant-temperature
 * simulation, citing Martyna, Klein, Tuckerman 1992).  One step is the
 * symmetric Trotter splitting
 *     chain(dt/2) . kick(dt/2) . drift(dt) . kick(dt/2) . chain(dt/2)
 * (velocity Verlet between two thermostat half-steps).  The chain half-step
 * is the sweep of Martyna, Tuckerman, Tobias, Klein (1996) with one
 * sub-step, on thermostat velocities w_k = p_k/Q_k with "forces"
 *     G_1 = (2K - g kT)/Q_1,   G_k = (Q_{k-1} w_{k-1}^2 - kT)/Q_k  (k > 1):
 *   w_M += dt/4 G_M
 *   k = M-1..1:  w_k *= exp(-dt/8 w_{k+1}); w_k += dt/4 G_k; w_k *= exp(-dt/8 w_{k+1})
 *   s = exp(-dt/2 w_1);  v *= s;  K *= s^2;  xi_k += dt/2 w_k (all k)
 *   k = 1..M-1:  w_k *= exp(-dt/8 w_{k+1}); w_k += dt/4 G_k; w_k *= exp(-dt/8 w_{k+1})
 *   w_M += dt/4 G_M
 * g = dim N degrees of freedom; Q_1 = g kT tau^2, Q_k = kT tau^2.  The
 * conserved quantity is H' = K + U + sum_k Q_k w_k^2 / 2 + g kT xi_1 +
 * kT sum_{k>1} xi_k.  therm (2M, in/out) holds (xi_1..xi_M, w_1..w_M).
 * PE, KE, Hext: nsteps+1 entries, entry 0 the initial state. */
static void nhc_half(int M, double *xi, double *w, const double *Q, double gkT, double kT, double dt, double *K,
                     double *scale)
{
    const double h4 = 0.25 * dt, h8 = 0.125 * dt;
    double G;
    G = (M > 1) ? (Q[M - 2] * w[M - 2] * w[M - 2] - kT) / Q[M - 1] : (2.0 * (*K) - gkT) / Q[0];
    w[M - 1] += h4 * G;
    for (int k = M - 2; k >= 0; --k) {
        const double e = exp(-h8 * w[k + 1]);
        w[k] *= e;
        G = (k == 0) ? (2.0 * (*K) - gkT) / Q[0] : (Q[k - 1] * w[k - 1] * w[k - 1] - kT) / Q[k];
        w[k] += h4 * G;
        w[k] *= e;
    }
    const double s = exp(-0.5 * dt * w[0]);
    *scale = s;
    *K *= s * s;
    for (int k = 0; k < M; ++k) xi[k] += 0.5 * dt * w[k];
    for (int k = 0; k < M - 1; ++k) {
        const double e = exp(-h8 * w[k + 1]);
        w[k] *= e;
        G = (k == 0) ? (2.0 * (*K) - gkT) / Q[0] : (Q[k - 1] * w[k - 1] * w[k - 1] - kT) / Q[k];
        w[k] += h4 * G;
        w[k] *= e;
    }
    G = (M > 1) ? (Q[M - 2] * w[M - 2] * w[M - 2] - kT) / Q[M - 1] : (2.0 * (*K) - gkT) / Q[0];
    w[M - 1] += h4 * G;
}

static double nhc_energy(int M, const double *xi, const double *w, const double *Q, double gkT, double kT)
{
    double e = 0.0;
    for (int k = 0; k < M; ++k) e += 0.5 * Q[k] * w[k] * w[k];
    e += gkT * xi[0];
    for (int k = 1; k < M; ++k) e += kT * xi[k];
    return e;
}

void or_nhc(int N, int dim, double *r, double *v, const double *diam, const double *L, int pot, const double *pp,
            double mass, double dt, double kT, double tau, int M, int nsteps, double *therm, double *PE, double *KE,
            double *Hext)
{
    double *f = (double *)calloc((size_t)3 * N + 1, sizeof(double));
    double Q[16], *xi = therm, *w = therm + M;
    const double g = (double)dim * N, gkT = g * kT;
    Q[0] = gkT * tau * tau;
    for (int k = 1; k < M; ++k) Q[k] = kT * tau * tau;
    double U = energy_forces(pot, N, dim, r, diam, L, pp, f);
    double K = kinetic(N, dim, v, mass);
    if (PE) PE[0] = U;
    if (KE) KE[0] = K;
    if (Hext) Hext[0] = K + U + nhc_energy(M, xi, w, Q, gkT, kT);
    for (int s = 1; s <= nsteps; ++s) {
        double sc;
        nhc_half(M, xi, w, Q, gkT, kT, dt, &K, &sc);
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < dim; ++k) {
                v[3 * i + k] = v[3 * i + k] * sc + 0.5 * dt * f[3 * i + k] / mass;
                r[3 * i + k] = wrap64(r[3 * i + k] + dt * v[3 * i + k], L[k]);
            }
        U = energy_forces(pot, N, dim, r, diam, L, pp, f);
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < dim; ++k) v[3 * i + k] += 0.5 * dt * f[3 * i + k] / mass;
        K = kinetic(N, dim, v, mass);
        nhc_half(M, xi, w, Q, gkT, kT, dt, &K, &sc);
        for (int i = 0; i < 3 * N; ++i) v[i] *= sc;
        if (PE) PE[s] = U;
        if (KE) KE[s] = K;
        if (Hext) Hext[s] = K + U + nhc_energy(M, xi, w, Q, gkT, kT);
    }
    free(f);
}

/* FIRE, the Fast Inertial Relaxation Engine (Bitzek, Koskinen, Gahler,
 * Moseler, Gumbsch, PRL 97, 170201 (2006); Sec. 3.3.1 lists it among the
 * minimisers), unit mass, unwrapped coordinates as in GD.  One step, in the
 * order of the published algorithm:
 *   MD step (velocity Verlet):  v += dt/2 F;  r += dt v;  F = F(r);  v += dt/2 F
 *   P = F . v over all degrees of freedom
 *   mixing:  v = (1 - alpha) v + alpha |v| F/|F|   (no F term when |F| = 0)
 *   P > 0:   npos += 1; if npos > n_min: dt = min(dt f_inc, dt_max), alpha *= f_alpha
 *   P <= 0:  dt *= f_dec; v = 0; alpha = alpha_start; npos = 0
 * prm = {dt_start, dt_max, f_inc, f_dec, alpha_start, f_alpha, n_min}.
 * Starts from rest.  Eser (nsteps+1, may be NULL): U before every step and
 * after the last; dtser (nsteps, may be NULL): dt after each step; v (3N,
 * may be NULL) receives the final velocities; st_out (3, may be NULL):
 * final dt, alpha, npos. */
void or_fire(int N, int dim, double *r, const double *diam, const double *L, int pot, const double *pp,
             const double *prm, int nsteps, double *Eser, double *dtser, double *v_out, double *st_out)
{
    double *f = (double *)calloc((size_t)3 * N + 1, sizeof(double));
    double *v = (double *)calloc((size_t)3 * N + 1, sizeof(double));
    double dt = prm[0], alpha = prm[4];
    const double dt_max = prm[1], f_inc = prm[2], f_dec = prm[3], alpha_start = prm[4], f_alpha = prm[5];
    const int n_min = (int)prm[6];
    int npos = 0;
    double U = energy_forces(pot, N, dim, r, diam, L, pp, f);
    for (int s = 0; s < nsteps; ++s) {
        if (Eser) Eser[s] = U;
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < dim; ++k) {
                v[3 * i + k] += 0.5 * dt * f[3 * i + k];
                r[3 * i + k] += dt * v[3 * i + k];
            }
        U = energy_forces(pot, N, dim, r, diam, L, pp, f);
        double P = 0.0, vv = 0.0, ff = 0.0;
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < dim; ++k) {
                v[3 * i + k] += 0.5 * dt * f[3 * i + k];
                P += f[3 * i + k] * v[3 * i + k];
                vv += v[3 * i + k] * v[3 * i + k];
                ff += f[3 * i + k] * f[3 * i + k];
            }
        const double c = ff > 0.0 ? alpha * sqrt(vv) / sqrt(ff) : 0.0;
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < dim; ++k) v[3 * i + k] = (1.0 - alpha) * v[3 * i + k] + c * f[3 * i + k];
        if (P > 0.0) {
            npos += 1;
            if (npos > n_min) {
                dt = fmin(dt * f_inc, dt_max);
                alpha *= f_alpha;
            }
        } else {
            dt *= f_dec;
            for (int i = 0; i < 3 * N; ++i) v[i] = 0.0;
            alpha = alpha_start;
            npos = 0;
        }
        if (dtser) dtser[s] = dt;
    }
    if (Eser) Eser[nsteps] = U;
    if (v_out)
        for (int i = 0; i < 3 * N; ++i) v_out[i] = v[i];
    if (st_out) {
        st_out[0] = dt;
        st_out[1] = alpha;
        st_out[2] = (double)npos;
    }
    free(v);
    free(f);
}

/* ----------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11), from its published definition.  One round maps
 * counter (c0,c1,c2,c3) and key (k0,k1) to
 *     (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
 * with M0 = 0xD2511F53, M1 = 0xCD9E8D57 (32x32->64-bit products); between
 * rounds the key is bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85. */
/* ----------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out)
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Standard normals for particle i at step s: one Philox block with counter
 * {i, s, stream, 0} and key {seed_lo, seed_hi}; uniforms
 * u = (x >> 8 + 1) 2^-24 in (0, 1]; Box-Muller pairs (u0,u1), (u2,u3):
 * z0 = sqrt(-2 ln u0) cos(2 pi u1), z1 = sqrt(-2 ln u0) sin(2 pi u1), z2 likewise. */
void or_normal3(uint32_t i, uint32_t s, uint32_t stream, uint64_t seed, double *z)
{
    uint32_t ctr[4] = {i, s, stream, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    double u[4];
    for (int k = 0; k < 4; ++k) u[k] = ((double)(x[k] >> 8) + 1.0) * (1.0 / 16777216.0);
    double ra = sqrt(-2.0 * log(u[0])), rb = sqrt(-2.0 * log(u[2]));
    z[0] = ra * cos(2.0 * M_PI * u[1]);
    z[1] = ra * sin(2.0 * M_PI * u[1]);
    z[2] = rb * cos(2.0 * M_PI * u[3]);
}

/* BAOAB Langevin (Sec. 3.3.1 "Langevin ... at constant temperature"):
 *   B: v += dt/2 F/m;  A: r += dt/2 v;  O: v = c1 v + c2 z;  A: r += dt/2 v;
 *   (forces)           B: v += dt/2 F/m
 * c1 = exp(-gamma dt), c2 = sqrt((1 - c1^2) kT / m).  z from or_normal3
 * with counter (i, step, 0).  Positions wrapped after the second A. */
void or_langevin(int N, double *r, double *v, const double *L, int pot, const double *pp, double mass,
                 double dt, double gamma, double kT, uint64_t seed, int step0, int nsteps, double *PE, double *KE)
{
    double *f = (double *)calloc((size_t)3 * N + 1, sizeof(double));
    energy_forces(pot, N, 3, r, NULL, L, pp, f);
    double c1 = exp(-gamma * dt), c2 = sqrt((1.0 - c1 * c1) * kT / mass);
    for (int s = 0; s < nsteps; ++s) {
        for (int i = 0; i < N; ++i) {
            double z[3];
            or_normal3((uint32_t)i, (uint32_t)(step0 + s), 0u, seed, z);
            for (int k = 0; k < 3; ++k) {
                double vk = v[3 * i + k] + 0.5 * dt * f[3 * i + k] / mass;
                double rk = r[3 * i + k] + 0.5 * dt * vk;
                vk = c1 * vk + c2 * z[k];
                rk = rk + 0.5 * dt * vk;
                v[3 * i + k] = vk;
                r[3 * i + k] = wrap64(rk, L[k]);
            }
        }
        double U = energy_forces(pot, N, 3, r, NULL, L, pp, f);
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < 3; ++k) v[3 * i + k] += 0.5 * dt * f[3 * i + k] / mass;
        if (PE) PE[s] = U;
        if (KE) KE[s] = kinetic(N, 3, v, mass);
    }
    free(f);
}

/* ----------------------------------------------------------------------- */
/* Differentiating the final energy of a minimisation (Sec. 4.2, App. A).
 *
 * Bidisperse 2-D disks: the first N/2 have diameter D, the rest 1; the box
 * keeps packing fraction phi:  L(D) = sqrt((N/2) pi (1 + D^2) / (4 phi)).
 * r_0 = L(D) s_0, r_{t+1} = r_t + eta F(r_t; D) for t < T (unwrapped),
 * E_final(D) = U(r_T; D).  Reverse mode (hand-written):
 *   lambda_T = grad U(r_T)
 *   dE/dD    = dU/dD|_{r_T}
 *   for t = T-1..0:  dE/dD += eta lambda_{t+1} . dF/dD|_{r_t}
 *                    lambda_t = lambda_{t+1} - eta H(r_t) lambda_{t+1}
 *   dE/dD += lambda_0 . s_0 L'(D)
 * H is the Hessian of U; the minimum image carries d_ij = r_i - r_j - n_ij L
 * with piecewise-constant n_ij, so dd_ij/dD = -n_ij L'(D).  All states are
 * kept (no checkpointing).  Returns E_final; *dEdD receives the derivative.
 * Energies use u = (eps/alpha)(1 - r/s)^alpha.                           */
/* ----------------------------------------------------------------------- */
typedef struct {
    double u, ur, urr, us, urs;
} soft_terms;

static soft_terms soft_pair_terms(double r, double s, double eps, double alpha)
{
    soft_terms t;
    double x = 1.0 - r / s;
    t.u = eps / alpha * pow(x, alpha);
    t.ur = -eps / s * pow(x, alpha - 1.0);
    t.urr = eps / (s * s) * (alpha - 1.0) * pow(x, alpha - 2.0);
    t.us = eps * pow(x, alpha - 1.0) * r / (s * s);
    t.urs = eps / (s * s) * (pow(x, alpha - 1.0) - (alpha - 1.0) * pow(x, alpha - 2.0) * r / s);
    return t;
}

double or_packing_box(int N, double D, double phi)
{
    return sqrt((N / 2) * M_PI * (D * D + 1.0) / 4.0 / phi);
}

/* dsigma_ij/dD: 1 for two large... i.e. both of species A (diameter D),
 * 1/2 for a mixed pair, 0 for two unit disks. */
static double dsig(int N, int i, int j)
{
    int a = i < N / 2, b = j < N / 2;
    return 0.5 * (double)(a + b);
}

double or_gd_adjoint(int N, const double *s0, double D, double phi, double eps, double alpha, double eta,
                     int T, double *dEdD, double *r_final)
{
    double L1 = or_packing_box(N, D, phi);
    double Lp = (N / 2) * M_PI * D / (4.0 * phi * L1);      /* L'(D) */
    double L[3] = {L1, L1, 1.0};
    double *diam = (double *)malloc(sizeof(double) * (size_t)N);
    for (int i = 0; i < N; ++i) diam[i] = i < N / 2 ? D : 1.0;
    size_t st = (size_t)3 * N;
    double *R = (double *)calloc(st * (size_t)(T + 1), sizeof(double));
    double *f = (double *)calloc(st, sizeof(double));
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < 2; ++k) R[3 * i + k] = L1 * s0[2 * i + k];
    for (int t = 0; t < T; ++t) {
        or_soft(N, 2, R + st * t, diam, L, eps, alpha, f, NULL);
        for (size_t q = 0; q < st; ++q) R[st * (t + 1) + q] = R[st * t + q] + eta * f[q];
    }
    double *rT = R + st * T;
    double E = or_soft(N, 2, rT, diam, L, eps, alpha, f, NULL);
    double *lam = (double *)calloc(st, sizeof(double));
    double *hl = (double *)calloc(st, sizeof(double));
    for (size_t q = 0; q < st; ++q) lam[q] = -f[q];
    double dmax = D > 1.0 ? D : 1.0;
    double g = 0.0;
    /* dU/dD at r_T (each unordered pair once) */
    {
        csr_t nb = neighbors(N, 2, rT, L, dmax, 0, 1);
        for (int i = 0; i < N; ++i)
            for (long s = nb.start[i]; s < nb.start[i + 1]; ++s) {
                int j = nb.idx[s];
                if (j <= i) continue;
                double d[3], n[3];
                min_image64(2, L, rT + 3 * i, rT + 3 * j, d);
                image_index64(2, L, rT + 3 * i, rT + 3 * j, n);
                double rr = sqrt(d[0] * d[0] + d[1] * d[1]);
                double sg = 0.5 * (diam[i] + diam[j]);
                if (rr >= sg) continue;
                soft_terms tt = soft_pair_terms(rr, sg, eps, alpha);
                g += tt.us * dsig(N, i, j);
                for (int k = 0; k < 2; ++k) g += tt.ur * d[k] / rr * (-n[k] * Lp);
            }
        csr_free(&nb);
    }
    for (int t = T - 1; t >= 0; --t) {
        const double *rt = R + st * t;
        csr_t nb = neighbors(N, 2, rt, L, dmax, 0, 1);
        memset(hl, 0, st * sizeof(double));
        double acc = 0.0;
        for (int i = 0; i < N; ++i)
            for (long s = nb.start[i]; s < nb.start[i + 1]; ++s) {
                int j = nb.idx[s];
                double d[3], n[3];
                min_image64(2, L, rt + 3 * i, rt + 3 * j, d);
                image_index64(2, L, rt + 3 * i, rt + 3 * j, n);
                double rr = sqrt(d[0] * d[0] + d[1] * d[1]);
                double sg = 0.5 * (diam[i] + diam[j]);
                if (rr >= sg) continue;
                soft_terms tt = soft_pair_terms(rr, sg, eps, alpha);
                double e[2] = {d[0] / rr, d[1] / rr};
                /* pair Hessian h = urr e e^T + ur/r (I - e e^T) */
                double h[2][2];
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        h[a][b] = tt.urr * e[a] * e[b] + tt.ur / rr * ((a == b) - e[a] * e[b]);
                /* (H lambda)_i = sum_j h (lambda_i - lambda_j) */
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) hl[3 * i + a] += h[a][b] * (lam[3 * i + b] - lam[3 * j + b]);
                /* dF_i/dD = -[urs dsig e + h dd/dD],  dd/dD = -n L' */
                double ds = dsig(N, i, j);
                for (int a = 0; a < 2; ++a) {
                    double dFa = -(tt.urs * ds * e[a]);
                    for (int b = 0; b < 2; ++b) dFa -= h[a][b] * (-n[b] * Lp);
                    acc += lam[3 * i + a] * dFa;
                }
            }
        csr_free(&nb);
        g += eta * acc;
        for (size_t q = 0; q < st; ++q) lam[q] -= eta * hl[q];
    }
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < 2; ++k) g += lam[3 * i + k] * s0[2 * i + k] * Lp;
    if (dEdD) *dEdD = g;
    if (r_final)
        for (size_t q = 0; q < st; ++q) r_final[q] = rT[q];
    free(hl);
    free(lam);
    free(f);
    free(R);
    free(diam);
    return E;
}

/* E_final(D) alone (forward only), for finite differences. */
double or_gd_final_energy(int N, const double *s0, double D, double phi, double eps, double alpha, double eta, int T)
{
    double L1 = or_packing_box(N, D, phi);
    double L[3] = {L1, L1, 1.0};
    double *diam = (double *)malloc(sizeof(double) * (size_t)N);
    for (int i = 0; i < N; ++i) diam[i] = i < N / 2 ? D : 1.0;
    double *r = (double *)calloc((size_t)3 * N, sizeof(double));
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < 2; ++k) r[3 * i + k] = L1 * s0[2 * i + k];
    double pp[2] = {eps, alpha};
    or_gd(N, 2, r, diam, L, OR_SOFT, pp, eta, T, NULL);
    double *f = (double *)calloc((size_t)3 * N, sizeof(double));
    double E = or_soft(N, 2, r, diam, L, eps, alpha, f, NULL);
    free(f);
    free(r);
    free(diam);
    return E;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
