/*
 * lsm_oracle.c -- plain FP64 CPU oracle of the lattice-spring method.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or call
 * this file: only the test suite, the smoke check and the bench's CPU-baseline
 * leg use it. It shares no code with the CUDA library.
 *
 * What it computes, step by step in the paper's order and notation
 * (arXiv 2201.04565, "ImageMech"):
 *   - potential, Eq. 1:  U = sum_springs 1/2 k (r - r0)^2 (1 - Xi(r - rc))
 *   - force, Eq. 2:      F_i = - sum_j k (r_ij - r0) (r_i - r_j)/r_ij (1 - Xi)
 *   - velocity Verlet in the half-step-velocity form, Eqs. 3-5 (Section 2.2)
 *   - irreversible breakage: a spring whose length exceeds rc is broken for
 *     good and gives no force from the step in which the test fires on
 *     (Section 2.3 force listing; Section 4 on keeping broken springs)
 *   - displacement-controlled loading of the boundary particles along x
 *     (Sections 2.3 and 3.1)
 *   - virial stress, Eq. 7 (xx component over the reference box)
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - lattice: square (2D) / cubic (3D) with first and second neighbours;
 *     r0 = |offset| a, k from a per-phase-pair table (times k2_ratio for the
 *     diagonal shell), rc = r0 (1 + eps_c) from a per-phase-pair table;
 *   - the Heaviside switch: a spring is intact while r^2 <= rc^2 (strict '>'
 *     breaks, as in the force listing), tested on the squared length;
 *   - damping: viscous force -gamma * vh on every free component, applied at
 *     force time: a = (F - gamma vh) / m;
 *   - loading: an increment remaps the x coordinate of every particle affinely
 *     about the specimen centre xc (load_mode 0) or moves only the grips
 *     (load_mode 1); prescribed grip components are then set exactly to
 *     X + eps (X - xc) with zero velocity;
 *   - grips are the particles in the first and last image column; in roller
 *     mode only their x component is prescribed, in clamped mode all are.
 *
 * Arithmetic is plain IEEE double, compiled with -ffp-contract=off so that
 * no multiply-add is fused. Summation order is the canonical spring order:
 * springs sorted by (i, j) with i < j.
 *
 * Layout: component-major arrays, component c of particle p at [c*n + p].
 *
 * Threads (orc_set_threads, OpenMP when compiled with -fopenmp): the spring
 * pass is then split into a per-spring loop (break test and force, stored
 * per spring) and a per-particle loop that adds each particle's springs in
 * ascending spring order (acc + f as the lower endpoint, acc - f as the
 * upper one, from +0). Every particle receives the same operations on the
 * same operands in the same order as in the sequential scatter, so the
 * result is bit-identical to the single-threaded pass; only the host time
 * changes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_ENOTCONV -4

typedef struct orc {
    int dim;
    int64_t n, m;
    double *X, *x, *v, *a, *F; /* [dim*n] */
    double *mass;              /* [n] */
    uint8_t *fix;              /* [dim*n] 1 = prescribed component */
    uint8_t *grip;             /* [n] 0 interior, 1 left grip, 2 right grip */
    int32_t *si, *sj;          /* [m] endpoints, si < sj, canonical order */
    double *k, *r0, *rc2;      /* [m] */
    uint8_t *broken;           /* [m] */
    int64_t *brk_step;         /* [m] index of the step in which it broke, or -1 */
    double dt, gamma, xc, omega, grip_area, eps;
    int load_mode;
    int64_t step, first_break;
    int rate_on;               /* constant strain-rate loading (orc_set_strain_rate) */
    double rate_eps0, rate_dt; /* strain when the rate was set, rate * dt */
    int64_t rate_step0;        /* step count when the rate was set */
    int nthreads;              /* > 1: the threaded spring pass below */
    int64_t *row, *inc;        /* [n+1], [2m]: springs of each particle, ascending, (s << 1) | upper */
    double *fs;                /* [dim*m] force of each spring on its lower endpoint */
} orc;

void orc_forces(const orc *o, const double *xs, double *F, double *U, double *W);
static void orc_init_accel(orc *o);
static orc *orc_build_tri(int nx, int ny, const uint8_t *phase, int nphase, const double *k_tab,
                          const double *epsc_tab, const double *mass_tab, double a, double dt,
                          double gamma, int grip_mode, int load_mode);

void orc_free(orc *o)
{
    if (!o) return;
    free(o->X); free(o->x); free(o->v); free(o->a); free(o->F);
    free(o->mass); free(o->fix); free(o->grip);
    free(o->si); free(o->sj); free(o->k); free(o->r0); free(o->rc2);
    free(o->broken); free(o->brk_step);
    free(o->row); free(o->inc); free(o->fs);
    free(o);
}

static orc *orc_alloc(int dim, int64_t n, int64_t m)
{
    orc *o = (orc *)calloc(1, sizeof(orc));
    if (!o) return NULL;
    o->dim = dim; o->n = n; o->m = m;
    size_t dn = (size_t)dim * (size_t)(n > 0 ? n : 1);
    size_t mm = (size_t)(m > 0 ? m : 1);
    o->X = calloc(dn, sizeof(double)); o->x = calloc(dn, sizeof(double));
    o->v = calloc(dn, sizeof(double)); o->a = calloc(dn, sizeof(double));
    o->F = calloc(dn, sizeof(double));
    o->mass = calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    o->fix = calloc(dn, 1); o->grip = calloc((size_t)(n > 0 ? n : 1), 1);
    o->si = calloc(mm, sizeof(int32_t)); o->sj = calloc(mm, sizeof(int32_t));
    o->k = calloc(mm, sizeof(double)); o->r0 = calloc(mm, sizeof(double));
    o->rc2 = calloc(mm, sizeof(double));
    o->broken = calloc(mm, 1); o->brk_step = calloc(mm, sizeof(int64_t));
    if (!o->X || !o->x || !o->v || !o->a || !o->F || !o->mass || !o->fix || !o->grip ||
        !o->si || !o->sj || !o->k || !o->r0 || !o->rc2 || !o->broken || !o->brk_step) {
        orc_free(o);
        return NULL;
    }
    for (int64_t s = 0; s < m; s++) o->brk_step[s] = -1;
    o->first_break = -1;
    return o;
}

/* ---------------------------------------------------------------- build -- */

/* Forward neighbour offsets (dx, dy, dz, shell). Shell 1 = first neighbours
 * (|offset| = 1), shell 2 = second neighbours (|offset| = sqrt 2). Each
 * unordered pair of lattice sites is reached exactly once from its lower
 * raster-order site. */
static const int OFF2[4][4] = {{1, 0, 0, 1}, {0, 1, 0, 1}, {1, 1, 0, 2}, {-1, 1, 0, 2}};
static const int OFF3[9][4] = {{1, 0, 0, 1},  {0, 1, 0, 1},  {0, 0, 1, 1},
                               {1, 1, 0, 2},  {-1, 1, 0, 2}, {1, 0, 1, 2},
                               {-1, 0, 1, 2}, {0, 1, 1, 2},  {0, -1, 1, 2}};

/* Image -> particles and springs (the paper's Img2Particle step, on a square
 * or cubic lattice; lattice 1 selects the triangular packing below). phase: nx*ny*nz bytes, x fastest; 0 = void, 1..nphase.
 * k_tab, epsc_tab: nphase*nphase, row-major, indexed (phase_i-1, phase_j-1).
 * mass_tab: nphase. grip_mode 0 = roller (x prescribed), 1 = clamped. */
orc *orc_build_image(int dim, int nx, int ny, int nz, const uint8_t *phase, int nphase,
                     const double *k_tab, const double *epsc_tab, const double *mass_tab,
                     double k2_ratio, double a, double dt, double gamma, int grip_mode,
                     int load_mode, int lattice)
{
    if (lattice == 1) {
        if (dim != 2) return NULL;
        return orc_build_tri(nx, ny, phase, nphase, k_tab, epsc_tab, mass_tab, a, dt, gamma, grip_mode,
                             load_mode);
    }
    if (lattice != 0) return NULL;
    if (dim != 2 && dim != 3) return NULL;
    if (dim == 2) nz = 1;
    if (nx < 2 || ny < 1 || nz < 1 || nphase < 1 || !phase || !k_tab || !epsc_tab) return NULL;
    int64_t nvox = (int64_t)nx * ny * nz;
    int64_t *idx = (int64_t *)malloc((size_t)nvox * sizeof(int64_t));
    if (!idx) return NULL;
    int64_t n = 0;
    for (int64_t vx = 0; vx < nvox; vx++) {
        if (phase[vx] > nphase) { free(idx); return NULL; }
        idx[vx] = phase[vx] ? n++ : -1;
    }
    int noff = dim == 2 ? 4 : 9;
    const int(*off)[4] = dim == 2 ? OFF2 : OFF3;

    /* count springs */
    int64_t m = 0;
    for (int iz = 0; iz < nz; iz++)
        for (int iy = 0; iy < ny; iy++)
            for (int ix = 0; ix < nx; ix++) {
                int64_t vx = ix + (int64_t)nx * (iy + (int64_t)ny * iz);
                if (idx[vx] < 0) continue;
                for (int t = 0; t < noff; t++) {
                    int jx = ix + off[t][0], jy = iy + off[t][1], jz = iz + off[t][2];
                    if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) continue;
                    if (idx[jx + (int64_t)nx * (jy + (int64_t)ny * jz)] >= 0) m++;
                }
            }
    orc *o = orc_alloc(dim, n, m);
    if (!o) { free(idx); return NULL; }
    const double r0_1 = a;
    const double r0_2 = a * sqrt(2.0);
    int64_t s = 0;
    for (int iz = 0; iz < nz; iz++)
        for (int iy = 0; iy < ny; iy++)
            for (int ix = 0; ix < nx; ix++) {
                int64_t vx = ix + (int64_t)nx * (iy + (int64_t)ny * iz);
                int64_t p = idx[vx];
                if (p < 0) continue;
                o->X[p] = ix * a;
                o->X[n + p] = iy * a;
                if (dim == 3) o->X[2 * n + p] = iz * a;
                int ph = phase[vx];
                o->mass[p] = mass_tab ? mass_tab[ph - 1] : 1.0;
                o->grip[p] = ix == 0 ? 1 : (ix == nx - 1 ? 2 : 0);
                if (o->grip[p]) {
                    o->fix[p] = 1;
                    if (grip_mode == 1)
                        for (int c = 1; c < dim; c++) o->fix[c * n + p] = 1;
                }
                int64_t s0 = s;
                for (int t = 0; t < noff; t++) {
                    int jx = ix + off[t][0], jy = iy + off[t][1], jz = iz + off[t][2];
                    if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) continue;
                    int64_t vq = jx + (int64_t)nx * (jy + (int64_t)ny * jz);
                    int64_t q = idx[vq];
                    if (q < 0) continue;
                    int pq = phase[vq];
                    double kk = k_tab[(ph - 1) * nphase + (pq - 1)];
                    double ec = epsc_tab[(ph - 1) * nphase + (pq - 1)];
                    double r0 = off[t][3] == 1 ? r0_1 : r0_2;
                    if (off[t][3] == 2) kk = kk * k2_ratio;
                    double rc = r0 * (1.0 + ec);
                    o->si[s] = (int32_t)p;
                    o->sj[s] = (int32_t)q;
                    o->k[s] = kk;
                    o->r0[s] = r0;
                    o->rc2[s] = rc * rc;
                    s++;
                }
                /* canonical order: within one lower endpoint p, sort by q
                 * (insertion sort of at most 9 entries); p itself ascends. */
                for (int64_t u = s0 + 1; u < s; u++) {
                    int64_t w = u;
                    while (w > s0 && o->sj[w - 1] > o->sj[w]) {
                        int32_t ti = o->sj[w]; o->sj[w] = o->sj[w - 1]; o->sj[w - 1] = ti;
                        double td = o->k[w]; o->k[w] = o->k[w - 1]; o->k[w - 1] = td;
                        td = o->r0[w]; o->r0[w] = o->r0[w - 1]; o->r0[w - 1] = td;
                        td = o->rc2[w]; o->rc2[w] = o->rc2[w - 1]; o->rc2[w - 1] = td;
                        w--;
                    }
                }
            }
    free(idx);
    memcpy(o->x, o->X, (size_t)dim * n * sizeof(double));
    o->dt = dt;
    o->gamma = gamma;
    o->xc = 0.5 * (nx - 1) * a;
    o->omega = (nx - 1) * a * (ny * a);
    o->grip_area = ny * a;
    if (dim == 3) {
        o->omega = o->omega * (nz * a);
        o->grip_area = o->grip_area * (nz * a);
    }
    o->load_mode = load_mode;
    orc_init_accel(o);
    return o;
}

/* ------------------------------------------------- triangular packing -- */

/* floor(sqrt(v)) for v >= 0, exactly. */
static int64_t orc_isqrt(int64_t v)
{
    int64_t r = (int64_t)sqrt((double)v);
    while (r > 0 && r * r > v) r--;
    while ((r + 1) * (r + 1) <= v) r++;
    return r;
}

/* Image -> particles and springs on the triangular packing that the paper's
 * Img2Particle emits (Section 1; first neighbours only, six per interior
 * particle, Section 1 on the spring count). Reading of the paper (which
 * gives no formula): lattice rows iy = 0..R-1 at height y = iy h with
 * h = (a sqrt 3) 0.5; row iy holds sites ix = 0..C-1, C = nx (even iy) or
 * nx - 1 (odd iy), at x = (ix + 0.5 (iy odd)) a; R is the number of rows
 * with iy sqrt(3)/2 <= ny - 1 (in pixels). A site takes the phase of the
 * pixel nearest to it: column ix + (iy odd), row round(iy sqrt(3)/2),
 * evaluated in integers. Springs join each site to its forward neighbours
 * (same row +1; the two sites of row iy + 1 at x -+ a/2), r0 = a. Grips are
 * the first and last site of each row. Omega = (nx - 1) a R h, grip area
 * R h. */
static orc *orc_build_tri(int nx, int ny, const uint8_t *phase, int nphase, const double *k_tab,
                          const double *epsc_tab, const double *mass_tab, double a, double dt,
                          double gamma, int grip_mode, int load_mode)
{
    if (nx < 2 || ny < 1 || nphase < 1 || !phase || !k_tab || !epsc_tab) return NULL;
    int64_t R = 0;
    while (3 * (R + 1) * (R + 1) <= 4 * (int64_t)(ny - 1) * (ny - 1)) R++;
    R += 1; /* rows 0..R-1 */
    /* site (ix, iy) -> particle index or -1; sites in row-major order */
    int64_t *base = (int64_t *)malloc((size_t)(R + 1) * sizeof(int64_t));
    if (!base) return NULL;
    base[0] = 0;
    for (int64_t iy = 0; iy < R; iy++) base[iy + 1] = base[iy] + (iy & 1 ? nx - 1 : nx);
    const int64_t nsite = base[R];
    int64_t *idx = (int64_t *)malloc((size_t)nsite * sizeof(int64_t));
    uint8_t *sph = (uint8_t *)malloc((size_t)nsite);
    if (!idx || !sph) { free(base); free(idx); free(sph); return NULL; }
    int64_t n = 0;
    for (int64_t iy = 0; iy < R; iy++) {
        const int64_t row = (orc_isqrt(3 * iy * iy) + 1) / 2;
        for (int64_t ix = 0; ix < base[iy + 1] - base[iy]; ix++) {
            const int64_t col = ix + (iy & 1);
            const uint8_t ph = phase[row * nx + col];
            if (ph > nphase) { free(base); free(idx); free(sph); return NULL; }
            sph[base[iy] + ix] = ph;
            idx[base[iy] + ix] = ph ? n++ : -1;
        }
    }
    /* forward neighbours of site (ix, iy) in ascending site order */
#define TRI_NB(ix, iy, t, jx, jy)                                               \
    do {                                                                        \
        if ((t) == 0) { jx = (ix) + 1; jy = (iy); }                             \
        else { jy = (iy) + 1; jx = (ix) + ((iy) & 1 ? 0 : -1) + ((t) == 2); }   \
    } while (0)
    int64_t m = 0;
    for (int64_t iy = 0; iy < R; iy++)
        for (int64_t ix = 0; ix < base[iy + 1] - base[iy]; ix++) {
            if (idx[base[iy] + ix] < 0) continue;
            for (int t = 0; t < 3; t++) {
                int64_t jx, jy;
                TRI_NB(ix, iy, t, jx, jy);
                if (jy >= R || jx < 0 || jx >= base[jy + 1] - base[jy]) continue;
                if (idx[base[jy] + jx] >= 0) m++;
            }
        }
    orc *o = orc_alloc(2, n, m);
    if (!o) { free(base); free(idx); free(sph); return NULL; }
    const double h = a * sqrt(3.0) * 0.5;
    int64_t s = 0;
    for (int64_t iy = 0; iy < R; iy++) {
        const int64_t C = base[iy + 1] - base[iy];
        for (int64_t ix = 0; ix < C; ix++) {
            const int64_t p = idx[base[iy] + ix];
            if (p < 0) continue;
            const int ph = sph[base[iy] + ix];
            o->X[p] = (ix + 0.5 * (double)(iy & 1)) * a;
            o->X[n + p] = iy * h;
            o->mass[p] = mass_tab ? mass_tab[ph - 1] : 1.0;
            o->grip[p] = ix == 0 ? 1 : (ix == C - 1 ? 2 : 0);
            if (o->grip[p]) {
                o->fix[p] = 1;
                if (grip_mode == 1) o->fix[n + p] = 1;
            }
            for (int t = 0; t < 3; t++) { /* targets ascend with t */
                int64_t jx, jy;
                TRI_NB(ix, iy, t, jx, jy);
                if (jy >= R || jx < 0 || jx >= base[jy + 1] - base[jy]) continue;
                const int64_t q = idx[base[jy] + jx];
                if (q < 0) continue;
                const int pq = sph[base[jy] + jx];
                const double ec = epsc_tab[(ph - 1) * nphase + (pq - 1)];
                const double rc = a * (1.0 + ec);
                o->si[s] = (int32_t)p;
                o->sj[s] = (int32_t)q;
                o->k[s] = k_tab[(ph - 1) * nphase + (pq - 1)];
                o->r0[s] = a;
                o->rc2[s] = rc * rc;
                s++;
            }
        }
    }
#undef TRI_NB
    free(base); free(idx); free(sph);
    memcpy(o->x, o->X, (size_t)2 * n * sizeof(double));
    o->dt = dt;
    o->gamma = gamma;
    o->xc = 0.5 * (nx - 1) * a;
    o->omega = (nx - 1) * a * (R * h);
    o->grip_area = R * h;
    o->load_mode = load_mode;
    orc_init_accel(o);
    return o;
}

/* General spring network (the paper's solver reads arbitrary particle/bond
 * data). Springs must already be in canonical order: si < sj, sorted by
 * (si, sj), no duplicates. rc2 is the squared break length (INFINITY for an
 * unbreakable spring). */
orc *orc_build_network(int dim, int64_t n, int64_t m, const double *X, const double *mass,
                       const uint8_t *fix, const uint8_t *grip, const int32_t *si,
                       const int32_t *sj, const double *k, const double *r0, const double *rc2,
                       double dt, double gamma, double xc, double omega, double grip_area,
                       int load_mode)
{
    if ((dim != 2 && dim != 3) || n < 1 || m < 0) return NULL;
    for (int64_t s = 0; s < m; s++) {
        if (si[s] < 0 || sj[s] >= n || si[s] >= sj[s]) return NULL;
        if (s > 0 && (si[s] < si[s - 1] || (si[s] == si[s - 1] && sj[s] <= sj[s - 1])))
            return NULL;
    }
    orc *o = orc_alloc(dim, n, m);
    if (!o) return NULL;
    memcpy(o->X, X, (size_t)dim * n * sizeof(double));
    memcpy(o->x, X, (size_t)dim * n * sizeof(double));
    for (int64_t p = 0; p < n; p++) o->mass[p] = mass ? mass[p] : 1.0;
    if (fix) memcpy(o->fix, fix, (size_t)dim * n);
    if (grip) memcpy(o->grip, grip, (size_t)n);
    if (m > 0) {
        memcpy(o->si, si, (size_t)m * sizeof(int32_t));
        memcpy(o->sj, sj, (size_t)m * sizeof(int32_t));
        memcpy(o->k, k, (size_t)m * sizeof(double));
        memcpy(o->r0, r0, (size_t)m * sizeof(double));
        memcpy(o->rc2, rc2, (size_t)m * sizeof(double));
    }
    o->dt = dt; o->gamma = gamma; o->xc = xc; o->omega = omega; o->grip_area = grip_area;
    o->load_mode = load_mode;
    orc_init_accel(o);
    return o;
}

/* ------------------------------------------------------------- queries -- */

void orc_sizes(const orc *o, int64_t *n, int64_t *m, int *dim)
{
    *n = o->n; *m = o->m; *dim = o->dim;
}

void orc_topology(const orc *o, int32_t *si, int32_t *sj, double *k, double *r0, double *rc2,
                  double *X, double *mass, uint8_t *fix, uint8_t *grip)
{
    size_t m = (size_t)o->m, dn = (size_t)o->dim * o->n;
    if (si) memcpy(si, o->si, m * sizeof(int32_t));
    if (sj) memcpy(sj, o->sj, m * sizeof(int32_t));
    if (k) memcpy(k, o->k, m * sizeof(double));
    if (r0) memcpy(r0, o->r0, m * sizeof(double));
    if (rc2) memcpy(rc2, o->rc2, m * sizeof(double));
    if (X) memcpy(X, o->X, dn * sizeof(double));
    if (mass) memcpy(mass, o->mass, (size_t)o->n * sizeof(double));
    if (fix) memcpy(fix, o->fix, dn);
    if (grip) memcpy(grip, o->grip, (size_t)o->n);
}

void orc_get_state(const orc *o, double *x, double *v, double *a)
{
    size_t dn = (size_t)o->dim * o->n * sizeof(double);
    if (x) memcpy(x, o->x, dn);
    if (v) memcpy(v, o->v, dn);
    if (a) memcpy(a, o->a, dn);
}

/* Replace positions and/or velocities. Without an explicit acceleration the
 * acceleration is re-evaluated from the new state (Eq. 4). */
void orc_set_state(orc *o, const double *x, const double *v, const double *a)
{
    size_t dn = (size_t)o->dim * o->n * sizeof(double);
    if (x) memcpy(o->x, x, dn);
    if (v) memcpy(o->v, v, dn);
    if (a) memcpy(o->a, a, dn);
    else orc_init_accel(o);
}

void orc_broken(const orc *o, uint8_t *mask, int64_t *brk_step, int64_t *first_break)
{
    if (mask) memcpy(mask, o->broken, (size_t)o->m);
    if (brk_step) memcpy(brk_step, o->brk_step, (size_t)o->m * sizeof(int64_t));
    if (first_break) *first_break = o->first_break;
}

/* -------------------------------------------------------------- physics -- */

/* Spring forces (Eq. 2) and potential (Eq. 1) at positions xs, over the
 * currently intact springs, without testing for breaks. Also returns the
 * virial sum W = sum_intact (x_j - x_i)_x f_x (f = force on i from j). */
void orc_forces(const orc *o, const double *xs, double *F, double *U, double *W)
{
    const int64_t n = o->n;
    const int dim = o->dim;
    memset(F, 0, (size_t)dim * n * sizeof(double));
    double u = 0.0, w = 0.0;
    for (int64_t s = 0; s < o->m; s++) {
        if (o->broken[s]) continue;
        int64_t i = o->si[s], j = o->sj[s];
        double d[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < dim; c++) d[c] = xs[c * n + j] - xs[c * n + i];
        double r2 = d[0] * d[0] + d[1] * d[1];
        if (dim == 3) r2 = r2 + d[2] * d[2];
        double r = sqrt(r2);
        double c_s = o->k[s] * (r - o->r0[s]) / r;
        for (int c = 0; c < dim; c++) {
            double f = c_s * d[c];
            F[c * n + i] += f;
            F[c * n + j] -= f;
        }
        double st = r - o->r0[s];
        u += 0.5 * o->k[s] * st * st;
        w += d[0] * (c_s * d[0]);
    }
    if (U) *U = u;
    if (W) *W = w;
}


/* Acceleration of the current state, Eq. 4 with the viscous term:
 * a = (F(x) - gamma v) / m on free components, 0 on prescribed ones.
 * Velocity Verlet needs a(t) before its first step; builds and state
 * uploads without an acceleration call this. Break tests are not run. */
static void orc_init_accel(orc *o)
{
    const int64_t n = o->n;
    const int64_t dn = (int64_t)o->dim * n;
    orc_forces(o, o->x, o->F, NULL, NULL);
    for (int64_t e = 0; e < dn; e++) {
        if (o->fix[e]) { o->a[e] = 0.0; continue; }
        o->a[e] = (o->F[e] - o->gamma * o->v[e]) / o->mass[e % n];
    }
}

/* The spring pass of one time step: break test on every intact spring in
 * canonical order, then the force of the springs still intact. */
static void orc_spring_pass(orc *o)
{
    const int64_t n = o->n;
    const int dim = o->dim;
    memset(o->F, 0, (size_t)dim * n * sizeof(double));
    for (int64_t s = 0; s < o->m; s++) {
        if (o->broken[s]) continue;
        int64_t i = o->si[s], j = o->sj[s];
        double d[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < dim; c++) d[c] = o->x[c * n + j] - o->x[c * n + i];
        double r2 = d[0] * d[0] + d[1] * d[1];
        if (dim == 3) r2 = r2 + d[2] * d[2];
        if (r2 > o->rc2[s]) { /* Heaviside switch: broken for good */
            o->broken[s] = 1;
            o->brk_step[s] = o->step;
            if (o->first_break < 0) o->first_break = o->step;
            continue;
        }
        double r = sqrt(r2);
        double c_s = o->k[s] * (r - o->r0[s]) / r;
        for (int c = 0; c < dim; c++) {
            double f = c_s * d[c];
            o->F[c * n + i] += f;
            o->F[c * n + j] -= f;
        }
    }
}

/* Number of host threads for the spring pass (1 = the sequential loop
 * above). Returns the number in use: 1 when built without OpenMP. */
int orc_set_threads(orc *o, int nthreads)
{
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#else
    nthreads = 1;
#endif
    if (nthreads > 1 && !o->row) {
        const int64_t n = o->n, m = o->m;
        o->row = calloc((size_t)n + 1, sizeof(int64_t));
        o->inc = calloc((size_t)(2 * m > 0 ? 2 * m : 1), sizeof(int64_t));
        o->fs = calloc((size_t)o->dim * (size_t)(m > 0 ? m : 1), sizeof(double));
        int64_t *fill = calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
        if (!o->row || !o->inc || !o->fs || !fill) {
            free(fill);
            return -1;
        }
        for (int64_t s = 0; s < m; s++) {
            o->row[o->si[s] + 1]++;
            o->row[o->sj[s] + 1]++;
        }
        for (int64_t p = 0; p < n; p++) o->row[p + 1] += o->row[p];
        for (int64_t p = 0; p < n; p++) fill[p] = o->row[p];
        for (int64_t s = 0; s < m; s++) { /* ascending s: each row comes out sorted */
            o->inc[fill[o->si[s]]++] = s << 1;
            o->inc[fill[o->sj[s]]++] = (s << 1) | 1;
        }
        free(fill);
    }
    o->nthreads = nthreads;
    return nthreads;
}

/* The threaded form of orc_spring_pass (see the header comment). */
static void orc_spring_pass_threads(orc *o)
{
    const int64_t n = o->n, m = o->m;
    const int dim = o->dim;
    const int64_t step = o->step;
    int64_t nbroke = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(o->nthreads) reduction(+ : nbroke)
#endif
    for (int64_t s = 0; s < m; s++) {
        for (int c = 0; c < dim; c++) o->fs[c * m + s] = 0.0;
        if (o->broken[s]) continue;
        int64_t i = o->si[s], j = o->sj[s];
        double d[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < dim; c++) d[c] = o->x[c * n + j] - o->x[c * n + i];
        double r2 = d[0] * d[0] + d[1] * d[1];
        if (dim == 3) r2 = r2 + d[2] * d[2];
        if (r2 > o->rc2[s]) {
            o->broken[s] = 1;
            o->brk_step[s] = step;
            nbroke += 1;
            continue;
        }
        double r = sqrt(r2);
        double c_s = o->k[s] * (r - o->r0[s]) / r;
        for (int c = 0; c < dim; c++) o->fs[c * m + s] = c_s * d[c];
    }
    if (nbroke > 0 && o->first_break < 0) o->first_break = step;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(o->nthreads)
#endif
    for (int64_t p = 0; p < n; p++) {
        for (int c = 0; c < dim; c++) {
            double acc = 0.0;
            for (int64_t e = o->row[p]; e < o->row[p + 1]; e++) {
                const int64_t w = o->inc[e], s = w >> 1;
                if (o->broken[s]) continue; /* no term, as in the scatter */
                if (w & 1) acc -= o->fs[c * m + s];
                else acc += o->fs[c * m + s];
            }
            o->F[c * n + p] = acc;
        }
    }
}

/* nsteps of damped velocity Verlet (Eqs. 3-5, half-step velocity form). */
void orc_step(orc *o, int64_t nsteps)
{
    const int64_t dn = (int64_t)o->dim * o->n;
    const double dt = o->dt, hdt = 0.5 * o->dt;
    for (int64_t t = 0; t < nsteps; t++) {
        /* Constant strain rate (Section 3.1: the boundary particles are
         * displaced apart at a fixed strain rate): the grips take the strain
         * of the step being computed, eps0 + (steps since the rate was set)
         * rate dt, before the positions advance; only the grips move. */
        if (o->rate_on) {
            const double eps = o->rate_eps0 + (double)(o->step + 1 - o->rate_step0) * o->rate_dt;
            for (int64_t p = 0; p < o->n; p++) {
                if (!o->fix[p]) continue;
                o->x[p] = o->X[p] + eps * (o->X[p] - o->xc);
                o->v[p] = 0.0;
                o->a[p] = 0.0;
            }
            o->eps = eps;
        }
        /* Eq. 3 via the half-step velocity: vh = v + dt/2 a; x += dt vh.
         * o->v holds vh until the end of the step. */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (o->nthreads > 1) num_threads(o->nthreads)
#endif
        for (int64_t e = 0; e < dn; e++) {
            if (o->fix[e]) continue;
            double vh = o->v[e] + hdt * o->a[e];
            o->v[e] = vh;
            o->x[e] = o->x[e] + dt * vh;
        }
        if (o->nthreads > 1)
            orc_spring_pass_threads(o);
        else
            orc_spring_pass(o);
        /* Eq. 4 with viscous damping, then Eq. 5: v = vh + dt/2 a(t+dt). */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (o->nthreads > 1) num_threads(o->nthreads)
#endif
        for (int64_t e = 0; e < dn; e++) {
            if (o->fix[e]) continue;
            int64_t p = e % o->n;
            double vh = o->v[e];
            o->a[e] = (o->F[e] - o->gamma * vh) / o->mass[p];
            o->v[e] = vh + hdt * o->a[e];
        }
        o->step += 1;
    }
}

/* Displacement-controlled load increment to engineering strain eps_new. */
void orc_apply_strain(orc *o, double eps_new)
{
    const int64_t n = o->n;
    if (o->load_mode == 0) {
        double s = (1.0 + eps_new) / (1.0 + o->eps);
        for (int64_t p = 0; p < n; p++) o->x[p] = o->xc + (o->x[p] - o->xc) * s;
    }
    for (int64_t p = 0; p < n; p++) {
        if (!o->fix[p]) continue;
        o->x[p] = o->X[p] + eps_new * (o->X[p] - o->xc);
        o->v[p] = 0.0;
        o->a[p] = 0.0;
    }
    o->eps = eps_new;
    if (o->rate_on) { /* the rate continues from the new strain */
        o->rate_eps0 = eps_new;
        o->rate_step0 = o->step;
    }
}

/* Constant strain-rate loading from the next step on (rate 0 stops it). */
void orc_set_strain_rate(orc *o, double rate)
{
    o->rate_on = rate != 0.0;
    o->rate_eps0 = o->eps;
    o->rate_step0 = o->step;
    o->rate_dt = rate * o->dt;
}

/* Observables of the current state:
 * out[0] eps, [1] sigma_xx virial (Eq. 7 over the reference box, tension
 * positive), [2] sigma_xx from the right-grip reaction, [3] PE (Eq. 1),
 * [4] KE, [5] number of broken springs, [6] residual = max over free
 * components of max(|F|, |v|), [7] step count. */
void orc_observe(const orc *o, double *out)
{
    const int64_t n = o->n;
    const int dim = o->dim;
    double *F = (double *)malloc((size_t)dim * n * sizeof(double));
    if (!F) { for (int q = 0; q < 8; q++) out[q] = NAN; return; }
    double U = 0.0, W = 0.0;
    orc_forces(o, o->x, F, &U, &W);
    double mvv = 0.0, ke = 0.0, res = 0.0, reac = 0.0;
    for (int64_t p = 0; p < n; p++) {
        mvv += o->mass[p] * o->v[p] * o->v[p];
        double v2 = 0.0;
        for (int c = 0; c < dim; c++) v2 += o->v[c * n + p] * o->v[c * n + p];
        ke += 0.5 * o->mass[p] * v2;
        if (o->grip[p] == 2) reac -= F[p];
        for (int c = 0; c < dim; c++) {
            int64_t e = c * n + p;
            if (o->fix[e]) continue;
            double af = fabs(F[e]), av = fabs(o->v[e]);
            double r = af > av ? af : av;
            if (r > res) res = r;
        }
    }
    int64_t nb = 0;
    for (int64_t s = 0; s < o->m; s++) nb += o->broken[s];
    out[0] = o->eps;
    out[1] = (W - mvv) / o->omega;
    out[2] = reac / o->grip_area;
    out[3] = U;
    out[4] = ke;
    out[5] = (double)nb;
    out[6] = res;
    out[7] = (double)o->step;
    free(F);
}

/* Per-particle fields of Section 3.2 at the current state.
 *
 * stress, Eq. 7 with the domain taken as one particle's cell (volume cell):
 *   sigma_ab(k) = (1/cell) [ 1/2 sum over the intact springs (k, l) of
 *                 (x_l - x_k)_a f^{kl}_b  -  m_k v_a v_b ],
 * f^{kl} the force on k from that spring (Eq. 2). With d = x_j - x_i and
 * c = k (r - r0) / r, the force on i is c d and on j is -c d, so each
 * endpoint receives 1/2 c d_a d_b.
 *
 * strain, Eq. 8 read as the Lagrangian strain 1/2 (J^T J - I) of the locally
 * affine map J: the least-squares J with (x_l - x_k) ~ J (X_l - X_k) over
 * the first-neighbour shell of k (its springs with the smallest rest
 * length, broken or not), J = B A^-1 with A = sum X X^T, B = sum d X^T. NaN
 * where the shell vectors do not span the space (|det A| tiny).
 *
 * Components, each an [n] block: 2D xx, yy, xy; 3D xx, yy, zz, xy, xz, yz.
 * Either output may be NULL. */
static const int ORC_PAIR[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
static const int ORC_PAIR2[3][2] = {{0, 0}, {1, 1}, {0, 1}};

void orc_fields(const orc *o, double cell, double *stress, double *strain)
{
    const int64_t n = o->n, m = o->m;
    const int dim = o->dim;
    const int nq = dim == 3 ? 6 : 3;
    const int (*pairs)[2] = dim == 3 ? ORC_PAIR : ORC_PAIR2;
    if (stress) {
        memset(stress, 0, (size_t)nq * n * sizeof(double));
        for (int64_t s = 0; s < m; s++) {
            if (o->broken[s]) continue;
            int64_t i = o->si[s], j = o->sj[s];
            double d[3] = {0.0, 0.0, 0.0};
            for (int c = 0; c < dim; c++) d[c] = o->x[c * n + j] - o->x[c * n + i];
            double r2 = d[0] * d[0] + d[1] * d[1];
            if (dim == 3) r2 = r2 + d[2] * d[2];
            double r = sqrt(r2);
            double c_s = o->k[s] * (r - o->r0[s]) / r;
            for (int q = 0; q < nq; q++) {
                double t = 0.5 * (d[pairs[q][0]] * (c_s * d[pairs[q][1]]));
                stress[q * n + i] += t;
                stress[q * n + j] += t;
            }
        }
        for (int64_t p = 0; p < n; p++)
            for (int q = 0; q < nq; q++) {
                double vv = o->mass[p] * o->v[pairs[q][0] * n + p] * o->v[pairs[q][1] * n + p];
                stress[q * n + p] = (stress[q * n + p] - vv) / cell;
            }
    }
    if (strain) {
        double *rmin = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
        double *A = (double *)calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double));
        double *B = (double *)calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double));
        if (!rmin || !A || !B) {
            free(rmin); free(A); free(B);
            for (int64_t e = 0; e < (int64_t)nq * n; e++) strain[e] = NAN;
            return;
        }
        for (int64_t p = 0; p < n; p++) rmin[p] = INFINITY;
        for (int64_t s = 0; s < m; s++) {
            if (o->r0[s] < rmin[o->si[s]]) rmin[o->si[s]] = o->r0[s];
            if (o->r0[s] < rmin[o->sj[s]]) rmin[o->sj[s]] = o->r0[s];
        }
        for (int64_t s = 0; s < m; s++) {
            int64_t i = o->si[s], j = o->sj[s];
            double X[3] = {0.0, 0.0, 0.0}, d[3] = {0.0, 0.0, 0.0};
            for (int c = 0; c < dim; c++) {
                X[c] = o->X[c * n + j] - o->X[c * n + i];
                d[c] = o->x[c * n + j] - o->x[c * n + i];
            }
            /* the products are the same seen from either endpoint */
            for (int end = 0; end < 2; end++) {
                int64_t p = end ? j : i;
                if (o->r0[s] > rmin[p] * (1.0 + 1e-12)) continue;
                for (int a = 0; a < dim; a++)
                    for (int b = 0; b < dim; b++) {
                        A[p * 9 + a * 3 + b] += X[a] * X[b];
                        B[p * 9 + a * 3 + b] += d[a] * X[b];
                    }
            }
        }
        for (int64_t p = 0; p < n; p++) {
            const double *Ap = A + p * 9, *Bp = B + p * 9;
            double inv[9] = {0}, J[9] = {0};
            double det, scale;
            if (dim == 2) {
                det = Ap[0] * Ap[4] - Ap[1] * Ap[3];
                scale = 0.5 * (Ap[0] + Ap[4]);
                inv[0] = Ap[4] / det; inv[1] = -Ap[1] / det;
                inv[3] = -Ap[3] / det; inv[4] = Ap[0] / det;
            } else {
                double c00 = Ap[4] * Ap[8] - Ap[5] * Ap[7];
                double c01 = Ap[5] * Ap[6] - Ap[3] * Ap[8];
                double c02 = Ap[3] * Ap[7] - Ap[4] * Ap[6];
                det = Ap[0] * c00 + Ap[1] * c01 + Ap[2] * c02;
                scale = (Ap[0] + Ap[4] + Ap[8]) / 3.0;
                inv[0] = c00 / det; inv[3] = c01 / det; inv[6] = c02 / det;
                inv[1] = (Ap[2] * Ap[7] - Ap[1] * Ap[8]) / det;
                inv[4] = (Ap[0] * Ap[8] - Ap[2] * Ap[6]) / det;
                inv[7] = (Ap[1] * Ap[6] - Ap[0] * Ap[7]) / det;
                inv[2] = (Ap[1] * Ap[5] - Ap[2] * Ap[4]) / det;
                inv[5] = (Ap[2] * Ap[3] - Ap[0] * Ap[5]) / det;
                inv[8] = (Ap[0] * Ap[4] - Ap[1] * Ap[3]) / det;
            }
            double sp = 1.0;
            for (int c = 0; c < dim; c++) sp *= scale;
            if (!(fabs(det) > 1e-12 * sp)) {
                for (int q = 0; q < nq; q++) strain[q * n + p] = NAN;
                continue;
            }
            for (int a = 0; a < dim; a++) /* J = B A^-1 */
                for (int b = 0; b < dim; b++) {
                    double t = 0.0;
                    for (int c = 0; c < dim; c++) t += Bp[a * 3 + c] * inv[c * 3 + b];
                    J[a * 3 + b] = t;
                }
            for (int q = 0; q < nq; q++) {
                int a = pairs[q][0], b = pairs[q][1];
                double t = 0.0;
                for (int c = 0; c < dim; c++) t += J[c * 3 + a] * J[c * 3 + b];
                strain[q * n + p] = 0.5 * (t - (a == b ? 1.0 : 0.0));
            }
        }
        free(rmin); free(A); free(B);
    }
}

/* Steps in batches of check_every until the residual is <= tol.
 * Returns ORC_OK, or ORC_ENOTCONV once max_steps were taken. */
int orc_relax(orc *o, double tol, int64_t max_steps, int64_t check_every, int64_t *taken)
{
    int64_t done = 0;
    double obs[8];
    if (check_every < 1) check_every = 1;
    for (;;) {
        if (done >= max_steps) { *taken = done; return ORC_ENOTCONV; }
        int64_t nb = max_steps - done < check_every ? max_steps - done : check_every;
        orc_step(o, nb);
        done += nb;
        orc_observe(o, obs);
        if (obs[6] <= tol) { *taken = done; return ORC_OK; }
    }
}
