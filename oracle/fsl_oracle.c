/*
 * fsl_oracle.c -- plain FP64 CPU oracle of the free-surface lattice Boltzmann
 * method (FSLBM) with the enhanced bubble model of Anderl et al.,
 * arXiv:1604.01632.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the library it checks.  It is
 * written for clarity, not speed: one pass per sub-step, plain loops over the
 * linear cell index, breadth-first flood fill for the bubbles every step.
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so every
 * floating-point operation is rounded exactly where it is written).
 *
 * Paper passages followed (equation numbers count the paper's displayed
 * equations in order):
 *   Sec. 2.1  Eq. 3 (equilibrium), Eqs. 4-5 (moments), Eqs. 6-7 (collide,
 *             stream), Eq. 8 (equation of state p = rho/3).
 *   Sec. 2.2  Eq. 9 (mass m = phi*rho), Eq. 10 (mass exchange), cell
 *             conversion text, Eq. 11 (free-surface reconstruction), Eq. 12
 *             (gas pressure p_V + dp_sigma), Eq. 13 (ideal gas p_V = (V*) over V times p0),
 *             Eq. 14 (p0 = rho0/3), Eq. 15 (dp_sigma = 2 sigma kappa),
 *             Parker-Youngs normals.
 *   Sec. 2.3  bubble data set, per-step volume update; Sec. 2.3.1 merge
 *             (V* and V summed); Sec. 2.3.2 split (flood fill, daughters keep
 *             the old pressure, volumes from gas cells plus interface cells by
 *             fill level).
 *
 * Where the paper is silent the oracle takes these readings (the CUDA library
 * takes the same ones):
 *   - D3Q19 order: rest; +x,-x,+y,-y,+z,-z; then (x,y), (x,z), (y,z) edge
 *     pairs, each direction followed by its opposite.  Weights 1/3, 1/18, 1/36.
 *   - Collision is two-relaxation-time; BGK is omega_minus = omega_plus.  Body
 *     force by Guo's scheme with F = rho*g on liquid and interface cells.
 *   - Reconstruction: an incoming direction alpha of an interface cell is
 *     rebuilt when its source cell is gas, or (normal rule) when the source is
 *     not a wall and g.c_alpha > 0, g the Parker-Youngs gradient of the fill
 *     level (n = -g points into the gas).  Gas velocity = velocity of the
 *     cell's own post-collision PDFs of the previous step.  rho_gas = 3 p_gas.
 *   - kappa = 1/2 div(n_hat) by central differences of n_hat at the six face
 *     neighbours; kappa < 0 on a bubble, so the liquid next to a bubble of
 *     radius R sees p_V - 2 sigma / R.
 *   - Conversion: filled if m > (1+eps) rho, emptied if m < -eps rho; an
 *     interface cell with no gas neighbour also counts as filled, one with no
 *     liquid neighbour as emptied (it no longer separates liquid from gas, and
 *     left alone it would form bubbles of zero volume); phase A
 *     (filled cells turn gas neighbours into interface, cancel emptied marks
 *     next to them), phase B (emptied cells turn liquid neighbours into
 *     interface).  New interface cells from gas get f = f_eq of the mean
 *     density and velocity of their liquid/interface neighbours, m = 0; new
 *     interface cells from liquid keep f, take m = rho and join the bubble of
 *     their first emptied neighbour in direction order.
 *   - Excess mass (filled: m - rho; emptied: m) is split equally among the
 *     neighbours that are interface after conversion; with no such neighbour
 *     it goes to a global pool (fixed point 2^-40) that is shared equally by
 *     all interface cells at the end of the same step.
 *   - A bubble is a connected component of gas + interface cells under the
 *     18-neighbourhood; its id is the minimum linear index of its cells.
 *     Volume V = sum over gas cells of 1 plus over interface cells of
 *     (1 - clamp(phi,0,1)), each term rounded to fixed point 2^-32 and summed
 *     exactly.  New V* of a component c = sum over old bubbles b of
 *     V*_b * V_{c,b} / V_b (V*_b copied when c holds all of b), so daughters
 *     keep p_old and merges add V*.
 */
#include "fsl_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* The OpenMP build (-fopenmp) runs the per-cell loops whose iterations touch
 * disjoint cells in parallel; its only reductions are integer counts and the
 * fixed-point pool, so it gives the serial build's results bit for bit.  The
 * serial build compiles these to nothing. */
#ifdef _OPENMP
#define FSL_ORA_PRAGMA(x) _Pragma(#x)
#define FSL_ORA_PARALLEL_FOR FSL_ORA_PRAGMA(omp parallel for schedule(static))
#define FSL_ORA_PARALLEL_FOR_SUM(a, b, c) FSL_ORA_PRAGMA(omp parallel for schedule(static) reduction(+ : a, b, c))
#define FSL_ORA_ATOMIC_WRITE FSL_ORA_PRAGMA(omp atomic write)
#else
#define FSL_ORA_PARALLEL_FOR
#define FSL_ORA_PARALLEL_FOR_SUM(a, b, c)
#define FSL_ORA_ATOMIC_WRITE
#endif

enum { LIQ = 0, IFC = 1, GAS = 2, OBS = 3, LID = 4 };
enum { MK_NONE = 0, MK_FILLED = 1, MK_EMPTIED = 2, MK_NEWG = 3, MK_NEWL = 4 };

static const int CX[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

static int opposite(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }
static double weight(int a) { return a == 0 ? 1.0 / 3.0 : (a <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

struct ora_sim {
    ora_params p;
    int64_t n;
    double omp, omm;
    double *f, *fn;           /* [19][n] post-collision PDFs, current and next */
    uint8_t *flag, *mark;
    double *m, *phi, *rhoi, *exs;
    int64_t *id;              /* canonical bubble id of gas/interface cells, else -1 */
    int64_t *slot;            /* canonical id -> index into bub, else -1 */
    int64_t *lab, *queue;     /* flood-fill scratch */
    ora_bubble *bub;
    int64_t nbub;
    int has_seed;
    int64_t seed, rate_fx;
    int64_t pool_fx;
    int64_t conversions;
    int status;
};

/* ---------------------------------------------------------------- geometry */

static int64_t nbr(const ora_sim* s, int64_t i, int dx, int dy, int dz) {
    int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
    x = (x + dx + nx) % nx;
    y = (y + dy + ny) % ny;
    z = (z + dz + nz) % nz;
    return (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
}

/* Fill level as seen by the normal stencil: walls and liquid read 1, gas 0. */
static double phi_stencil(const ora_sim* s, int64_t j) {
    switch (s->flag[j]) {
    case LIQ: case OBS: case LID: return 1.0;
    case GAS: return 0.0;
    default: {
        double v = s->phi[j];
        return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
    }
    }
}

/* Parker-Youngs gradient of the fill level: central differences summed over
 * the 3x3 cross-section with weights 4 (face), 2 (edge), 1 (corner). */
void ora_gradient(const ora_sim* s, int64_t i, double* g) {
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (int b = -1; b <= 1; ++b) {
        for (int a = -1; a <= 1; ++a) {
            double W = (a == 0 && b == 0) ? 4.0 : ((a == 0 || b == 0) ? 2.0 : 1.0);
            gx = gx + W * (phi_stencil(s, nbr(s, i, 1, a, b)) - phi_stencil(s, nbr(s, i, -1, a, b)));
            gy = gy + W * (phi_stencil(s, nbr(s, i, a, 1, b)) - phi_stencil(s, nbr(s, i, a, -1, b)));
            gz = gz + W * (phi_stencil(s, nbr(s, i, a, b, 1)) - phi_stencil(s, nbr(s, i, a, b, -1)));
        }
    }
    g[0] = gx; g[1] = gy; g[2] = gz;
}

/* Unit normal pointing into the gas, n_hat = -g/|g| (zero where g = 0). */
static void unit_normal(const ora_sim* s, int64_t i, double* n) {
    double g[3];
    ora_gradient(s, i, g);
    double q = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    if (q > 0.0) {
        double len = sqrt(q);
        n[0] = -(g[0] / len); n[1] = -(g[1] / len); n[2] = -(g[2] / len);
    } else {
        n[0] = 0.0; n[1] = 0.0; n[2] = 0.0;
    }
}

/* Curvature kappa = 1/2 div(n_hat), central differences (Sec. 2.2, Eq. 15). */
double ora_curvature(const ora_sim* s, int64_t i) {
    double np[3], nm[3];
    unit_normal(s, nbr(s, i, 1, 0, 0), np);
    unit_normal(s, nbr(s, i, -1, 0, 0), nm);
    double dX = np[0] - nm[0];
    unit_normal(s, nbr(s, i, 0, 1, 0), np);
    unit_normal(s, nbr(s, i, 0, -1, 0), nm);
    double dY = np[1] - nm[1];
    unit_normal(s, nbr(s, i, 0, 0, 1), np);
    unit_normal(s, nbr(s, i, 0, 0, -1), nm);
    double dZ = np[2] - nm[2];
    return 0.25 * ((dX + dY) + dZ);
}

/* ------------------------------------------------------------- LBM pieces */

void ora_lattice(int32_t* c, double* w, int32_t* opp) {
    for (int a = 0; a < 19; ++a) {
        c[3 * a + 0] = CX[a]; c[3 * a + 1] = CY[a]; c[3 * a + 2] = CZ[a];
        w[a] = weight(a);
        opp[a] = opposite(a);
    }
}

static double cdot(int a, double vx, double vy, double vz) {
    return ((double)CX[a] * vx + (double)CY[a] * vy) + (double)CZ[a] * vz;
}

/* Second-order equilibrium (Sec. 2.1, Eq. 3) written as the symmetric part
 * w rho (1 + 9/2 (c.u)^2 - 3/2 u.u) plus/minus the antisymmetric part
 * w rho 3 c.u for each opposite pair. */
void ora_feq(double rho, const double* u, double* out) {
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    out[0] = (weight(0) * rho) * (1.0 - 1.5 * usq);
    for (int a = 1; a < 19; a += 2) {
        double cu = cdot(a, u[0], u[1], u[2]);
        double wr = weight(a) * rho;
        double fp = wr * ((1.0 + 4.5 * (cu * cu)) - 1.5 * usq);
        double fm = wr * (3.0 * cu);
        out[a] = fp + fm;
        out[a + 1] = fp - fm;
    }
}

/* Density and momentum (Sec. 2.1, Eqs. 4-5). */
static void moments(const double* f, double* rho, double* j) {
    double r = f[0];
    for (int a = 1; a < 19; ++a) r = r + f[a];
    *rho = r;
    j[0] = f[1] - f[2] + f[7] - f[8] + f[9] - f[10] + f[11] - f[12] + f[13] - f[14];
    j[1] = f[3] - f[4] + f[7] - f[8] - f[9] + f[10] + f[15] - f[16] + f[17] - f[18];
    j[2] = f[5] - f[6] + f[11] - f[12] - f[13] + f[14] + f[15] - f[16] - f[17] + f[18];
}

static void relaxation_rates(const ora_params* p, double* omp, double* omm) {
    *omp = 1.0 / p->tau;
    if (p->collision == 1)
        *omm = 1.0 / (p->magic / (p->tau - 0.5) + 0.5);
    else
        *omm = *omp;
}

/* Collision (Sec. 2.1, Eq. 6) in two-relaxation-time form with Guo forcing.
 * Returns the density. */
static double collide_rates(double omp, double omm, const double* gvec, const double* fin, double* fout) {
    double rho, j[3];
    moments(fin, &rho, j);
    double F[3] = {rho * gvec[0], rho * gvec[1], rho * gvec[2]};
    double ux = (j[0] + 0.5 * F[0]) / rho;
    double uy = (j[1] + 0.5 * F[1]) / rho;
    double uz = (j[2] + 0.5 * F[2]) / rho;
    double usq = ux * ux + uy * uy + uz * uz;
    double uF = ux * F[0] + uy * F[1] + uz * F[2];
    double cp = 1.0 - 0.5 * omp, cm = 1.0 - 0.5 * omm;
    double feq0 = (weight(0) * rho) * (1.0 - 1.5 * usq);
    double S0 = weight(0) * (-3.0 * uF);
    fout[0] = (fin[0] - omp * (fin[0] - feq0)) + cp * S0;
    for (int a = 1; a < 19; a += 2) {
        int b = a + 1;
        double w = weight(a);
        double cu = cdot(a, ux, uy, uz);
        double cF = cdot(a, F[0], F[1], F[2]);
        double wr = w * rho;
        double feqp = wr * ((1.0 + 4.5 * (cu * cu)) - 1.5 * usq);
        double feqm = wr * (3.0 * cu);
        double fp = 0.5 * (fin[a] + fin[b]);
        double fm = 0.5 * (fin[a] - fin[b]);
        double Sp = w * ((9.0 * cu) * cF - 3.0 * uF);
        double Sm = w * (3.0 * cF);
        double A = omp * (fp - feqp);
        double B = omm * (fm - feqm);
        double sp = cp * Sp, sm = cm * Sm;
        fout[a] = (((fin[a] - A) - B) + sp) + sm;
        fout[b] = (((fin[b] - A) + B) + sp) - sm;
    }
    return rho;
}

double ora_collide(const ora_params* p, const double* fin, double* fout) {
    double omp, omm;
    relaxation_rates(p, &omp, &omm);
    return collide_rates(omp, omm, p->g, fin, fout);
}

/* ----------------------------------------------------------- bubble model */

static int64_t volume_term(uint8_t t, double phi) {
    if (t == GAS) return (int64_t)4294967296LL;
    if (t == IFC) {
        double c = phi < 0.0 ? 0.0 : (phi > 1.0 ? 1.0 : phi);
        return llrint((1.0 - c) * 4294967296.0);
    }
    return 0;
}

double ora_bubble_pressure(const ora_bubble* b) {
    const double p0 = 1.0 / 3.0;
    if (b->constp) return p0;
    double V = (double)(b->vfx + b->vxfx) * ldexp(1.0, -32);
    if (V <= 1e-3) return p0;
    double Vs = (double)b->vsfx * ldexp(1.0, -32);
    return (Vs / V) * p0;
}

/* Connected components of fg (nonzero) under the 18-neighbourhood with wrap;
 * label = minimum linear index of the component, -1 for background.  Each
 * component is flooded breadth-first from its lowest cell (Sec. 2.3.2). */
static void label_into(const uint8_t* fg, int nx, int ny, int nz, int64_t* lab, int64_t* queue) {
    int64_t n = (int64_t)nx * ny * nz;
    for (int64_t i = 0; i < n; ++i) lab[i] = -1;
    for (int64_t i = 0; i < n; ++i) {
        if (!fg[i] || lab[i] >= 0) continue;
        int64_t head = 0, tail = 0;
        queue[tail++] = i;
        lab[i] = i;
        while (head < tail) {
            int64_t c = queue[head++];
            int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((int64_t)nx * ny));
            for (int a = 1; a < 19; ++a) {
                int xx = (x + CX[a] + nx) % nx, yy = (y + CY[a] + ny) % ny, zz = (z + CZ[a] + nz) % nz;
                int64_t j = (int64_t)xx + (int64_t)nx * ((int64_t)yy + (int64_t)ny * zz);
                if (fg[j] && lab[j] < 0) {
                    lab[j] = i;
                    queue[tail++] = j;
                }
            }
        }
    }
}

void ora_label(const uint8_t* fg, int32_t nx, int32_t ny, int32_t nz, int64_t* label) {
    int64_t n = (int64_t)nx * ny * nz;
    int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    label_into(fg, nx, ny, nz, label, queue);
    free(queue);
}

typedef struct { int64_t c, b, t; } pair_rec;

static int cmp_pair(const void* x, const void* y) {
    const pair_rec* a = (const pair_rec*)x;
    const pair_rec* b = (const pair_rec*)y;
    if (a->c != b->c) return a->c < b->c ? -1 : 1;
    if (a->b != b->b) return a->b < b->b ? -1 : 1;
    return 0;
}

/* Flood fill every step and rebuild the bubble table (Secs. 2.3.1, 2.3.2). */
static void rebuild_bubbles(ora_sim* s, int initial) {
    int64_t n = s->n;
    uint8_t* fg = (uint8_t*)malloc((size_t)n);
    for (int64_t i = 0; i < n; ++i) fg[i] = (s->flag[i] == GAS || s->flag[i] == IFC);
    label_into(fg, s->p.nx, s->p.ny, s->p.nz, s->lab, s->queue);

    int64_t nfg = 0;
    for (int64_t i = 0; i < n; ++i) nfg += fg[i];
    pair_rec* pr = (pair_rec*)malloc(sizeof(pair_rec) * (size_t)(nfg > 0 ? nfg : 1));
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!fg[i]) continue;
        pr[k].c = s->lab[i];
        pr[k].b = initial ? -1 : s->id[i];
        pr[k].t = volume_term(s->flag[i], s->phi[i]);
        ++k;
    }
    qsort(pr, (size_t)nfg, sizeof(pair_rec), cmp_pair);

    /* collapse to (c, b, V_cb, count) */
    int64_t np = 0;
    int64_t* pc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nfg + 1));
    int64_t* pb = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nfg + 1));
    int64_t* pv = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nfg + 1));
    int64_t* pvx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nfg + 1));
    int64_t* pn = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nfg + 1));
    for (int64_t q = 0; q < nfg; ++q) {
        if (np == 0 || pc[np - 1] != pr[q].c || pb[np - 1] != pr[q].b) {
            pc[np] = pr[q].c; pb[np] = pr[q].b; pv[np] = 0; pvx[np] = 0; pn[np] = 0; ++np;
        }
        pv[np - 1] += pr[q].t;
        pn[np - 1] += 1;
    }

    /* the reservoir's extra volume rides on the pair holding the seed cell */
    int64_t seed_c = -1, seed_b = -1, seed_vx = 0;
    if (!initial && s->has_seed && fg[s->seed]) {
        seed_c = s->lab[s->seed];
        seed_b = s->id[s->seed];
        int64_t ob = s->slot[seed_b];
        if (ob >= 0) seed_vx = s->bub[ob].vxfx;
        for (int64_t q = 0; q < np; ++q)
            if (pc[q] == seed_c && pb[q] == seed_b) pvx[q] = seed_vx;
    }

    /* old-bubble totals V_b and the lowest component holding each old bubble */
    int64_t* vtot = NULL;
    int64_t* minc = NULL;
    if (!initial) {
        vtot = (int64_t*)calloc((size_t)s->nbub + 1, sizeof(int64_t));
        minc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s->nbub + 1));
        for (int64_t q = 0; q <= s->nbub; ++q) minc[q] = -1;
        for (int64_t q = 0; q < np; ++q) {
            int64_t ob = s->slot[pb[q]];
            vtot[ob] += pv[q] + pvx[q];
            if (minc[ob] < 0 || pc[q] < minc[ob]) minc[ob] = pc[q];
        }
    }

    /* new table, in ascending canonical id (pairs are sorted by c) */
    ora_bubble* nb = (ora_bubble*)calloc((size_t)(np > 0 ? np : 1), sizeof(ora_bubble));
    int64_t nn = 0;
    for (int64_t q = 0; q < np; ++q) {
        if (nn == 0 || nb[nn - 1].id != pc[q]) {
            memset(&nb[nn], 0, sizeof(ora_bubble));
            nb[nn].id = pc[q];
            ++nn;
        }
        ora_bubble* c = &nb[nn - 1];
        c->vfx += pv[q];
        c->ncells += pn[q];
        if (initial) {
            c->vsfx += pv[q];
            continue;
        }
        int64_t ob = s->slot[pb[q]];
        const ora_bubble* o = &s->bub[ob];
        int64_t vcb = pv[q] + pvx[q];
        int64_t contrib;
        if (vtot[ob] == 0)
            contrib = (pc[q] == minc[ob]) ? o->vsfx : 0;
        else if (vcb == vtot[ob])
            contrib = o->vsfx;
        else {
            double r = (double)vcb / (double)vtot[ob];
            contrib = llrint((double)o->vsfx * r);
        }
        c->vsfx += contrib;
        c->vxfx += pvx[q];
        if (o->constp) c->constp = 1;
    }

    /* install */
    for (int64_t i = 0; i < n; ++i) s->id[i] = fg[i] ? s->lab[i] : -1;
    for (int64_t q = 0; q < s->nbub; ++q) s->slot[s->bub[q].id] = -1;
    free(s->bub);
    s->bub = nb;
    s->nbub = nn;
    for (int64_t q = 0; q < nn; ++q) s->slot[nb[q].id] = q;

    free(vtot); free(minc);
    free(pc); free(pb); free(pv); free(pvx); free(pn);
    free(pr); free(fg);
}

/* -------------------------------------------------------------- lifecycle */

ora_sim* ora_create(const ora_params* p) {
    if (p->nx <= 0 || p->ny <= 0 || p->nz <= 0) return NULL;
    ora_sim* s = (ora_sim*)calloc(1, sizeof(ora_sim));
    s->p = *p;
    s->n = (int64_t)p->nx * p->ny * p->nz;
    relaxation_rates(p, &s->omp, &s->omm);
    size_t n = (size_t)s->n;
    s->f = (double*)calloc(19 * n, sizeof(double));
    s->fn = (double*)calloc(19 * n, sizeof(double));
    s->flag = (uint8_t*)calloc(n, 1);
    s->mark = (uint8_t*)calloc(n, 1);
    s->m = (double*)calloc(n, sizeof(double));
    s->phi = (double*)calloc(n, sizeof(double));
    s->rhoi = (double*)calloc(n, sizeof(double));
    s->exs = (double*)calloc(n, sizeof(double));
    s->id = (int64_t*)malloc(n * sizeof(int64_t));
    s->slot = (int64_t*)malloc(n * sizeof(int64_t));
    s->lab = (int64_t*)malloc(n * sizeof(int64_t));
    s->queue = (int64_t*)malloc(n * sizeof(int64_t));
    for (size_t i = 0; i < n; ++i) { s->id[i] = -1; s->slot[i] = -1; }
    return s;
}

void ora_destroy(ora_sim* s) {
    if (!s) return;
    free(s->f); free(s->fn); free(s->flag); free(s->mark); free(s->m); free(s->phi);
    free(s->rhoi); free(s->exs); free(s->id); free(s->slot); free(s->lab); free(s->queue);
    free(s->bub);
    free(s);
}

int ora_init(ora_sim* s, const uint8_t* flags, const double* fill, const double* rho, const double* u) {
    int64_t n = s->n;
    for (int64_t i = 0; i < n; ++i) {
        if (flags[i] > LID) return -1;
        s->flag[i] = flags[i];
    }
    /* the interface cells must close the liquid off from the gas (Sec. 2.2) */
    for (int64_t i = 0; i < n; ++i) {
        if (s->flag[i] != LIQ) continue;
        for (int a = 1; a < 19; ++a)
            if (s->flag[nbr(s, i, CX[a], CY[a], CZ[a])] == GAS) return -2;
    }
    for (int64_t i = 0; i < n; ++i) {
        uint8_t t = s->flag[i];
        s->mark[i] = MK_NONE;
        s->id[i] = -1;
        s->m[i] = 0.0; s->rhoi[i] = 0.0; s->exs[i] = 0.0;
        s->phi[i] = (t == LIQ) ? 1.0 : (t == IFC ? fill[i] : 0.0);
        for (int a = 0; a < 19; ++a) s->f[(size_t)a * n + i] = 0.0;
        if (t == LIQ || t == IFC) {
            double uu[3] = {u[i], u[n + i], u[2 * n + i]};
            double fe[19];
            ora_feq(rho[i], uu, fe);
            for (int a = 0; a < 19; ++a) s->f[(size_t)a * n + i] = fe[a];
            s->rhoi[i] = rho[i];
            s->m[i] = (t == IFC) ? fill[i] * rho[i] : rho[i];
        }
    }
    s->pool_fx = 0;
    s->has_seed = 0;
    s->status = 0;
    free(s->bub);
    s->bub = NULL;
    s->nbub = 0;
    for (int64_t i = 0; i < n; ++i) s->slot[i] = -1;
    rebuild_bubbles(s, 1);
    return 0;
}

int ora_set_source(ora_sim* s, int64_t seed_cell, double extra0, double rate, int32_t constp) {
    if (seed_cell < 0 || seed_cell >= s->n) return -1;
    int64_t b = s->id[seed_cell];
    if (b < 0) return -1;
    ora_bubble* o = &s->bub[s->slot[b]];
    if (constp) {
        o->constp = 1;
        return 0;
    }
    int64_t x0 = llrint(extra0 * 4294967296.0);
    o->vxfx = x0;
    o->vsfx += x0;
    s->has_seed = 1;
    s->seed = seed_cell;
    s->rate_fx = llrint(rate * 4294967296.0);
    return 0;
}

static double bubble_p(const ora_sim* s, int64_t id) {
    int64_t q = s->slot[id];
    if (q < 0) return 1.0 / 3.0;
    return ora_bubble_pressure(&s->bub[q]);
}

static int new_type(uint8_t t, uint8_t mk) {
    if (t == IFC) {
        if (mk == MK_FILLED) return LIQ;
        if (mk == MK_EMPTIED) return GAS;
        return IFC;
    }
    if (t == GAS && mk == MK_NEWG) return IFC;
    if (t == LIQ && mk == MK_NEWL) return IFC;
    return t;
}

static int is_converted(uint8_t t, uint8_t mk) {
    return t == IFC && (mk == MK_FILLED || mk == MK_EMPTIED);
}

/* One time step. */
static void step_once(ora_sim* s) {
    const int64_t n = s->n;
    const ora_params* P = &s->p;
    double* F = s->f;
    double* FN = s->fn;
    const double eps = P->eps;

    /* S1: stream with bounce-back (Eq. 7), mass exchange (Eq. 10),
     * reconstruction (Eq. 11), collision (Eq. 6), fill level and marks. */
    FSL_ORA_PARALLEL_FOR
    for (int64_t i = 0; i < n; ++i) {
        uint8_t t = s->flag[i];
        if (t != LIQ && t != IFC) continue;
        double fin[19], fout[19], fg[19];
        double g[3] = {0.0, 0.0, 0.0};
        if (t == IFC) {
            double fs[19], rs, js[3];
            for (int a = 0; a < 19; ++a) fs[a] = F[(size_t)a * n + i];
            moments(fs, &rs, js);
            double ug[3] = {js[0] / rs, js[1] / rs, js[2] / rs};
            double kappa = ora_curvature(s, i);
            double pv = bubble_p(s, s->id[i]);
            double pg = pv + (2.0 * P->sigma) * kappa;   /* Eqs. 12, 15 */
            double rg = 3.0 * pg;                        /* Eq. 8 */
            ora_feq(rg, ug, fg);
            ora_gradient(s, i, g);
        }
        fin[0] = F[i];
        for (int a = 1; a < 19; ++a) {
            int ab = opposite(a);
            int64_t y = nbr(s, i, -CX[a], -CY[a], -CZ[a]);
            uint8_t ty = s->flag[y];
            if (ty == OBS) {
                fin[a] = F[(size_t)ab * n + i];
            } else if (ty == LID) {
                double cuw = cdot(a, P->lid[0], P->lid[1], P->lid[2]);
                fin[a] = F[(size_t)ab * n + i] + (6.0 * weight(a)) * cuw;
            } else if (ty == GAS) {
                if (t == LIQ) {
                    FSL_ORA_ATOMIC_WRITE
                    s->status = -2;
                    fin[a] = F[(size_t)ab * n + i];
                } else {
                    fin[a] = (fg[a] + fg[ab]) - F[(size_t)ab * n + i];
                }
            } else {
                fin[a] = F[(size_t)a * n + y];
                if (t == IFC && P->normal_rule && cdot(a, g[0], g[1], g[2]) > 0.0)
                    fin[a] = (fg[a] + fg[ab]) - F[(size_t)ab * n + i];
            }
        }
        double mnew = 0.0;
        if (t == IFC) {
            double dm = 0.0;
            for (int a = 1; a < 19; ++a) {
                int ab = opposite(a);
                int64_t z = nbr(s, i, CX[a], CY[a], CZ[a]);
                uint8_t tz = s->flag[z];
                double ex = F[(size_t)ab * n + z] - F[(size_t)a * n + i];
                if (tz == LIQ) dm = dm + ex;
                else if (tz == IFC) dm = dm + (0.5 * (s->phi[i] + s->phi[z])) * ex;
            }
            mnew = s->m[i] + dm;
        }
        double rho = collide_rates(s->omp, s->omm, P->g, fin, fout);
        if (!(rho == rho)) {
            FSL_ORA_ATOMIC_WRITE
            s->status = -4;
        }
        for (int a = 0; a < 19; ++a) FN[(size_t)a * n + i] = fout[a];
        s->mark[i] = MK_NONE;
        if (t == IFC) {
            s->m[i] = mnew;
            s->rhoi[i] = rho;
            if (mnew > (1.0 + eps) * rho) s->mark[i] = MK_FILLED;
            else if (mnew < (-eps) * rho) s->mark[i] = MK_EMPTIED;
            else if (P->lonely_rule) {
                /* an interface cell that no longer separates liquid from gas:
                 * without a gas neighbour it becomes liquid, without a liquid
                 * neighbour it becomes gas (types at the start of the step) */
                int has_gas = 0, has_liq = 0;
                for (int a = 1; a < 19; ++a) {
                    uint8_t tz = s->flag[nbr(s, i, CX[a], CY[a], CZ[a])];
                    if (tz == GAS) has_gas = 1;
                    if (tz == LIQ) has_liq = 1;
                }
                if (!has_gas) s->mark[i] = MK_FILLED;
                else if (!has_liq) s->mark[i] = MK_EMPTIED;
            }
        }
    }
    FSL_ORA_PARALLEL_FOR
    for (int64_t i = 0; i < n; ++i) {
        uint8_t t = s->flag[i];
        if (t != LIQ && t != IFC) s->mark[i] = MK_NONE;
    }

    /* S2: conversion phase A -- filled cells claim their gas neighbours and
     * cancel emptied marks next to them. */
    for (int64_t i = 0; i < n; ++i) {
        uint8_t t = s->flag[i];
        int gas = (t == GAS);
        int emp = (t == IFC && s->mark[i] == MK_EMPTIED);
        if (!gas && !emp) continue;
        int hit = 0;
        for (int a = 1; a < 19 && !hit; ++a) {
            int64_t z = nbr(s, i, CX[a], CY[a], CZ[a]);
            if (s->flag[z] == IFC && s->mark[z] == MK_FILLED) hit = 1;
        }
        if (hit) s->mark[i] = gas ? MK_NEWG : MK_NONE;
    }

    /* S3: conversion phase B -- remaining emptied cells turn their liquid
     * neighbours into interface; new interface cells from gas are
     * initialised from their liquid/interface neighbours. */
    FSL_ORA_PARALLEL_FOR
    for (int64_t i = 0; i < n; ++i) {
        if (s->flag[i] != LIQ) continue;
        /* the new interface cell joins the bubble of its first emptied
         * neighbour in direction order */
        int64_t best = -1;
        for (int a = 1; a < 19 && best < 0; ++a) {
            int64_t z = nbr(s, i, CX[a], CY[a], CZ[a]);
            if (s->flag[z] == IFC && s->mark[z] == MK_EMPTIED) best = s->id[z];
        }
        if (best >= 0) {
            double fo[19], r, j[3];
            for (int a = 0; a < 19; ++a) fo[a] = FN[(size_t)a * n + i];
            moments(fo, &r, j);
            s->mark[i] = MK_NEWL;
            s->id[i] = best;
            s->m[i] = r;
            s->rhoi[i] = r;
        }
    }
    FSL_ORA_PARALLEL_FOR
    for (int64_t i = 0; i < n; ++i) {
        if (s->flag[i] != GAS || s->mark[i] != MK_NEWG) continue;
        double sr = 0.0, su[3] = {0.0, 0.0, 0.0};
        int cnt = 0;
        for (int a = 1; a < 19; ++a) {
            int64_t z = nbr(s, i, CX[a], CY[a], CZ[a]);
            uint8_t tz = s->flag[z];
            if (tz == LIQ || (tz == IFC && s->mark[z] != MK_EMPTIED)) {
                double fo[19], r, j[3];
                for (int b = 0; b < 19; ++b) fo[b] = FN[(size_t)b * n + z];
                moments(fo, &r, j);
                sr = sr + r;
                su[0] = su[0] + j[0] / r;
                su[1] = su[1] + j[1] / r;
                su[2] = su[2] + j[2] / r;
                ++cnt;
            }
        }
        double rbar = sr / (double)cnt;
        double ubar[3] = {su[0] / (double)cnt, su[1] / (double)cnt, su[2] / (double)cnt};
        double fe[19];
        ora_feq(rbar, ubar, fe);
        for (int a = 0; a < 19; ++a) FN[(size_t)a * n + i] = fe[a];
        s->m[i] = 0.0;
        s->rhoi[i] = rbar;
    }

    /* S4: excess mass of converted cells, shares for the receivers. */
    int64_t n_if = 0;
    int64_t conv = 0;
    int64_t pooled = 0;   /* integer sums: the same in any order */
    FSL_ORA_PARALLEL_FOR_SUM(n_if, conv, pooled)
    for (int64_t i = 0; i < n; ++i) {
        uint8_t t = s->flag[i], mk = s->mark[i];
        if (new_type(t, mk) == IFC) ++n_if;
        if (!is_converted(t, mk)) continue;
        ++conv;
        double mex = (mk == MK_FILLED) ? s->m[i] - s->rhoi[i] : s->m[i];
        int k = 0;
        for (int a = 1; a < 19; ++a) {
            int64_t z = nbr(s, i, CX[a], CY[a], CZ[a]);
            if (new_type(s->flag[z], s->mark[z]) == IFC) ++k;
        }
        if (k > 0) s->exs[i] = mex / (double)k;
        else pooled += llrint(mex * 1099511627776.0);
    }
    s->pool_fx += pooled;
    s->conversions = conv;

    /* S5: receivers pull the shares in direction order, add the pool share,
     * and refresh the fill level phi = m / rho (Eq. 9). */
    double share = 0.0;
    if (n_if > 0) share = ((double)s->pool_fx * ldexp(1.0, -40)) / (double)n_if;
    FSL_ORA_PARALLEL_FOR
    for (int64_t i = 0; i < n; ++i) {
        if (new_type(s->flag[i], s->mark[i]) != IFC) continue;
        double sm = s->m[i];
        for (int a = 1; a < 19; ++a) {
            int64_t z = nbr(s, i, CX[a], CY[a], CZ[a]);
            if (is_converted(s->flag[z], s->mark[z])) sm = sm + s->exs[z];
        }
        if (n_if > 0) sm = sm + share;
        s->exs[i] = sm;   /* staged: flags are still needed by other cells */
    }
    FSL_ORA_PARALLEL_FOR
    for (int64_t i = 0; i < n; ++i) {
        uint8_t t = s->flag[i], mk = s->mark[i];
        int nt = new_type(t, mk);
        if (nt == IFC) {
            s->m[i] = s->exs[i];
            s->phi[i] = s->m[i] / s->rhoi[i];
        } else if (is_converted(t, mk)) {
            if (mk == MK_FILLED) {
                s->phi[i] = 1.0;
                s->id[i] = -1;
            } else {
                s->phi[i] = 0.0;
                s->m[i] = 0.0;
            }
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        s->flag[i] = (uint8_t)new_type(s->flag[i], s->mark[i]);
        s->mark[i] = MK_NONE;
        s->exs[i] = 0.0;
    }
    if (n_if > 0) s->pool_fx = 0;

    /* S6: reservoir drain, flood fill, merge/split of the bubble table. */
    if (s->has_seed && s->id[s->seed] >= 0) {
        int64_t q = s->slot[s->id[s->seed]];
        if (q >= 0) s->bub[q].vxfx -= s->rate_fx;
    }
    rebuild_bubbles(s, 0);

    /* swap PDF buffers */
    s->f = FN;
    s->fn = F;
}

int ora_step(ora_sim* s, int64_t nsteps) {
    for (int64_t k = 0; k < nsteps; ++k) step_once(s);
    return s->status;
}

int ora_status(const ora_sim* s) { return s->status; }

/* -------------------------------------------------------------- accessors */

void ora_get_f(const ora_sim* s, double* out) { memcpy(out, s->f, sizeof(double) * 19 * (size_t)s->n); }
void ora_get_flags(const ora_sim* s, uint8_t* out) { memcpy(out, s->flag, (size_t)s->n); }
void ora_get_phi(const ora_sim* s, double* out) { memcpy(out, s->phi, sizeof(double) * (size_t)s->n); }
void ora_get_mass(const ora_sim* s, double* out) { memcpy(out, s->m, sizeof(double) * (size_t)s->n); }
void ora_get_ids(const ora_sim* s, int64_t* out) { memcpy(out, s->id, sizeof(int64_t) * (size_t)s->n); }

int64_t ora_get_bubbles(const ora_sim* s, ora_bubble* out, int64_t cap) {
    int64_t k = s->nbub < cap ? s->nbub : cap;
    if (out && k > 0) memcpy(out, s->bub, sizeof(ora_bubble) * (size_t)k);
    return s->nbub;
}

int64_t ora_pool_fx(const ora_sim* s) { return s->pool_fx; }
int64_t ora_last_conversions(const ora_sim* s) { return s->conversions; }
