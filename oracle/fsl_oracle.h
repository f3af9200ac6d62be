/*
 * fsl_oracle.h -- plain FP64 CPU oracle of the free-surface lattice Boltzmann
 * method with bubble model (Anderl et al., "Free Surface Lattice Boltzmann with
 * Enhanced Bubble Model", arXiv:1604.01632).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA library
 * against an independent, slow, obviously correct implementation.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or constant with the CUDA path.
 *
 * Lattice: nx*ny*nz cells, linear index i = x + nx*(y + ny*z), every axis wraps
 * (walls are expressed as obstacle cells).  PDFs are stored [19][n].
 * Cell types: 0 liquid, 1 interface, 2 gas, 3 obstacle, 4 moving wall (lid).
 */
#ifndef FSL_ORACLE_H
#define FSL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ora_sim ora_sim;

typedef struct {
    int32_t nx, ny, nz;
    int32_t collision;      /* 0 BGK (omega_minus = omega_plus), 1 TRT */
    double tau;             /* omega_plus = 1/tau */
    double magic;           /* TRT magic parameter Lambda */
    double sigma;           /* surface tension (lattice units) */
    double g[3];            /* gravity (body force per unit density) */
    double eps;             /* conversion threshold */
    double lid[3];          /* moving-wall velocity (cell type 4) */
    int32_t normal_rule;    /* 1: also rebuild PDFs with n.c < 0; 0: gas links only */
    int32_t lonely_rule;    /* 1: interface cells without gas (liquid) neighbours fill (empty) */
} ora_params;

typedef struct {
    int64_t id;        /* canonical id: minimum linear index of the bubble's cells */
    int64_t vfx;       /* volume of the cells, fixed point 2^-32 */
    int64_t vxfx;      /* extra (reservoir) volume, fixed point 2^-32 */
    int64_t vsfx;      /* initial volume V*, fixed point 2^-32 */
    int64_t ncells;    /* gas + interface cells */
    int32_t constp;    /* constant-pressure (atmosphere) bubble */
    int32_t pad;
} ora_bubble;

ora_sim* ora_create(const ora_params* p);
void ora_destroy(ora_sim* s);
/* 0 on success, -2 if the geometry breaks the closed interface layer. */
int ora_init(ora_sim* s, const uint8_t* flags, const double* fill, const double* rho,
             const double* u /* [3][n] */);
int ora_set_source(ora_sim* s, int64_t seed_cell, double extra0, double rate, int32_t constp);
int ora_step(ora_sim* s, int64_t nsteps);
int ora_status(const ora_sim* s);

void ora_get_f(const ora_sim* s, double* out /* [19][n] */);
void ora_get_flags(const ora_sim* s, uint8_t* out);
void ora_get_phi(const ora_sim* s, double* out);
void ora_get_mass(const ora_sim* s, double* out);
void ora_get_ids(const ora_sim* s, int64_t* out);
int64_t ora_get_bubbles(const ora_sim* s, ora_bubble* out, int64_t cap);
double ora_bubble_pressure(const ora_bubble* b);
int64_t ora_pool_fx(const ora_sim* s);
int64_t ora_last_conversions(const ora_sim* s);

/* Building blocks exposed for the pins. */
void ora_lattice(int32_t* c /* [19][3] */, double* w /* [19] */, int32_t* opp /* [19] */);
void ora_feq(double rho, const double* u, double* out /* [19] */);
double ora_collide(const ora_params* p, const double* fin, double* fout);
void ora_label(const uint8_t* fg, int32_t nx, int32_t ny, int32_t nz, int64_t* label);
double ora_curvature(const ora_sim* s, int64_t i);
void ora_gradient(const ora_sim* s, int64_t i, double* g);

#ifdef __cplusplus
}
#endif
#endif
