/*
 * fsl.h -- C ABI of the GB300 (sm_103a) free-surface lattice Boltzmann library
 * with the enhanced bubble model of Anderl, Bogner, Rauh, Ruede and Delgado,
 * "Free Surface Lattice Boltzmann with Enhanced Bubble Model" (arXiv:1604.01632).
 *
 * One handle (fsl_domain) holds one or more independent lattices ("domains")
 * that advance together, one GPU, one CUDA stream.  All state lives in device
 * memory owned by the library; inputs are copied in, outputs copied out.
 *
 * Lattice conventions (every call):
 *   - domain d has nx*ny*nz cells; linear index i = x + nx*(y + ny*z); every
 *     axis wraps, walls are obstacle cells;
 *   - cell types (uint8): FSL_LIQUID, FSL_INTERFACE, FSL_GAS, FSL_OBSTACLE
 *     (no-slip wall), FSL_LID (wall moving at lid_velocity) -- paper Sec. 2.2,
 *     "Different cell types": only liquid and interface cells carry PDFs;
 *   - vector fields are structure-of-arrays: u[c*n + i], c = 0,1,2; PDF fields
 *     are f[a*n + i] in the D3Q19 order rest, +x, -x, +y, -y, +z, -z, then the
 *     (x,y), (x,z), (y,z) edge pairs with each direction followed by its
 *     opposite (paper Sec. 2.1, D3Q19).
 *
 * Errors: every call returns an fsl_status.  Errors found on the device
 * (NaN density, a broken interface layer, a full bubble table, a labelling pass
 * that did not converge) latch into a device status word that the next
 * synchronising call (fsl_sync, fsl_bubbles, fsl_fields) returns; the handle
 * stays usable for reading state.  No call throws; no device wait is
 * unbounded.  fsl_last_error() gives a one-line description.
 */
#ifndef FSL_H
#define FSL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fsl_domain fsl_domain;

typedef enum {
    FSL_OK = 0,
    FSL_ERR_ARG = -1,                 /* bad argument or call order */
    FSL_ERR_GEOMETRY = -2,            /* a liquid cell touches a gas cell */
    FSL_ERR_OOM = -3,                 /* device allocation failed */
    FSL_ERR_NAN = -4,                 /* a cell density became NaN */
    FSL_ERR_CCL_NOT_CONVERGED = -5,   /* union-find pass hit its iteration cap */
    FSL_ERR_TABLE_FULL = -6,          /* more bubbles than bubble_capacity */
    FSL_ERR_CUDA = -7,                /* a CUDA runtime call failed */
    FSL_ERR_SYNC = -8                 /* a grid barrier of the conversion kernel timed out */
} fsl_status;

enum { FSL_LIQUID = 0, FSL_INTERFACE = 1, FSL_GAS = 2, FSL_OBSTACLE = 3, FSL_LID = 4 };
enum { FSL_BGK = 0, FSL_TRT = 1 };

/* Storage precision of the PDFs.  FP64 collides in FP64; the others collide in
 * FP32.  The F16S/BF16S forms store the deviation f_a - w_a (rho0 = 1).  Mass,
 * fill level and every bubble quantity stay FP64 in all forms. */
typedef enum { FSL_P_FP64 = 0, FSL_P_FP32 = 1, FSL_P_F16S = 2, FSL_P_BF16S = 3 } fsl_precision;

/* Physical parameters of one domain, lattice units. */
typedef struct {
    int32_t nx, ny, nz;
    int32_t collision;        /* FSL_BGK or FSL_TRT (paper Sec. 2.1 uses BGK) */
    double tau;               /* relaxation time, omega+ = 1/tau (paper Eq. 6) */
    double magic;             /* TRT magic parameter Lambda, e.g. 3/16 */
    double sigma;             /* surface tension (paper Eq. 15) */
    double gravity[3];        /* body force per unit density, Guo forcing */
    double eps;               /* conversion threshold: filled m > (1+eps) rho, emptied m < -eps rho */
    double lid_velocity[3];   /* velocity of FSL_LID cells */
    int32_t normal_rule;      /* 1: also rebuild PDFs whose direction has n.c < 0 (paper Eq. 11 text) */
    int32_t bubble_capacity;  /* bubble-table slots for this domain; 0 = default */
    int32_t lonely_rule;      /* 1: an interface cell with no gas neighbour fills, one with no liquid
                                 neighbour empties (it no longer separates liquid from gas) */
    int32_t split_trigger;    /* when a bubble that loses a cell to the liquid is relabelled (a split
                                 is possible only then, paper Sec. 2.3.2): 0 = the removed cell's gas
                                 and interface neighbours are not connected inside its 3x3x3 cube
                                 (exact: never misses a split); 1 = the paper's trigger, two
                                 interface neighbours of its bubble with anti-parallel normals
                                 (n_i . n_j < -1/2), which relabels less often and can miss a
                                 split the local test would catch */
} fsl_params;

/* One bubble (paper Sec. 2.3): id = minimum linear index of its gas and
 * interface cells; volume = V(t) including extra_volume; init_volume = V*;
 * pressure = p_V of paper Eq. 13 (p0 = 1/3). */
typedef struct {
    int64_t id;
    double volume;
    double init_volume;
    double pressure;
    int64_t n_cells;
    int32_t const_pressure;
    int32_t pad;
    double extra_volume;
} fsl_bubble;

/* Field selectors for fsl_fields; dst[k] receives the k-th selected field in
 * this bit order. */
enum {
    FSL_F_FLAGS = 1,   /* uint8[n] */
    FSL_F_FILL = 2,    /* double[n], fill level phi (paper Eq. 9) */
    FSL_F_MASS = 4,    /* double[n], interface mass m (meaningful on interface cells) */
    FSL_F_ID = 8,      /* int64[n], bubble id of gas/interface cells, -1 elsewhere */
    FSL_F_RHO = 16,    /* double[n], density of the stored (post-collision) PDFs (Eq. 4) */
    FSL_F_U = 32,      /* double[3n], velocity of the stored PDFs (Eq. 5) */
    FSL_F_PDF = 64     /* double[19n], stored post-collision PDFs, unshifted */
};

/* Create a handle for n_domains independent domains; params[d] describes
 * domain d.  cuda_stream: the cudaStream_t every call enqueues on (NULL =
 * legacy default stream).  Allocates all device state.  FSL_ERR_ARG when a
 * parameter is out of range or the domains, each padded to a multiple of 256
 * cells, hold more than 226,050,910 cells together (19 PDFs per cell must be
 * addressable with 32-bit offsets). */
fsl_status fsl_create(const fsl_params* params, int32_t n_domains, int32_t precision,
                      void* cuda_stream, fsl_domain** out);

/* Load the initial state of domain d (paper Sec. 2.2): cell types, fill
 * levels (interface cells), density and velocity; f = f_eq(rho, u), m = phi
 * rho.  Pointers are host memory (on_device = 0) or device memory on the
 * handle's GPU (on_device = 1); the caller keeps them.  Host data pass through
 * a device staging buffer owned by the handle, allocated by fsl_create for the
 * largest domain's initial state (41 bytes per cell) and grown when a later
 * call needs more (FSL_ERR_CUDA when that fails); fill, rho and u in
 * page-locked host memory (all three) are read by the initialisation kernel in
 * place instead, and must hold their n (3n for u) values.  Rejects
 * (FSL_ERR_GEOMETRY) a liquid cell with a gas neighbour.  Every domain must be
 * initialised before the first step; bubbles are found (flood fill, paper Sec.
 * 2.3.2) with V* = V, p = p0.  Synchronises. */
fsl_status fsl_init_geometry(fsl_domain* h, int32_t d, const uint8_t* flags, const double* fill,
                             const double* rho, const double* u, int32_t on_device);

/* Attach a source to the bubble holding seed_cell of domain d: a reservoir of
 * extra volume extra0 that shrinks by rate per step (gas inflow, paper Sec.
 * 3.2), or a constant-pressure atmosphere (const_pressure = 1, p = p0).  Call
 * after fsl_init_geometry, before stepping.  One reservoir per domain. */
fsl_status fsl_set_bubble_source(fsl_domain* h, int32_t d, int64_t seed_cell, double extra0,
                                 double rate, int32_t const_pressure);

/* Advance every domain by nsteps time steps: stream/bounce-back, mass
 * exchange (paper Eq. 10), free-surface reconstruction (Eq. 11-15),
 * collision (Eq. 6), cell conversion with excess-mass redistribution, bubble
 * volume update, and merge/split detection by connected-component labelling
 * (Secs. 2.3.1, 2.3.2).  Asynchronous on the handle's stream. */
fsl_status fsl_step(fsl_domain* h, int64_t nsteps);

/* Wait for the stream and return the latched device status. */
fsl_status fsl_sync(fsl_domain* h);

/* Bubble table of domain d sorted by id; writes min(cap, count) records and
 * the number of bubbles to *count.  Synchronises. */
fsl_status fsl_bubbles(fsl_domain* h, int32_t d, fsl_bubble* out, int64_t cap, int64_t* count);

/* Copy the fields selected by mask of domain d into dst[0..] (one pointer per
 * selected field, in bit order; caller-owned), host memory (on_device = 0) or
 * device memory (on_device = 1).  Host copies go through the handle's device
 * staging buffer (grown when needed; FSL_ERR_CUDA when that fails).
 * Synchronises. */
fsl_status fsl_fields(fsl_domain* h, int32_t d, uint32_t mask, void* const* dst, int32_t on_device);

/* Liquid mass of domain d (paper Eq. 9 and the mass balance of Eq. 10):
 * the density of the stored PDFs summed over liquid cells, plus the mass m of
 * the interface cells, plus excess mass pooled and not yet shared out.  Summed
 * in a fixed order (the same value for the same state).  Synchronises. */
fsl_status fsl_total_mass(fsl_domain* h, int32_t d, double* mass);

/* Free the handle and its device memory. */
fsl_status fsl_destroy(fsl_domain* h);

/* Last error text of this handle ("" if none); valid until the next call. */
const char* fsl_last_error(const fsl_domain* h);

/* Number of kernels this handle has launched (graph replays count each of
 * their kernels). */
int64_t fsl_kernel_launches(const fsl_domain* h);

/* Number of merge/split labelling passes run since initialisation (the pass
 * runs only in steps whose conversions may have changed a bubble's
 * connectivity); synchronises.  -1 on error. */
int64_t fsl_labelling_runs(fsl_domain* h);

/* Number of bubbles those passes relabelled, summed over the passes after
 * initialisation (a pass takes only the bubbles that phase C marked as
 * possibly merged or split, and only their cells); synchronises.  -1 on
 * error. */
int64_t fsl_relabelled_bubbles(fsl_domain* h);

/* Device time of the stream-collide kernels of the steps run since timing was
 * switched on or since the previous fsl_sync, in milliseconds, summed over
 * those steps; fsl_sync evaluates it (0 when timing is off).  Timing is
 * switched on with fsl_set_timing(h, 1); it brackets each stream-collide
 * launch with CUDA events on the handle's stream. */
fsl_status fsl_set_timing(fsl_domain* h, int32_t on);
double fsl_stream_collide_ms(const fsl_domain* h);

/* on = 1 (default): fsl_step replays CUDA graphs of one or two steps; on = 0:
 * every kernel of a step is a separate launch (for per-phase timing and
 * profilers).  Results are identical. */
fsl_status fsl_set_graphs(fsl_domain* h, int32_t on);

/* Failure-path limits, for tests of the error reporting (0 restores a
 * default):
 *   ccl_max_iter   cap on the union / find loops of the labelling (default
 *                  2^24); a pass that reaches it latches
 *                  FSL_ERR_CCL_NOT_CONVERGED and leaves the bubble table of
 *                  the labelled domains unreliable;
 *   barrier_polls  polls a block of the conversion kernel makes at a grid
 *                  barrier before it latches FSL_ERR_SYNC and returns (default
 *                  2^22);
 *   barrier_absent 1 makes every grid barrier wait for one block more than
 *                  the grid holds, so that each wait runs out after
 *                  barrier_polls polls (0: normal barriers).
 * Waits for the handle's stream; the next fsl_step rebuilds its graphs.
 * FSL_ERR_ARG for values out of range. */
fsl_status fsl_set_limits(fsl_domain* h, int64_t ccl_max_iter, int64_t barrier_polls, int32_t barrier_absent);

/* Form of the stream-collide kernel (the same results in every form; each
 * cell runs the same arithmetic).  By default (form -1) the library tunes it:
 * the first fsl_step calls of a handle run real steps that each time one
 * candidate form (every usable form twice: the slab form only with the
 * interface list in cell order, the tile-fused forms not in FP64; direct
 * launches, the call waits for each), then keep the fastest and record it in a process-wide cache keyed by
 * precision, one or many domains, SM count, lattice size (log2 of the padded
 * cells) and interface share (1/64 steps); a later handle of the same key
 * takes the cached form without tuning.  Forms:
 *   0  split: blocks [0, 2 x SMs) take the interface list in 32-cell chunks
 *      (16 in FP64), the other blocks one liquid tile each;
 *   1, 2, 3  persistent: a resident grid walks one sequence of work items in
 *      which the interface chunks are spread evenly among liquid items of 1,
 *      2 or 4 tiles (a tile is 512 cells in the 16-bit forms, 256 otherwise);
 *   4  slab: each block of a resident grid owns a contiguous range of tiles
 *      and processes their liquid cells and the interface cells among them,
 *      interleaved (only with the interface list in cell order, see
 *      fsl_set_interface_order; FSL_ERR_ARG otherwise);
 *   5  two kernels: the liquid cells (a tile per block), then the interface
 *      cells one per thread with every direction unrolled;
 *   6, 7  tile-fused: each block takes 2 or 4 tiles, streams and collides
 *      their liquid cells, then their interface cells one per thread (FP32
 *      and 16-bit storage only; FSL_ERR_ARG for FP64);
 *   8  the two kernels of form 5 side by side: the interface kernel on a
 *      second stream of the handle with half its resident blocks per SM,
 *      the liquid kernel beside it, joined before the conversion.
 * Forms 5-8 first run a normals pass (one kernel over the lattice) that
 * stores the unit normal of every interface cell and face neighbour of one
 * and each interface cell's reconstruction directions; their interface cells
 * read the curvature's normals from it.  Kernels per step: 4 in forms 5 and
 * 8, 3 in forms 6 and 7, 2 otherwise (the conversion kernel included).
 * -1 restarts the tuning.  Waits for the handle's stream; the next fsl_step
 * rebuilds its graphs.  FSL_ERR_ARG for another value.  fsl_stream_form
 * returns the form in use (the one tried next while tuning). */
fsl_status fsl_set_stream_form(fsl_domain* h, int32_t form);
int32_t fsl_stream_form(const fsl_domain* h);

/* Autotuner record of the handle: ms_per_form (array of 9, may be NULL) the
 * fastest stream-collide time measured per form (0 = not run); *form the
 * chosen form (-1 while tuning); *source 0 = not decided, 1 = measured on
 * this handle, 2 = from the process cache, 3 = set by the caller. */
fsl_status fsl_tuning(const fsl_domain* h, double* ms_per_form, int32_t* form, int32_t* source);

/* Empty the process-wide tuning cache. */
fsl_status fsl_forget_tuning(void);

/* Order of the interface list the stream-collide kernel walks: 1 = rebuilt
 * after each step's conversion in increasing cell index (two passes over the
 * cell types), 0 = in the order the conversion kernel appends it, -1 (default)
 * = 1 where the two PDF arrays exceed twice the L2 cache.  The same results in
 * every mode.  Waits for the handle's stream; FSL_ERR_ARG for another value.
 * fsl_interface_order returns the mode in effect (0 or 1). */
fsl_status fsl_set_interface_order(fsl_domain* h, int32_t mode);
int32_t fsl_interface_order(const fsl_domain* h);

/* Device time per phase of the steps timed since fsl_set_timing(h, 1), summed,
 * in milliseconds, when the handle runs without graphs (fsl_set_graphs(h, 0)):
 * out (array of 4): [0] stream-collide kernel (liquid and interface cells in
 * one launch), [1] and [2] start of the step to the end of that kernel (one
 * entry each for its liquid and interface cells, which end together), [3] cell
 * conversion and, on steps that set a merge / split trigger, the labelling
 * (one cooperative kernel).  Read after fsl_sync. */
fsl_status fsl_phase_ms(const fsl_domain* h, double* out);

/* Counts of the cell types of domain d (array of 5), synchronises. */
fsl_status fsl_cell_counts(fsl_domain* h, int32_t d, int64_t* counts);

/* Allocation-free bubble labelling.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory (latency-critical
 * loops in which an allocation may synchronise the device, deployments that
 * give all device memory to their own pool, host frameworks that forbid a
 * library to allocate).  It labels the connected components of the gas and
 * interface cells of one lattice under the 18-neighbourhood with every axis
 * wrapping, label = minimum linear index of the component, -1 elsewhere: the
 * same labels fsl_fields(FSL_F_ID) reports after fsl_init_geometry.
 *   flags  : device pointer, uint8[nx*ny*nz] cell types (bits above the type
 *            are ignored), read only;
 *   labels : device pointer, int64[nx*ny*nz], written;
 *   cuda_stream : stream the three kernels are enqueued on (NULL = legacy
 *            default stream); the call returns without waiting.
 * It calls no allocator: its scratch is a fixed array of 2^21 int32 labels
 * (8 MiB) compiled into the library, held by every GPU that loads it until the
 * process exits.  nx*ny*nz above 2^21 returns FSL_ERR_ARG.  The first call on
 * a device looks up the scratch's device address (cudaGetSymbolAddress with
 * that device current) and caches it for the life of the process (safe from
 * several host threads); make that first call before any stream capture.  A
 * cudaDeviceReset invalidates the cached address: do not call this entry
 * point on a device after resetting it.  All calls on a device share the scratch, and each call rewrites it
 * from the start; calls whose kernels overlap on the GPU (different streams,
 * not ordered) race and give wrong labels. */
fsl_status fsl_label_bubbles_static(const uint8_t* flags, int32_t nx, int32_t ny, int32_t nz, int64_t* labels,
                                    void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
