// fsl_device.cuh -- device-side definitions of the GB300 FSLBM library:
// lattice constants, cell/mark codes, per-domain descriptors, PDF storage
// forms, the stream-collide kernels, the cooperative conversion kernel and
// the labelling phases, templated on the storage form where they differ.
//
// Method: Anderl et al., arXiv:1604.01632.  Equation numbers count the
// paper's displayed equations in order (Eq. 3 equilibrium, Eqs. 4-5 moments,
// Eq. 6 collision, Eq. 7 streaming, Eq. 8 p = rho c_s^2, Eq. 9 m = phi rho,
// Eq. 10 mass exchange, Eq. 11 reconstruction, Eq. 12 p_gas = p_V + dp,
// Eq. 13 p_V = p0 V*/V, Eq. 15 dp = 2 sigma kappa).
//
// Layout in HBM: every per-cell array is indexed by a global cell number g;
// domain d owns cells [off_d, off_d + n_d) in x-fastest order, padded to a
// multiple of FSL_BLOCK cells with obstacle cells that belong to no lattice.
// PDFs are structure-of-arrays, f[a * stride + g].
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <limits.h>
#include <stdint.h>

#define FSL_BLOCK 256
#define FSL_CONV_THREADS 256   // block of the cooperative conversion kernel

namespace fsl {

// Cell types live in bits 0-2 of the flag byte; bit 3 (K_WALL) marks a cell
// with an obstacle or lid among its 18 neighbours (walls never change).
enum : uint8_t { LIQ = 0, IFC = 1, GAS = 2, OBS = 3, LID = 4 };
enum : uint8_t { K_TYPE = 7, K_WALL = 8 };
__host__ __device__ inline uint8_t ctype(uint8_t f) { return (uint8_t)(f & K_TYPE); }
// Conversion marks (paper Sec. 2.2, cell conversion).  K1 writes NONE /
// FILLED / EMPTIED on interface cells; phase A writes NEWG on gas cells and
// clears EMPTIED next to FILLED; phase B writes NEWL / NONE on liquid cells;
// phase C turns FILLED / EMPTIED into CFILLED / CEMPTIED (same meaning).
enum : uint8_t { MK_NONE = 0, MK_FILLED = 1, MK_EMPTIED = 2, MK_NEWG = 3, MK_NEWL = 4,
                 MK_CFILLED = 5, MK_CEMPTIED = 6 };

// status codes latched by kernels (same values as fsl_status)
enum { ST_GEOMETRY = -2, ST_NAN = -4, ST_CCL = -5, ST_TABLE_FULL = -6, ST_SYNC = -8 };

// Fixed-point scales: bubble volumes 2^-32 cells^3, pooled mass 2^-40.
#define FSL_VOL_ONE 4294967296LL

struct Dom {
    int nx, ny, nz, n;          // lattice dims, n = nx*ny*nz
    long long off;              // first global cell
    int slot_off, slot_cap;     // bubble-table slot range
    int seed;                   // reservoir seed cell (local index), -1 none
    int normal_rule;
    long long rate_fx;          // reservoir drain per step, fixed point
    double omp, omm;            // omega+ = 1/tau, omega- (TRT) or omega+ (BGK)
    double sigma2;              // 2 sigma
    double g[3];                // gravity
    double eps;                 // conversion threshold
    double lid[3];              // lid velocity
    unsigned mgx, mgy;          // x = l - nx*(l/nx) etc. by multiply-high: l/nx = umulhi(l, mgx) >> shx
    int shx, shy;               // (shift -1: the divisor is 1)
    int has_force;              // gravity is not zero
    int lonely_rule;            // interface cells without gas / liquid neighbours fill / empty
    int split_trigger;          // 0: exact local test, 1: anti-parallel normals (the paper's)
    // the same parameters rounded to FP32 once on the host: the FP32-collide
    // kernels read these, so that no thread converts from FP64 (the FP64 pipe
    // is a small fraction of the FP32 rate on this GPU)
    float fomp, fomm, fsigma2, fg[3], flid[3], feps;
};

// Relaxation rates, 2 sigma, gravity and lid velocity in the arithmetic type C.
template <typename C> struct Par {
    C omp, omm, sigma2, g[3], lid[3];
};
template <typename C> __device__ inline Par<C> par_of(const Dom& D) {
    Par<C> P;
    if constexpr (sizeof(C) == 8) {
        P.omp = D.omp; P.omm = D.omm; P.sigma2 = D.sigma2;
        for (int k = 0; k < 3; ++k) { P.g[k] = D.g[k]; P.lid[k] = D.lid[k]; }
    } else {
        P.omp = D.fomp; P.omm = D.fomm; P.sigma2 = D.fsigma2;
        for (int k = 0; k < 3; ++k) { P.g[k] = D.fg[k]; P.lid[k] = D.flid[k]; }
    }
    return P;
}

// Invariant-divisor division for 0 <= n < 2^31: with s = ceil(log2 d) and
// m = ceil(2^(31+s) / d) < 2^32, n / d = (n * m) >> (31 + s) (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994).
__host__ inline void div_magic(int d, unsigned& m, int& sh) {
    int s = 0;
    while ((1LL << s) < d) ++s;
    const unsigned long long num = 1ULL << (31 + s);
    m = (unsigned)((num + (unsigned long long)d - 1) / (unsigned long long)d);
    sh = s - 1;
}
__device__ inline int fast_div(int n, unsigned m, int sh) {
    return sh < 0 ? n : (int)(__umulhi((unsigned)n, m) >> sh);
}
__device__ inline void local_xyz(const Dom& D, int l, int& x, int& y, int& z) {
    const int q = fast_div(l, D.mgx, D.shx);
    x = l - q * D.nx;
    z = fast_div(q, D.mgy, D.shy);
    y = q - z * D.ny;
}

// Everything a step kernel needs, passed by value.
struct StepArgs {
    const Dom* doms;
    const int* blk_dom;         // block -> domain
    const int4* ntiles;         // normals pass of a batch: (domain, x0, y0, z0) per tile, or null
                                // when a domain is smaller than a tile
    int nntiles;
    long long stride;           // cells in the padded global lattice
    const void* fsrc;           // PDFs after the previous step (post-collision)
    void* fdst;                 // PDFs written by this step
    uint8_t* flag;
    uint8_t* mark;
    double* m;                  // interface mass
    double* phi;                // fill level
    double* phit;               // fill level as the normal stencil reads it: walls and
                                // liquid 1, gas 0, interface clamp(phi, 0, 1)
    float* phif;                // FP32 copies of phi and phit for the FP32-collide
    float* phitf;               // forms (null for the FP64 form)
    double* rhoi;               // density of interface cells at their last collision
    double* exs;                // excess-mass share of converted cells
    int* id;                    // bubble slot of gas/interface cells, -1 elsewhere
    long long* vfx;             // bubble volume of the cells (slot)
    long long* vxfx;            // bubble extra volume (slot)
    const long long* vsfx;      // bubble V* (slot)
    long long* ncells;          // bubble cell count (slot)
    const int* constp;          // bubble constant-pressure flag (slot)
    long long* pool;            // per-domain pooled excess mass, fixed point 2^-40
    long long* nif;             // per-domain interface count after conversion
    int* trig;                  // merge/split trigger: [0] any domain, [1 + d] domain d
    int* status;
    int ndom;
    int* ilist;                 // interface cells at the start of this step
    int* icount;
    int* ilist_next;            // interface cells after this step's conversion (phase D)
    int* icount_next;
    int* mlist;                 // interface cells marked filled / emptied (interface kernel)
    int* mcount;
    int* glist;                 // gas cells that become interface (phase A)
    int* gcount;
    int* llist;                 // liquid cells that become interface (phase B)
    int* lcount;
    int* cstep;                 // step number at which each cell was last converted
    int* recv;                  // step number at which each cell last received excess mass
    int* stepno;                // device step counter
    long long* icnt;            // per-domain interface count at the end of the step
    unsigned* bar;              // grid barrier of the conversion kernel: count, generation
    int order;                  // 1: the conversion kernel rebuilds the next interface list in
                                // cell order (after phase D), 0: phase D appends it
    int* ocnt;                  // interface cells per conversion block (ordered rebuild)
    int spins;                  // polls a block waits at a grid barrier before it gives up
    int bar_extra;              // arrivals a barrier waits for beyond the grid (0; 1 only to
                                // test the timeout path: no block is then the last)
    int* bbox;                  // per bubble slot: the box [6 s .. 6 s + 2] min x, y, z and
                                // [6 s + 3 .. 6 s + 5] max x, y, z (domain coordinates) that holds
                                // all of its cells; a box spanning a periodic seam is the full axis
    void* nrm;                  // normals pass: unit normals of the cells that need one,
                                // three planes of the arithmetic type (x, y, z), stride apart
    unsigned* nmask;            // normals pass: per interface cell, bit a set when the
                                // reconstruction's normal test holds for direction a
    void* pvc;                  // normals pass: per interface cell, its bubble's pressure
                                // p_V (Eq. 13) in the arithmetic type
    Dom d0;                     // domain 0, read from the parameter space when ndom == 1
};

// Domain descriptor and domain of a cell: a handle with one domain reads
// them from the kernel parameters, a batch from its device tables.
// (the device table holds every domain, the single one too; reading fields
// through the reference loads only those fields, where a copy of a descriptor
// chosen at run time would go through local memory)
__device__ inline const Dom& get_dom(const StepArgs& A, int d) { return A.doms[d]; }
__device__ inline int block_dom(const StepArgs& A, long long g) { return A.ndom == 1 ? 0 : A.blk_dom[g / FSL_BLOCK]; }
// The same for the hot kernels, which exist once for a single domain (ONE:
// the descriptor is read straight from the kernel parameters) and once for a
// batch (read from the device table), so that no thread copies a descriptor
// chosen at run time.
template <bool ONE>
__device__ inline const Dom& dom_at(const StepArgs& A, long long g) {
    if constexpr (ONE) return A.d0;
    else return A.doms[A.blk_dom[g / FSL_BLOCK]];
}

// D3Q19 velocities; constexpr so that unrolled loops fold them into offsets
__host__ __device__ constexpr int cx(int a) {
    return (a == 1 || a == 7 || a == 9 || a == 11 || a == 13) ? 1
           : ((a == 2 || a == 8 || a == 10 || a == 12 || a == 14) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int a) {
    return (a == 3 || a == 7 || a == 10 || a == 15 || a == 17) ? 1
           : ((a == 4 || a == 8 || a == 9 || a == 16 || a == 18) ? -1 : 0);
}
__host__ __device__ constexpr int cz(int a) {
    return (a == 5 || a == 11 || a == 14 || a == 15 || a == 18) ? 1
           : ((a == 6 || a == 12 || a == 13 || a == 16 || a == 17) ? -1 : 0);
}

// the same velocities for a run-time direction: two bits (c + 1) per direction
__device__ inline int rcx(int a) { return (int)((0x1548889549ULL >> (2 * a)) & 3) - 1; }
__device__ inline int rcy(int a) { return (int)((0x895609495ULL >> (2 * a)) & 3) - 1; }
__device__ inline int rcz(int a) { return (int)((0x20a0954955ULL >> (2 * a)) & 3) - 1; }

__host__ __device__ inline int opp(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }
__host__ __device__ inline double weight(int a) {
    return a == 0 ? 1.0 / 3.0 : (a <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}
// the same weights in the arithmetic type C (for C = float the FP32 roundings
// of the FP64 constants, folded at compile time)
template <typename C> __host__ __device__ inline C weightc(int a) {
    return a == 0 ? (C)(1.0 / 3.0) : (a <= 6 ? (C)(1.0 / 18.0) : (C)(1.0 / 36.0));
}

__device__ inline void set_status(int* st, int code) { atomicCAS(st, 0, code); }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation waits here until its predecessor has finished and its writes
// are visible; a predecessor lets its dependent start launching early.
__device__ inline void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ inline void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch a kernel whose predecessor on the stream is a kernel, overlapping its
// launch with the predecessor's tail (the kernel must call pdl_wait() first).
template <typename... Args>
inline cudaError_t launch_pdl(void (*k)(Args...), unsigned grid, unsigned block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// Append v to list for every lane with pred set, one atomic per warp.  Every
// lane of the warp must call.
// Grow bubble slot b's box to hold the cell (x, y, z).
__device__ inline void bbox_extend(int* bbox, int b, int x, int y, int z) {
    if (b < 0) return;
    int* q = bbox + 6 * (long long)b;
    atomicMin(q + 0, x); atomicMin(q + 1, y); atomicMin(q + 2, z);
    atomicMax(q + 3, x); atomicMax(q + 4, y); atomicMax(q + 5, z);
}

__device__ inline void list_append(int* list, int* count, bool pred, int v) {
    const unsigned full = 0xffffffffu;
    const unsigned m = __ballot_sync(full, pred);
    if (m == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(full, base, leader);
    if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = v;
}

// ------------------------------------------------------------ cell geometry

// Coordinates of a cell and wrapped neighbour indices inside its domain.
struct Cell {
    int x, y, z;
    int nx, ny, nz;
    long long off;
    __device__ inline long long at(int dx, int dy, int dz) const {
        int xx = x + dx, yy = y + dy, zz = z + dz;
        xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
        yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
        zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
        return off + (long long)xx + (long long)nx * ((long long)yy + (long long)ny * zz);
    }
    // any offset (used by the 5x5x5 curvature stencil on tiny lattices too)
    __device__ inline long long at_far(int dx, int dy, int dz) const {
        int xx = ((x + dx) % nx + nx) % nx;
        int yy = ((y + dy) % ny + ny) % ny;
        int zz = ((z + dz) % nz + nz) % nz;
        return off + (long long)xx + (long long)nx * ((long long)yy + (long long)ny * zz);
    }
};

__device__ inline Cell make_cell(const Dom& D, long long g) {
    Cell c;
    c.nx = D.nx; c.ny = D.ny; c.nz = D.nz; c.off = D.off;
    local_xyz(D, (int)(g - D.off), c.x, c.y, c.z);
    return c;
}

// ------------------------------------------------------------ storage forms

template <typename T> struct Form;
template <> struct Form<double> {
    using C = double;
    static constexpr bool shifted = false;
    __device__ static inline double ld(const double* p, int) { return *p; }
    __device__ static inline void st(double* p, int, double v) { *p = v; }
};
template <> struct Form<float> {
    using C = float;
    static constexpr bool shifted = false;
    __device__ static inline float ld(const float* p, int) { return *p; }
    __device__ static inline void st(float* p, int, float v) { *p = v; }
};
// shifted forms store f_a - w_a (rho0 = 1)
template <> struct Form<__half> {
    using C = float;
    static constexpr bool shifted = true;
    __device__ static inline float ld_dev(const __half* p) { return __half2float(*p); }
    __device__ static inline void st_dev2(__half* p, float2 v) { *(__half2*)p = __floats2half2_rn(v.x, v.y); }
    __device__ static inline float2 ld_dev2(const __half* p) { return __half22float2(*(const __half2*)p); }
    __device__ static inline void st_dev(__half* p, float v) { *p = __float2half_rn(v); }
    // the pair rounded once; stored whole, or only its low / high half
    __device__ static inline void st_dev2m(__half* p, float2 v, bool both, bool lo, bool hi) {
        const __half2 h = __floats2half2_rn(v.x, v.y);
        if (both) *(__half2*)p = h;
        if (lo) p[0] = __low2half(h);
        if (hi) p[1] = __high2half(h);
    }
    __device__ static inline float ld(const __half* p, int a) { return weightc<float>(a) + __half2float(*p); }
    __device__ static inline void st(__half* p, int a, float v) { *p = __float2half_rn(v - weightc<float>(a)); }
};
template <> struct Form<__nv_bfloat16> {
    using C = float;
    static constexpr bool shifted = true;
    __device__ static inline float ld_dev(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    __device__ static inline void st_dev2(__nv_bfloat16* p, float2 v) { *(__nv_bfloat162*)p = __floats2bfloat162_rn(v.x, v.y); }
    __device__ static inline float2 ld_dev2(const __nv_bfloat16* p) { return __bfloat1622float2(*(const __nv_bfloat162*)p); }
    __device__ static inline void st_dev(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
    __device__ static inline void st_dev2m(__nv_bfloat16* p, float2 v, bool both, bool lo, bool hi) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        if (both) *(__nv_bfloat162*)p = h;
        if (lo) p[0] = __low2bfloat16(h);
        if (hi) p[1] = __high2bfloat16(h);
    }
    __device__ static inline float ld(const __nv_bfloat16* p, int a) {
        return weightc<float>(a) + __bfloat162float(*p);
    }
    __device__ static inline void st(__nv_bfloat16* p, int a, float v) {
        *p = __float2bfloat16_rn(v - weightc<float>(a));
    }
};

// ---------------------------------------------------------- LBM arithmetic
// Written operation by operation in the same order as the oracle so that the
// FP64 path (compiled without FMA contraction) rounds identically.

template <typename C>
__device__ inline C cdot(int a, C vx, C vy, C vz) {
    return ((C)cx(a) * vx + (C)cy(a) * vy) + (C)cz(a) * vz;
}

// Moments (Eqs. 4-5).
template <typename C>
__device__ inline void moments(const C* f, C& rho, C& jx, C& jy, C& jz) {
    C r = f[0];
#pragma unroll
    for (int a = 1; a < 19; ++a) r = r + f[a];
    rho = r;
    jx = f[1] - f[2] + f[7] - f[8] + f[9] - f[10] + f[11] - f[12] + f[13] - f[14];
    jy = f[3] - f[4] + f[7] - f[8] - f[9] + f[10] + f[15] - f[16] + f[17] - f[18];
    jz = f[5] - f[6] + f[11] - f[12] - f[13] + f[14] + f[15] - f[16] - f[17] + f[18];
}

// Equilibrium (Eq. 3), symmetric part +/- antisymmetric part per pair.
template <typename C>
__device__ inline void feq_all(C rho, C ux, C uy, C uz, C* out) {
    C usq = ux * ux + uy * uy + uz * uz;
    out[0] = (weightc<C>(0) * rho) * ((C)1 - (C)1.5 * usq);
#pragma unroll
    for (int a = 1; a < 19; a += 2) {
        C cu = cdot<C>(a, ux, uy, uz);
        C wr = weightc<C>(a) * rho;
        C fp = wr * (((C)1 + (C)4.5 * (cu * cu)) - (C)1.5 * usq);
        C fm = wr * ((C)3 * cu);
        out[a] = fp + fm;
        out[a + 1] = fp - fm;
    }
}

// Two-relaxation-time collision with Guo forcing (Eq. 6); returns rho.
// Without a force every forcing term is an exact zero, so the FORCE = false
// form drops them (same results).  The FP32 form multiplies by 1/rho.
template <typename C, bool FORCE>
__device__ inline C collide(const C* fin, C* fout, C omp, C omm, C gx, C gy, C gz) {
    C rho, jx, jy, jz;
    moments<C>(fin, rho, jx, jy, jz);
    C Fx = (C)0, Fy = (C)0, Fz = (C)0;
    C ux, uy, uz;
    if constexpr (FORCE) {
        Fx = rho * gx; Fy = rho * gy; Fz = rho * gz;
        jx = jx + (C)0.5 * Fx;
        jy = jy + (C)0.5 * Fy;
        jz = jz + (C)0.5 * Fz;
    }
    if constexpr (sizeof(C) == 4) {
        const C ir = (C)1 / rho;
        ux = jx * ir; uy = jy * ir; uz = jz * ir;
    } else {
        ux = jx / rho; uy = jy / rho; uz = jz / rho;
    }
    const C usq = ux * ux + uy * uy + uz * uz;
    const C cp = (C)1 - (C)0.5 * omp, cm = (C)1 - (C)0.5 * omm;
    const C feq0 = (weightc<C>(0) * rho) * ((C)1 - (C)1.5 * usq);
    fout[0] = fin[0] - omp * (fin[0] - feq0);
    C uF = (C)0;
    if constexpr (FORCE) {
        uF = ux * Fx + uy * Fy + uz * Fz;
        const C S0 = weightc<C>(0) * ((C)-3 * uF);
        fout[0] = fout[0] + cp * S0;
    }
#pragma unroll
    for (int a = 1; a < 19; a += 2) {
        const int b = a + 1;
        const C w = weightc<C>(a);
        const C cu = cdot<C>(a, ux, uy, uz);
        const C wr = w * rho;
        const C feqp = wr * (((C)1 + (C)4.5 * (cu * cu)) - (C)1.5 * usq);
        const C feqm = wr * ((C)3 * cu);
        const C fp = (C)0.5 * (fin[a] + fin[b]);
        const C fm = (C)0.5 * (fin[a] - fin[b]);
        const C A = omp * (fp - feqp);
        const C B = omm * (fm - feqm);
        fout[a] = (fin[a] - A) - B;
        fout[b] = (fin[b] - A) + B;
        if constexpr (FORCE) {
            const C cF = cdot<C>(a, Fx, Fy, Fz);
            const C Sp = w * (((C)9 * cu) * cF - (C)3 * uF);
            const C Sm = w * ((C)3 * cF);
            const C sp = cp * Sp, sm = cm * Sm;
            fout[a] = (fout[a] + sp) + sm;
            fout[b] = (fout[b] + sp) - sm;
        }
    }
    return rho;
}

// The same collision on deviations d_a = f_a - w_a (rho0 = 1), for the
// shifted 16-bit storage forms: rho = 1 + sum d, j = sum c d, and
// d_eq = f_eq - w = w [(rho - 1) + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u.u)].
template <bool FORCE>
__device__ inline void collide_dev(const float* d, float* dout, float omp, float omm, float gx, float gy, float gz) {
    float drho = d[0];
#pragma unroll
    for (int a = 1; a < 19; ++a) drho += d[a];
    const float rho = 1.f + drho;
    float jx = d[1] - d[2] + d[7] - d[8] + d[9] - d[10] + d[11] - d[12] + d[13] - d[14];
    float jy = d[3] - d[4] + d[7] - d[8] - d[9] + d[10] + d[15] - d[16] + d[17] - d[18];
    float jz = d[5] - d[6] + d[11] - d[12] - d[13] + d[14] + d[15] - d[16] - d[17] + d[18];
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    if constexpr (FORCE) {
        Fx = rho * gx; Fy = rho * gy; Fz = rho * gz;
        jx += 0.5f * Fx; jy += 0.5f * Fy; jz += 0.5f * Fz;
    }
    const float ir = 1.f / rho;
    const float ux = jx * ir, uy = jy * ir, uz = jz * ir;
    const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
    const float cp = 1.f - 0.5f * omp, cm = 1.f - 0.5f * omm;
    const float w0 = weightc<float>(0);
    dout[0] = d[0] - omp * (d[0] - w0 * (drho - rho * usq15));
    float uF = 0.f;
    if constexpr (FORCE) {
        uF = ux * Fx + uy * Fy + uz * Fz;
        dout[0] += cp * (w0 * (-3.f * uF));
    }
#pragma unroll
    for (int a = 1; a < 19; a += 2) {
        const int b = a + 1;
        const float w = weightc<float>(a);
        const float cu = cdot<float>(a, ux, uy, uz);
        const float eqp = w * (drho + rho * (4.5f * cu * cu - usq15));
        const float eqm = w * rho * 3.f * cu;
        const float A = omp * (0.5f * (d[a] + d[b]) - eqp);
        const float B = omm * (0.5f * (d[a] - d[b]) - eqm);
        dout[a] = d[a] - A - B;
        dout[b] = d[b] - A + B;
        if constexpr (FORCE) {
            const float cF = cdot<float>(a, Fx, Fy, Fz);
            const float sp = cp * (w * (9.f * cu * cF - 3.f * uF));
            const float sm = cm * (w * 3.f * cF);
            dout[a] += sp + sm;
            dout[b] += sp - sm;
        }
    }
}

// Packed FP32 (two cells in one float2, Blackwell's paired FP32 add / mul /
// fma): collide_dev for two cells at once, the same formulas with the
// operations regrouped for fused multiply-adds.
__device__ __forceinline__ float2 p2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p2sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 p2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p2(float x) { return make_float2(x, x); }

// c_a . v for an odd direction a (its first non-zero component is +1)
template <int a>
__device__ __forceinline__ float2 cdot2(float2 vx, float2 vy, float2 vz) {
    constexpr int X = cx(a), Y = cy(a), Z = cz(a);
    if constexpr (X != 0) {
        if constexpr (Y > 0) return p2add(vx, vy);
        else if constexpr (Y < 0) return p2sub(vx, vy);
        else if constexpr (Z > 0) return p2add(vx, vz);
        else if constexpr (Z < 0) return p2sub(vx, vz);
        else return vx;
    } else if constexpr (Y != 0) {
        if constexpr (Z > 0) return p2add(vy, vz);
        else if constexpr (Z < 0) return p2sub(vy, vz);
        else return vy;
    } else {
        return vz;
    }
}

struct Collide2 {
    float2 ux, uy, uz, drho, rho, nusq15, hp, hm, Fx, Fy, Fz, uF;
};

// One TRT pair (a, a+1) of two cells; w = w_a, cp/cm the forcing prefactors;
// out(a, value) receives each output as soon as it is formed.
template <int a, bool FORCE, class Out>
__device__ __forceinline__ void trt_pair2(const float2* d, Out&& out, const Collide2& K, float omp, float omm,
                                          float w, float cp, float cm) {
    constexpr int b = a + 1;
    const float2 cu = cdot2<a>(K.ux, K.uy, K.uz);
    // f_eq+ - w = w [drho + rho (9/2 (c.u)^2 - 3/2 u.u)],  A = omp (f+ - f_eq+)
    float2 t = p2fma(p2mul(p2(4.5f), cu), cu, K.nusq15);
    t = p2fma(K.rho, t, K.drho);
    const float2 A = p2fma(K.hp, p2add(d[a], d[b]), p2mul(p2(-omp * w), t));
    // f_eq- = 3 w rho c.u,  B = omm (f- - f_eq-)
    const float2 B = p2fma(K.hm, p2sub(d[a], d[b]), p2mul(p2mul(K.rho, p2(-omm * 3.f * w)), cu));
    float2 oa = p2sub(d[a], p2add(A, B));
    float2 ob = p2sub(d[b], p2sub(A, B));
    if constexpr (FORCE) {
        const float2 cF = cdot2<a>(K.Fx, K.Fy, K.Fz);
        const float2 sp = p2fma(p2(9.f * cp * w), p2mul(cu, cF), p2mul(p2(-3.f * cp * w), K.uF));
        const float2 sm = p2mul(p2(3.f * cm * w), cF);
        oa = p2add(oa, p2add(sp, sm));
        ob = p2add(ob, p2sub(sp, sm));
    }
    out(a, oa);
    out(b, ob);
}

// The outputs go to out(a, value) in the order 0, 1, 2, ..., 18 (so that the
// caller can store them without holding all nineteen).
template <bool FORCE, class Out>
__device__ __forceinline__ void collide_dev2(const float2* d, Out&& out, float omp, float omm, float gx, float gy,
                                             float gz) {
    Collide2 K;
    K.drho = p2add(p2add(p2add(p2add(d[0], d[1]), p2add(d[2], d[3])), p2add(p2add(d[4], d[5]), p2add(d[6], d[7]))),
                   p2add(p2add(p2add(p2add(d[8], d[9]), p2add(d[10], d[11])),
                               p2add(p2add(d[12], d[13]), p2add(d[14], d[15]))),
                         p2add(p2add(d[16], d[17]), d[18])));
    K.rho = p2add(K.drho, p2(1.f));
    const float2 e78 = p2sub(d[7], d[8]), e1112 = p2sub(d[11], d[12]), e1516 = p2sub(d[15], d[16]);
    float2 jx = p2add(p2add(p2add(p2sub(d[1], d[2]), e78), p2add(p2sub(d[9], d[10]), e1112)), p2sub(d[13], d[14]));
    float2 jy = p2add(p2add(p2add(p2sub(d[3], d[4]), e78), p2add(p2sub(d[10], d[9]), e1516)), p2sub(d[17], d[18]));
    float2 jz = p2add(p2add(p2add(p2sub(d[5], d[6]), e1112), p2add(p2sub(d[14], d[13]), e1516)), p2sub(d[18], d[17]));
    K.Fx = p2(0.f); K.Fy = p2(0.f); K.Fz = p2(0.f); K.uF = p2(0.f);
    if constexpr (FORCE) {
        K.Fx = p2mul(K.rho, p2(gx)); K.Fy = p2mul(K.rho, p2(gy)); K.Fz = p2mul(K.rho, p2(gz));
        jx = p2fma(p2(0.5f), K.Fx, jx);
        jy = p2fma(p2(0.5f), K.Fy, jy);
        jz = p2fma(p2(0.5f), K.Fz, jz);
    }
    // 1 / rho by the fast reciprocal (within 2 ulp of FP32; the 16-bit storage
    // these forms serve rounds the deviations to 11 or 8 bits)
    const float2 ir = make_float2(__fdividef(1.f, K.rho.x), __fdividef(1.f, K.rho.y));
    K.ux = p2mul(jx, ir); K.uy = p2mul(jy, ir); K.uz = p2mul(jz, ir);
    K.nusq15 = p2mul(p2fma(K.uz, K.uz, p2fma(K.uy, K.uy, p2mul(K.ux, K.ux))), p2(-1.5f));
    if constexpr (FORCE) K.uF = p2fma(K.uz, K.Fz, p2fma(K.uy, K.Fy, p2mul(K.ux, K.Fx)));
    K.hp = p2(0.5f * omp);
    K.hm = p2(0.5f * omm);
    const float cp = 1.f - 0.5f * omp, cm = 1.f - 0.5f * omm;
    const float w0 = weightc<float>(0), w1 = weightc<float>(1), w2 = weightc<float>(7);
    {
        // rest direction: d0 - omp (d0 - w0 (drho - rho 3/2 u.u))
        const float2 t = p2fma(K.rho, K.nusq15, K.drho);
        float2 o0 = p2fma(p2(-omp), p2sub(d[0], p2mul(p2(w0), t)), d[0]);
        if constexpr (FORCE) o0 = p2fma(p2(cp * w0 * -3.f), K.uF, o0);
        out(0, o0);
    }
    trt_pair2<1, FORCE>(d, out, K, omp, omm, w1, cp, cm);
    trt_pair2<3, FORCE>(d, out, K, omp, omm, w1, cp, cm);
    trt_pair2<5, FORCE>(d, out, K, omp, omm, w1, cp, cm);
    trt_pair2<7, FORCE>(d, out, K, omp, omm, w2, cp, cm);
    trt_pair2<9, FORCE>(d, out, K, omp, omm, w2, cp, cm);
    trt_pair2<11, FORCE>(d, out, K, omp, omm, w2, cp, cm);
    trt_pair2<13, FORCE>(d, out, K, omp, omm, w2, cp, cm);
    trt_pair2<15, FORCE>(d, out, K, omp, omm, w2, cp, cm);
    trt_pair2<17, FORCE>(d, out, K, omp, omm, w2, cp, cm);
}

template <typename C>
__device__ inline C collide_any(bool force, const C* fin, C* fout, C omp, C omm, C gx, C gy, C gz) {
    return force ? collide<C, true>(fin, fout, omp, omm, gx, gy, gz) : collide<C, false>(fin, fout, omp, omm, gx, gy, gz);
}

// --------------------------------------------------------- free surface

// Ideal-gas bubble pressure (Eq. 13), p0 = rho0 c_s^2 = 1/3 (Eq. 14).
__device__ inline double bubble_pressure(long long vfx, long long vxfx, long long vsfx, int constp) {
    const double p0 = 1.0 / 3.0;
    if (constp) return p0;
    double V = (double)(vfx + vxfx) * 2.3283064365386962890625e-10;
    if (V <= 1e-3) return p0;
    double Vs = (double)vsfx * 2.3283064365386962890625e-10;
    return (Vs / V) * p0;
}

// The same pressure in FP32 from the fixed-point volumes, for the FP32-collide
// forms: v 2^-32 = hi + lo 2^-32 with 32-bit halves (no FP64 arithmetic).
__device__ inline float fx_to_float(long long v) {
    return (float)(int)(v >> 32) + (float)(unsigned)(v & 0xffffffffLL) * 2.3283064365386962890625e-10f;
}
__device__ inline float bubble_pressure_f(long long vfx, long long vxfx, long long vsfx, int constp) {
    const float p0 = (float)(1.0 / 3.0);
    if (constp) return p0;
    const float V = fx_to_float(vfx + vxfx);
    if (V <= 1e-3f) return p0;
    return (fx_to_float(vsfx) / V) * p0;
}

__device__ inline long long volume_term(uint8_t t, double phi) {
    if (t == GAS) return FSL_VOL_ONE;
    if (t == IFC) {
        double c = phi < 0.0 ? 0.0 : (phi > 1.0 ? 1.0 : phi);
        return __double2ll_rn((1.0 - c) * 4294967296.0);
    }
    return 0;
}

// The same term from an FP32 fill level, for the FP32-collide forms (every
// place that forms a volume term of those forms uses this one, so the
// per-step differences stay exact): (1 - c) 2^32 with c = clamp(phi, 0, 1)
// taken apart into its 24-bit significand and exponent, integer arithmetic
// only (the FP64 pipe of this GPU is slow), rounded half up.
__device__ inline long long volume_term_f(uint8_t t, float phi) {
    if (t == GAS) return FSL_VOL_ONE;
    if (t != IFC) return 0;
    const float c = fminf(fmaxf(phi, 0.f), 1.f);
    const unsigned u = __float_as_uint(c);
    const int E = (int)(u >> 23);
    const unsigned long long M = (u & 0x7fffffu) | (E ? 0x800000u : 0u);
    const int sh = (E ? E : 1) - 150 + 32;   // c 2^32 = M 2^sh
    unsigned long long v;
    if (sh >= 0) v = M << sh;
    else if (sh > -40) v = (M + (1ull << (-sh - 1))) >> (-sh);
    else v = 0;
    return FSL_VOL_ONE - (long long)v;
}

__device__ inline uint8_t new_type(uint8_t t, uint8_t mk) {
    if (t == IFC) {
        if (mk == MK_FILLED || mk == MK_CFILLED) return LIQ;
        if (mk == MK_EMPTIED || mk == MK_CEMPTIED) return GAS;
        return IFC;
    }
    if (t == GAS && mk == MK_NEWG) return IFC;
    if (t == LIQ && mk == MK_NEWL) return IFC;
    return t;
}

// ================================================================ kernels

// Wrapped +-1 neighbour offsets of one cell, for the streaming pull.
struct Pull {
    long long g;
    int ox[3], oy[3], oz[3];   // offset for a step of -1, 0, +1 along each axis
    __device__ inline long long at(int dx, int dy, int dz) const { return g + ox[dx + 1] + oy[dy + 1] + oz[dz + 1]; }
};

__device__ inline Pull make_pull(const Dom& D, long long g) {
    Pull p;
    p.g = g;
    int x, y, z;
    local_xyz(D, (int)(g - D.off), x, y, z);
    const int sy = D.nx, sz = D.nx * D.ny;
    p.ox[0] = x == 0 ? D.nx - 1 : -1;
    p.ox[1] = 0;
    p.ox[2] = x == D.nx - 1 ? -(D.nx - 1) : 1;
    p.oy[0] = y == 0 ? (D.ny - 1) * sy : -sy;
    p.oy[1] = 0;
    p.oy[2] = y == D.ny - 1 ? -(D.ny - 1) * sy : sy;
    p.oz[0] = z == 0 ? (D.nz - 1) * sz : -sz;
    p.oz[1] = 0;
    p.oz[2] = z == D.nz - 1 ? -(D.nz - 1) * sz : sz;
    return p;
}

// Liquid cells: stream with half-way bounce-back (Eq. 7) and collide (Eq. 6) for
// liquid cells.  Only cells flagged as touching a wall read the types of
// their neighbours; a liquid cell never touches gas (closed interface layer).
template <typename T, bool ONE>
__device__ __forceinline__ void liquid_one(const StepArgs& A, long long g, uint8_t f) {
    using C = typename Form<T>::C;
    const Dom& D = dom_at<ONE>(A, g);
    const Par<C> R = par_of<C>(D);
    const Pull P = make_pull(D, g);
    const unsigned gi = (unsigned)g;
    const long long S = A.stride;
    const T* __restrict__ src = (const T*)A.fsrc;
    T* __restrict__ dst = (T*)A.fdst;
    if constexpr (Form<T>::shifted) {
        // deviations from w_a all the way through
        float d[19];
        d[0] = Form<T>::ld_dev(src + gi);
        if (!(f & K_WALL)) {
#pragma unroll
            for (int a = 1; a < 19; ++a)
                d[a] = Form<T>::ld_dev(src + a * S + (unsigned)(gi + P.ox[1 - cx(a)] + P.oy[1 - cy(a)] + P.oz[1 - cz(a)]));
        } else {
            // all neighbour types first, then every load with its address
            // chosen without a branch (two memory latencies, not eighteen)
#pragma unroll
            for (int a = 1; a < 19; ++a) {
                const unsigned y = (unsigned)(gi + P.ox[1 - cx(a)] + P.oy[1 - cy(a)] + P.oz[1 - cz(a)]);
                const uint8_t t = ctype(A.flag[y]);
                // bounce-back reads the cell's own opposite PDF (w_a = w_abar)
                const float v = Form<T>::ld_dev(src + ((t == OBS || t == LID) ? opp(a) * S + gi : a * S + y));
                d[a] = t == LID ? v + (6.f * weightc<float>(a)) * cdot<float>(a, R.lid[0], R.lid[1], R.lid[2]) : v;
            }
        }
        float dout[19];
        if (D.has_force)
            collide_dev<true>(d, dout, R.omp, R.omm, R.g[0], R.g[1], R.g[2]);
        else
            collide_dev<false>(d, dout, R.omp, R.omm, 0.f, 0.f, 0.f);
        if (!(dout[0] == dout[0])) set_status(A.status, ST_NAN);
#pragma unroll
        for (int a = 0; a < 19; ++a) Form<T>::st_dev(dst + a * S + gi, dout[a]);
    } else {
        C fin[19];
        fin[0] = Form<T>::ld(src + gi, 0);
        if (!(f & K_WALL)) {
#pragma unroll
            for (int a = 1; a < 19; ++a)
                fin[a] = Form<T>::ld(src + a * S + (unsigned)(gi + P.ox[1 - cx(a)] + P.oy[1 - cy(a)] + P.oz[1 - cz(a)]), a);
        } else {
            unsigned bm = 0, lm = 0;   // links from an obstacle / the lid
#pragma unroll
            for (int a = 1; a < 19; ++a) {
                const uint8_t t = ctype(A.flag[(unsigned)(gi + P.ox[1 - cx(a)] + P.oy[1 - cy(a)] + P.oz[1 - cz(a)])]);
                bm |= (unsigned)(t == OBS || t == LID) << a;
                lm |= (unsigned)(t == LID) << a;
            }
#pragma unroll
            for (int a = 1; a < 19; ++a) {
                const unsigned y = (unsigned)(gi + P.ox[1 - cx(a)] + P.oy[1 - cy(a)] + P.oz[1 - cz(a)]);
                // w_a = w_abar, so the stored form of direction abar reads the same
                fin[a] = Form<T>::ld(src + (((bm >> a) & 1u) ? opp(a) * S + gi : a * S + y), a);
            }
            if (lm) {
#pragma unroll
                for (int a = 1; a < 19; ++a)
                    if ((lm >> a) & 1u) fin[a] = fin[a] + ((C)6 * weightc<C>(a)) * cdot<C>(a, R.lid[0], R.lid[1], R.lid[2]);
            }
        }
        C fout[19];
        C rho = collide_any<C>(D.has_force, fin, fout, R.omp, R.omm, R.g[0], R.g[1], R.g[2]);
        if (!(rho == rho)) set_status(A.status, ST_NAN);
#pragma unroll
        for (int a = 0; a < 19; ++a) Form<T>::st(dst + a * S + gi, a, fout[a]);
    }
}

// One liquid cell per thread (FP32 and FP64 storage); block `bid` of the
// liquid part of the stream-collide kernel.
template <typename T, bool ONE>
__device__ __forceinline__ void liquid_single(const StepArgs& A, long long bid) {
    const long long g = bid * FSL_BLOCK + threadIdx.x;
    const uint8_t f = A.flag[g];
    if (ctype(f) != LIQ) return;
    liquid_one<T, ONE>(A, g, f);
}

// Two cells per thread, cells 2t and 2t+1 (16-bit shifted storage), collided
// together in packed FP32.  A pair with a cell next to a wall reads that
// cell's neighbour types first and picks each link's address without a
// branch; a pair with one liquid cell computes both lanes and stores only the
// liquid one (the other lane's loads stay inside the lattice and its result
// is dropped).  Both liquid: one 32-bit store per direction.  (Cells 2t and
// 2t+1 always lie in the same domain: domains start on multiples of 256.)
template <typename T, bool ONE>
__device__ __forceinline__ void liquid_pairs(const StepArgs& A, long long bid) {
    const long long g0 = 2 * (bid * FSL_BLOCK + threadIdx.x);
    if (g0 >= A.stride) return;
    const unsigned short ff = *(const unsigned short*)(A.flag + g0);
    const uint8_t f0 = (uint8_t)(ff & 0xff), f1 = (uint8_t)(ff >> 8);
    const bool v0 = ctype(f0) == LIQ, v1 = ctype(f1) == LIQ;
    if (!v0 && !v1) return;
    const Dom& D = dom_at<ONE>(A, g0);
    const Par<float> R = par_of<float>(D);
    const unsigned S = (unsigned)A.stride, gi = (unsigned)g0;
    const T* __restrict__ src = (const T*)A.fsrc;
    T* __restrict__ dst = (T*)A.fdst;
    float2 d[19];
    if (!((f0 | f1) & K_WALL) && !(D.nx & 1)) {
        // even nx: x0 is even and both cells lie in one row, so the y / z
        // offsets of a link are common to the pair and only its x offsets
        // differ: cell 0 pulls x - 1 from the row's end when x0 = 0, cell 1
        // pulls x + 1 from the row's start when x0 + 1 = nx - 1.  Links along
        // x = const read both sources with one aligned 32-bit load.
        int x, y, z;
        local_xyz(D, (int)(g0 - D.off), x, y, z);
        const int sy = D.nx, sz = D.nx * D.ny;
        const int oy[3] = {y == 0 ? (D.ny - 1) * sy : -sy, 0, y == D.ny - 1 ? -(D.ny - 1) * sy : sy};
        const int oz[3] = {z == 0 ? (D.nz - 1) * sz : -sz, 0, z == D.nz - 1 ? -(D.nz - 1) * sz : sz};
        const int xm0 = x == 0 ? D.nx - 1 : -1;                 // cell 0, source x - 1
        const int xp1 = x + 2 == D.nx ? 2 - D.nx : 2;           // cell 1, source x + 1 (from cell 0)
#pragma unroll
        for (int a = 0; a < 19; ++a) {
            const unsigned r = gi + (unsigned)(oy[1 - cy(a)] + oz[1 - cz(a)]);
            if (cx(a) == 0) {
                d[a] = Form<T>::ld_dev2(src + (a * S + r));
            } else if (cx(a) > 0) {   // sources x - 1: cell 0's per x0, cell 1's is cell 0's column
                d[a] = make_float2(Form<T>::ld_dev(src + (a * S + r + (unsigned)xm0)), Form<T>::ld_dev(src + (a * S + r)));
            } else {                  // sources x + 1: cell 0's is cell 1's column
                d[a] = make_float2(Form<T>::ld_dev(src + (a * S + r + 1u)), Form<T>::ld_dev(src + (a * S + r + (unsigned)xp1)));
            }
        }
    } else {
        const Pull P0 = make_pull(D, g0), P1 = make_pull(D, g0 + 1);
        // walls, or odd nx (the pair may straddle two rows): every link of
        // each cell on its own, a wall cell's bounced links chosen without a
        // branch
        const bool k0 = v0 && (f0 & K_WALL), k1 = v1 && (f1 & K_WALL);
        d[0] = make_float2(Form<T>::ld_dev(src + gi), Form<T>::ld_dev(src + gi + 1u));
#pragma unroll
        for (int a = 1; a < 19; ++a) {
            const unsigned y0 = gi + (unsigned)(P0.ox[1 - cx(a)] + P0.oy[1 - cy(a)] + P0.oz[1 - cz(a)]);
            const unsigned y1 = gi + 1u + (unsigned)(P1.ox[1 - cx(a)] + P1.oy[1 - cy(a)] + P1.oz[1 - cz(a)]);
            const uint8_t t0 = k0 ? ctype(A.flag[y0]) : (uint8_t)LIQ;
            const uint8_t t1 = k1 ? ctype(A.flag[y1]) : (uint8_t)LIQ;
            // bounce-back reads the cell's own opposite PDF (w_a = w_abar)
            float x0 = Form<T>::ld_dev(src + ((t0 == OBS || t0 == LID) ? opp(a) * S + gi : a * S + y0));
            float x1 = Form<T>::ld_dev(src + ((t1 == OBS || t1 == LID) ? opp(a) * S + gi + 1u : a * S + y1));
            const float lidt = (6.f * weightc<float>(a)) * cdot<float>(a, R.lid[0], R.lid[1], R.lid[2]);
            if (t0 == LID) x0 += lidt;
            if (t1 == LID) x1 += lidt;
            d[a] = make_float2(x0, x1);
        }
    }
    // each output is stored as soon as it is formed: one 32-bit store per
    // direction when both cells are liquid, else the liquid lane's 16 bits of
    // the same rounded pair (a rounded pair's halves are the values rounded
    // one by one), as predicated stores rather than divergent paths
    const bool both = v0 && v1;
    auto out = [&](int a, float2 v) {
        if (a == 0 && ((v0 && !(v.x == v.x)) || (v1 && !(v.y == v.y)))) set_status(A.status, ST_NAN);
        Form<T>::st_dev2m(dst + (a * S + gi), v, both, v0 && !v1, v1 && !v0);
    };
    if (D.has_force)
        collide_dev2<true>(d, out, R.omp, R.omm, R.g[0], R.g[1], R.g[2]);
    else
        collide_dev2<false>(d, out, R.omp, R.omm, 0.f, 0.f, 0.f);
}

// Coordinates of one interface cell, for the 5x5x5 fill-level stencil of the
// curvature and its +-1 neighbours; offsets up to 2 wrap around the domain.
__device__ inline int wrap2(int v, int n) {   // v in [-2, n+1]
    v = v < 0 ? v + n : v;
    v = v < 0 ? v + n : v;
    v = v >= n ? v - n : v;
    v = v >= n ? v - n : v;
    return v;
}

// (32-bit cell numbers: the library keeps every cell number, and 19 times the
// lattice size, below 2^32)
struct Stencil {
    int x, y, z, nx, ny, nz, sz;
    unsigned off, g;
    bool inner;   // two cells from every face: no wrap needed
    __device__ inline unsigned at(int dx, int dy, int dz) const {
        if (inner) return g + (unsigned)(dx + nx * dy + sz * dz);
        return off + (unsigned)(wrap2(x + dx, nx) + nx * wrap2(y + dy, ny) + sz * wrap2(z + dz, nz));
    }
};

__device__ inline Stencil make_stencil(const Dom& D, long long g) {
    Stencil s;
    local_xyz(D, (int)(g - D.off), s.x, s.y, s.z);
    s.nx = D.nx; s.ny = D.ny; s.nz = D.nz;
    s.sz = D.nx * D.ny;
    s.off = (unsigned)D.off;
    s.g = (unsigned)g;
    s.inner = s.x >= 2 && s.x < D.nx - 2 && s.y >= 2 && s.y < D.ny - 2 && s.z >= 2 && s.z < D.nz - 2;
    return s;
}


// Equilibrium (Eq. 3) of the pair that holds direction a (1-18): the
// symmetric part fp and antisymmetric part fm of the pair's first (odd)
// direction, as feq_all forms them; f_eq,a = fp + fm for odd a, fp - fm for
// even a.
template <typename C>
__device__ inline void feq_pair(int a, C rho, C ux, C uy, C uz, C usq, C& fp, C& fm) {
    const int p = (a & 1) ? a : a - 1;
    const C cu = ((C)rcx(p) * ux + (C)rcy(p) * uy) + (C)rcz(p) * uz;
    const C wr = weightc<C>(p) * rho;
    fp = wr * (((C)1 + (C)4.5 * (cu * cu)) - (C)1.5 * usq);
    fm = wr * ((C)3 * cu);
}

// The collision of `collide` (Eq. 6, TRT with Guo forcing) split so that
// several threads can share the outputs of one cell: CollidePrep forms the
// cell's moments and velocity once, collide_out gives output a, each with
// every operation in the same order as `collide`.
template <typename C>
struct CollidePrep {
    C rho, ux, uy, uz, usq, Fx, Fy, Fz, uF;
};
template <typename C, bool FORCE>
__device__ inline CollidePrep<C> collide_prep(const C* fin, C gx, C gy, C gz) {
    CollidePrep<C> P;
    C jx, jy, jz;
    moments<C>(fin, P.rho, jx, jy, jz);
    P.Fx = (C)0; P.Fy = (C)0; P.Fz = (C)0;
    if constexpr (FORCE) {
        P.Fx = P.rho * gx; P.Fy = P.rho * gy; P.Fz = P.rho * gz;
        jx = jx + (C)0.5 * P.Fx;
        jy = jy + (C)0.5 * P.Fy;
        jz = jz + (C)0.5 * P.Fz;
    }
    if constexpr (sizeof(C) == 4) {
        const C ir = (C)1 / P.rho;
        P.ux = jx * ir; P.uy = jy * ir; P.uz = jz * ir;
    } else {
        P.ux = jx / P.rho; P.uy = jy / P.rho; P.uz = jz / P.rho;
    }
    P.usq = P.ux * P.ux + P.uy * P.uy + P.uz * P.uz;
    P.uF = (C)0;
    if constexpr (FORCE) P.uF = P.ux * P.Fx + P.uy * P.Fy + P.uz * P.Fz;
    return P;
}
template <typename C, bool FORCE>
__device__ inline C collide_out(int a, const C* fin, const CollidePrep<C>& P, C omp, C omm) {
    const C cp = (C)1 - (C)0.5 * omp, cm = (C)1 - (C)0.5 * omm;
    if (a == 0) {
        const C feq0 = (weightc<C>(0) * P.rho) * ((C)1 - (C)1.5 * P.usq);
        C out = fin[0] - omp * (fin[0] - feq0);
        if constexpr (FORCE) {
            const C S0 = weightc<C>(0) * ((C)-3 * P.uF);
            out = out + cp * S0;
        }
        return out;
    }
    const int p = (a & 1) ? a : a - 1;
    const C w = weightc<C>(p);
    const C cu = ((C)rcx(p) * P.ux + (C)rcy(p) * P.uy) + (C)rcz(p) * P.uz;
    const C wr = w * P.rho;
    const C feqp = wr * (((C)1 + (C)4.5 * (cu * cu)) - (C)1.5 * P.usq);
    const C feqm = wr * ((C)3 * cu);
    const C fp = (C)0.5 * (fin[p] + fin[p + 1]);
    const C fm = (C)0.5 * (fin[p] - fin[p + 1]);
    const C A = omp * (fp - feqp);
    const C B = omm * (fm - feqm);
    C out = (a == p) ? (fin[p] - A) - B : (fin[p + 1] - A) + B;
    if constexpr (FORCE) {
        const C cF = ((C)rcx(p) * P.Fx + (C)rcy(p) * P.Fy) + (C)rcz(p) * P.Fz;
        const C Sp = w * (((C)9 * cu) * cF - (C)3 * P.uF);
        const C Sm = w * ((C)3 * cF);
        const C sp = cp * Sp, sm = cm * Sm;
        out = (a == p) ? (out + sp) + sm : (out + sp) - sm;
    }
    return out;
}

// Interface cells: from the list of interface cells built at the end of
// the previous step.  A block of 128 threads takes 16 cells per pass, eight
// threads per cell.  Load phase: the 81 fill levels of the curvature stencil
// (rows along x), and for the directions q, q+8, q+16 the cell's PDFs, the PDF
// streaming in, the neighbour types and the mass-exchange terms.  Gradient
// phase: Parker-Youngs gradients at the cell and at its six face neighbours
// (unit normals there).  Compute phase, the cell's threads sharing its
// directions, each output formed with the oracle's operations in the oracle's
// order: stream with bounce-back (Eq. 7), mass exchange over the 18 links
// (Eq. 10), reconstruction of the PDFs coming from the gas side with the gas
// density 3 (p_V + 2 sigma kappa) of the cell's bubble (Eqs. 8, 11-15, kappa =
// 1/2 div n_hat by central differences of the face normals), collision
// (Eq. 6), then the filled / emptied marks.  The FP32-collide forms do all of
// this in FP32 except the cell mass, which accumulates in FP64.
#ifndef FSL_IF_GRID
#define FSL_IF_GRID 2     // interface blocks per SM in the grid (ifb is two per SM)
#endif
#ifndef FSL_STREAM_MINB
#define FSL_STREAM_MINB 3 // resident stream-collide blocks per SM the FP32-collide forms are compiled for
#endif
#ifndef FSL_IF_CELLS
#define FSL_IF_CELLS 32   // interface cells per pass of the FP32-collide forms (256 / threads per cell)
#endif
template <typename T> struct IfCells {   // cells per pass of a 256-thread block
    static constexpr int n = sizeof(typename Form<T>::C) == 8 ? 16 : FSL_IF_CELLS;
};
template <typename T>
struct IfStage {
    using C = typename Form<T>::C;
    static constexpr int N = IfCells<T>::n;
    C ph[N][125];      // fill levels, 5x5x5 box around the cell
    C fs[N][19];       // own post-collision PDFs of the previous step
    C fy[N][19];       // PDF streaming in from the source cell
    C fin[N][19];      // PDFs after streaming and reconstruction
    C ex[N][19];       // mass-exchange term of each link (Eq. 10); until the gradient
                       // phase, the fill level of the link's neighbour x + c_a
    C nrm[N][7][3];    // gradient at the cell, unit normals at the face neighbours
    C pv[N];           // bubble pressure (Eq. 13)
    C px[N];           // fill level of the cell
    double m[N];       // mass
    int g[N];          // cell
    uint8_t tz[N][19]; // type of the neighbour x + c_a (the source of direction opp(a))
};

__device__ inline int ph_index(int dx, int dy, int dz) { return (dx + 2) + 5 * (dy + 2) + 25 * (dz + 2); }
// (dy, dz) of stencil row r (0-20): rows 0-8 are |dy|,|dz| <= 1 (five points
// along x), rows 9-20 have |dy| = 2 or |dz| = 2 (three points along x)
__device__ inline void ph_row(int r, int& dy, int& dz) {
    if (r < 9) {
        dy = r % 3 - 1;
        dz = r / 3 - 1;
    } else {
        const int e = r - 9, side = e / 3, t = e % 3 - 1;
        const int s2 = (side & 1) ? -2 : 2;
        if (side < 2) { dy = s2; dz = t; }
        else { dy = t; dz = s2; }
    }
}

// Per-step counters, reset by one block of the stream-collide kernel (the
// previous step's kernels are done with them; nothing in the stream-collide
// kernel reads them).
__device__ inline void step_counters(const StepArgs& A) {
    for (int d = threadIdx.x; d < A.ndom; d += blockDim.x) {
        if (A.nif[d] > 0) A.pool[d] = 0;   // the pool was shared out last step
        A.nif[d] = A.icnt[d];
        A.trig[1 + d] = 0;
    }
    if (threadIdx.x == 0) {
        *A.stepno += 1;
        *A.gcount = 0;
        *A.lcount = 0;
        *A.trig = 0;
    }
}

// One pass over the interface cells i0 .. i0 + N - 1 of the list (those below
// cnt), by the whole block; ends with a block barrier.
template <typename T, bool ONE>
__device__ __forceinline__ void interface_chunk(const StepArgs& A, int i0, int cnt, IfStage<T>& sh) {
    using C = typename Form<T>::C;
    constexpr int N = IfCells<T>::n;
    constexpr int TPC = FSL_BLOCK / N;   // threads per cell
    const unsigned S = (unsigned)A.stride;
    const T* __restrict__ src = (const T*)A.fsrc;
    T* __restrict__ dst = (T*)A.fdst;
    // fill levels in the arithmetic type (FP32 copies for the FP32-collide forms)
    const C* __restrict__ phic;
    const C* __restrict__ phtc;
    if constexpr (sizeof(C) == 8) { phic = A.phi; phtc = A.phit; }
    else { phic = A.phif; phtc = A.phitf; }
    const int c = threadIdx.x / TPC;      // cell of this thread in the load and gradient phases
    const int q = threadIdx.x % TPC;
    {
        // ---------------- load phase: every global load of the thread is
        // issued before the first shared-memory store, so that the phase costs
        // about two memory latencies (the list entry, then everything else)
        if (i0 + c < cnt) {
            const long long g = A.ilist[i0 + c];
            const Dom& D = dom_at<ONE>(A, g);
            const Stencil st = make_stencil(D, g);
            // the 81 stencil points as 21 rows along x: 9 rows |dy|,|dz| <= 1 of
            // five points (x = -2..2), then 12 rows with |dy| = 2 or |dz| = 2 of
            // three points (x = -1..1); no other point is read
            constexpr int NR = (21 + TPC - 1) / TPC;   // rows of this thread
            constexpr int ND = (19 + TPC - 1) / TPC;   // directions of this thread
            C rowv[NR][5];
            const bool xin = st.x >= 2 && st.x < st.nx - 2;
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const int r = q + TPC * k;
                if (r < 21) {
                    int dy, dz;
                    ph_row(r, dy, dz);
                    const int w = r < 9 ? 2 : 1;   // half width of the row
                    if (xin) {
                        const unsigned b = st.at(0, dy, dz);
#pragma unroll
                        for (int e = 0; e < 5; ++e)
                            if (e - 2 >= -w && e - 2 <= w) rowv[k][e] = phtc[b + (e - 2)];
                    } else {
#pragma unroll
                        for (int e = 0; e < 5; ++e)
                            if (e - 2 >= -w && e - 2 <= w) rowv[k][e] = phtc[st.at(e - 2, dy, dz)];
                    }
                }
            }
            // per direction a: the own PDF, the PDF streaming in from x - c_a,
            // and type and fill level of x + c_a.  The source x - c_a of
            // direction a is the neighbour x + c_b of b = opp(a), so the
            // source's type and the PDF f_b(x + c_a) of the mass exchange are
            // loads the thread of the opposite direction makes (each neighbour
            // is read once)
            C fsv[ND], fyv[ND], phz[ND];
            uint8_t tzv[ND];
#pragma unroll
            for (int k = 0; k < ND; ++k) {
                const int a = q + TPC * k;
                if (a < 19) {
                    fsv[k] = Form<T>::ld(src + ((unsigned)a * S + (unsigned)g), a);
                    if (a > 0) {
                        const int ax = rcx(a), ay = rcy(a), az = rcz(a);
                        const unsigned y = st.at(-ax, -ay, -az);
                        const unsigned z = st.at(ax, ay, az);
                        fyv[k] = Form<T>::ld(src + ((unsigned)a * S + y), a);
                        tzv[k] = ctype(A.flag[z]);
                        phz[k] = phic[z];
                    }
                }
            }
            if (q == TPC - 1) {
                sh.px[c] = phic[g];
                sh.m[c] = A.m[g];
                sh.g[c] = (int)g;
                const int bub = A.id[g];
                if constexpr (sizeof(C) == 8)
                    sh.pv[c] = bub >= 0 ? bubble_pressure(A.vfx[bub], A.vxfx[bub], A.vsfx[bub], A.constp[bub]) : 1.0 / 3.0;
                else
                    sh.pv[c] = bub >= 0 ? bubble_pressure_f(A.vfx[bub], A.vxfx[bub], A.vsfx[bub], A.constp[bub])
                                        : (float)(1.0 / 3.0);
            }
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const int r = q + TPC * k;
                if (r < 21) {
                    int dy, dz;
                    ph_row(r, dy, dz);
                    const int w = r < 9 ? 2 : 1;
                    C* row = &sh.ph[c][ph_index(0, dy, dz)];
#pragma unroll
                    for (int e = 0; e < 5; ++e)
                        if (e - 2 >= -w && e - 2 <= w) row[e - 2] = rowv[k][e];
                }
            }
#pragma unroll
            for (int k = 0; k < ND; ++k) {
                const int a = q + TPC * k;
                if (a < 19) {
                    sh.fs[c][a] = fsv[k];
                    if (a > 0) {
                        sh.fy[c][a] = fyv[k];
                        sh.tz[c][a] = tzv[k];
                        sh.ex[c][a] = phz[k];
                    }
                }
            }
        }
        __syncthreads();
        // ---------------- gradient phase: first the exchange term of each of
        // the thread's directions a (Eq. 10) from f_b(x + c_a) - f_a(x), b =
        // opp(a), weighted by the mean fill level when x + c_a is an interface
        // cell; then point j (the cell, then its +x, -x, +y, -y, +z, -z
        // neighbours) for j = q, q + TPC, ...
        if (i0 + c < cnt) {
            for (int a = q > 0 ? q : TPC; a < 19; a += TPC) {
                const uint8_t tz = sh.tz[c][a];
                if (tz == LIQ || tz == IFC) {
                    const C e = sh.fy[c][opp(a)] - sh.fs[c][a];
                    sh.ex[c][a] = tz == IFC ? ((C)0.5 * (sh.px[c] + sh.ex[c][a])) * e : e;
                }
            }
            for (int j = q; j < 7; j += TPC) {
                const int ox = j == 1 ? 1 : (j == 2 ? -1 : 0);
                const int oy = j == 3 ? 1 : (j == 4 ? -1 : 0);
                const int oz = j == 5 ? 1 : (j == 6 ? -1 : 0);
                const C* P = &sh.ph[c][ph_index(ox, oy, oz)];   // P[dx + 5 dy + 25 dz]
                C gx = (C)0, gy = (C)0, gz = (C)0;
#pragma unroll
                for (int b = -1; b <= 1; ++b) {
#pragma unroll
                    for (int a = -1; a <= 1; ++a) {
                        const C W = (a == 0 && b == 0) ? (C)4 : ((a == 0 || b == 0) ? (C)2 : (C)1);
                        gx = gx + W * (P[1 + 5 * a + 25 * b] - P[-1 + 5 * a + 25 * b]);
                        gy = gy + W * (P[a + 5 + 25 * b] - P[a - 5 + 25 * b]);
                        gz = gz + W * (P[a + 5 * b + 25] - P[a + 5 * b - 25]);
                    }
                }
                if (j > 0) {
                    const C qq = gx * gx + gy * gy + gz * gz;
                    if (qq > (C)0) {
                        const C len = sqrt(qq);
                        gx = -(gx / len); gy = -(gy / len); gz = -(gz / len);
                    } else {
                        gx = (C)0; gy = (C)0; gz = (C)0;
                    }
                }
                sh.nrm[c][j][0] = gx;
                sh.nrm[c][j][1] = gy;
                sh.nrm[c][j][2] = gz;
            }
        }
        __syncthreads();
        // ---------------- compute phase, the cell's TPC threads share its
        // directions (a = q, q + TPC, ...); the cell's moments are formed by
        // each of them in the same order
        {
            const bool act = i0 + c < cnt;
            long long g = 0;
            uint8_t mk = MK_NONE;
            if (act) {
                g = sh.g[c];
                const Dom& D = dom_at<ONE>(A, g);
                const Par<C> R = par_of<C>(D);
                C rs, jsx, jsy, jsz;
                moments<C>(sh.fs[c], rs, jsx, jsy, jsz);
                const C ugx = jsx / rs, ugy = jsy / rs, ugz = jsz / rs;
                const C usg = ugx * ugx + ugy * ugy + ugz * ugz;
                const C dX = sh.nrm[c][1][0] - sh.nrm[c][2][0];
                const C dY = sh.nrm[c][3][1] - sh.nrm[c][4][1];
                const C dZ = sh.nrm[c][5][2] - sh.nrm[c][6][2];
                const C kappa = (C)0.25 * ((dX + dY) + dZ);
                const C gx = sh.nrm[c][0][0], gy = sh.nrm[c][0][1], gz = sh.nrm[c][0][2];
                const C rg = (C)3 * (sh.pv[c] + R.sigma2 * kappa);
                for (int a = q; a < 19; a += TPC) {
                    C fin;
                    if (a == 0) {
                        fin = sh.fs[c][0];
                    } else {
                        const int ab = opp(a);
                        const C fsb = sh.fs[c][ab];
                        const uint8_t ty = sh.tz[c][ab];   // type of x - c_a = x + c_ab
                        if (ty == OBS) {
                            fin = fsb;
                        } else if (ty == LID) {
                            const C cuw = ((C)rcx(a) * R.lid[0] + (C)rcy(a) * R.lid[1]) + (C)rcz(a) * R.lid[2];
                            fin = fsb + ((C)6 * weightc<C>(a)) * cuw;
                        } else {
                            C fp, fm;
                            feq_pair<C>(a, rg, ugx, ugy, ugz, usg, fp, fm);
                            const C fga = (a & 1) ? fp + fm : fp - fm;
                            const C fgb = (a & 1) ? fp - fm : fp + fm;
                            if (ty == GAS) {
                                fin = (fga + fgb) - fsb;
                            } else {
                                fin = sh.fy[c][a];
                                if (D.normal_rule && ((C)rcx(a) * gx + (C)rcy(a) * gy) + (C)rcz(a) * gz > (C)0)
                                    fin = (fga + fgb) - fsb;
                            }
                        }
                    }
                    sh.fin[c][a] = fin;
                }
            }
            __syncwarp();
            if (act) {
                const Dom& D = dom_at<ONE>(A, g);
                const Par<C> R = par_of<C>(D);
                C rho;
                if (D.has_force) {
                    const CollidePrep<C> P = collide_prep<C, true>(sh.fin[c], R.g[0], R.g[1], R.g[2]);
                    rho = P.rho;
                    for (int a = q; a < 19; a += TPC)
                        Form<T>::st(dst + ((unsigned)a * S + (unsigned)g), a, collide_out<C, true>(a, sh.fin[c], P, R.omp, R.omm));
                } else {
                    const CollidePrep<C> P = collide_prep<C, false>(sh.fin[c], (C)0, (C)0, (C)0);
                    rho = P.rho;
                    for (int a = q; a < 19; a += TPC)
                        Form<T>::st(dst + ((unsigned)a * S + (unsigned)g), a, collide_out<C, false>(a, sh.fin[c], P, R.omp, R.omm));
                }
                if (q == 0) {
                    if (!(rho == rho)) set_status(A.status, ST_NAN);
                    // mass exchange, summed in direction order (Eq. 10); the
                    // cell mass itself accumulates in FP64 for every form
                    C dm = (C)0;
                    bool has_gas = false, has_liq = false;
#pragma unroll
                    for (int a = 1; a < 19; ++a) {
                        const uint8_t tz = sh.tz[c][a];
                        if (tz == LIQ || tz == IFC) dm = dm + sh.ex[c][a];
                        has_gas |= tz == GAS;
                        has_liq |= tz == LIQ;
                    }
                    const double mnew = sh.m[c] + (double)dm;
                    A.m[g] = mnew;
                    A.rhoi[g] = (double)rho;
                    bool filled, emptied;
                    if constexpr (sizeof(C) == 8) {
                        filled = mnew > (1.0 + D.eps) * rho;
                        emptied = mnew < (-D.eps) * rho;
                    } else {
                        const float mf = (float)mnew;
                        filled = mf > (1.f + D.feps) * rho;
                        emptied = mf < (-D.feps) * rho;
                    }
                    if (filled) mk = MK_FILLED;
                    else if (emptied) mk = MK_EMPTIED;
                    else if (D.lonely_rule) {
                        // a cell that no longer separates liquid from gas
                        if (!has_gas) mk = MK_FILLED;
                        else if (!has_liq) mk = MK_EMPTIED;
                    }
                    A.mark[g] = mk;
                }
            }
            list_append(A.mlist, A.mcount, mk != MK_NONE, (int)g);
        }
        __syncthreads();
    }
}

// Block `bid` of the `nbl` blocks of the interface part of the split
// stream-collide kernel: list chunks bid, bid + nbl, bid + 2 nbl, ...
template <typename T, bool ONE>
__device__ __forceinline__ void interface_cells(const StepArgs& A, int bid, int nbl, IfStage<T>& sh) {
    constexpr int N = IfCells<T>::n;
    if (bid == 0) step_counters(A);
    const int cnt = *A.icount;
    for (int i0 = bid * N; i0 < cnt; i0 += nbl * N) interface_chunk<T, ONE>(A, i0, cnt, sh);
}

// ------------------------------------------- interface cells, one per thread
// Threads (cells) per block of the one-thread-per-cell interface kernel.
template <typename T> struct IfThreads {
    static constexpr int n = sizeof(typename Form<T>::C) == 8 ? 64 : 128;
};

// ------------------------------------------------------------ normals pass
// The Parker-Youngs gradient at a cell from its 27 stencil values v(dx, dy, dz),
// summed in the order of pyg (and of the oracle's two-level loop).
template <typename C, class V>
__device__ __forceinline__ void pyg_of(V&& v, C& gx, C& gy, C& gz) {
    gx = (C)0; gy = (C)0; gz = (C)0;
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
#pragma unroll
        for (int a = -1; a <= 1; ++a) {
            const C W = (a == 0 && b == 0) ? (C)4 : ((a == 0 || b == 0) ? (C)2 : (C)1);
            gx = gx + W * (v(1, a, b) - v(-1, a, b));
            gy = gy + W * (v(a, 1, b) - v(a, -1, b));
            gz = gz + W * (v(a, b, 1) - v(a, b, -1));
        }
    }
}

// Stores of the normals pass for a cell g that needs a normal: the normal-test
// bits of an interface cell, and the unit normal -grad/|grad| (0 where the
// gradient is 0), with the arithmetic of the interface kernels (in FP64; the
// FP32-collide forms scale by a reciprocal square root).
template <typename C>
__device__ __forceinline__ void normal_out(const StepArgs& A, unsigned g, bool ifc, C gx, C gy, C gz) {
    if (ifc) {
        // the bubble pressure the interface kernel would look up through the
        // cell's bubble (a load that waits on another): looked up here
        const int bub = A.id[g];
        C pv;
        if constexpr (sizeof(C) == 8)
            pv = bub >= 0 ? bubble_pressure(A.vfx[bub], A.vxfx[bub], A.vsfx[bub], A.constp[bub]) : 1.0 / 3.0;
        else
            pv = bub >= 0 ? bubble_pressure_f(A.vfx[bub], A.vxfx[bub], A.vsfx[bub], A.constp[bub])
                          : (float)(1.0 / 3.0);
        ((C*)A.pvc)[g] = pv;
        unsigned mk = 0;
#pragma unroll
        for (int a = 1; a < 19; ++a)
            mk |= (unsigned)(((C)cx(a) * gx + (C)cy(a) * gy) + (C)cz(a) * gz > (C)0) << a;
        A.nmask[g] = mk;
    }
    C nx = gx, ny = gy, nz = gz;
    const C qq = nx * nx + ny * ny + nz * nz;
    if (qq > (C)0) {
        if constexpr (sizeof(C) == 8) {
            const C len = sqrt(qq);
            nx = -(nx / len); ny = -(ny / len); nz = -(nz / len);
        } else {
            // FP32-collide forms: one reciprocal square root (within 2 ulp)
            const float il = rsqrtf(qq);
            nx = -(nx * il); ny = -(ny * il); nz = -(nz * il);
        }
    } else {
        nx = (C)0; ny = (C)0; nz = (C)0;
    }
    C* __restrict__ nr = (C*)A.nrm;
    const unsigned S = (unsigned)A.stride;
    nr[g] = nx;
    nr[S + g] = ny;
    nr[2u * S + g] = nz;
}

// Normals pass, one thread per cell of the padded lattice, ahead of the
// stream-collide kernels that take the interface cells one per thread.  The
// curvature of an interface cell x (Eq. 15) is half the divergence of the unit
// normals -grad(phi)/|grad(phi)| at its six face neighbours, and the
// reconstruction's normal test (Eq. 11) uses the gradient at x itself.  Each
// normal is computed here once, for every cell that is an interface cell or a
// face neighbour of one (walls included: the stencil reads walls as full), and
// stored in nrm; each interface cell also stores its 18 normal-test bits in
// nmask, and the pressure of its bubble (Eq. 13) in pvc.  The stencil values
// are the stored copy phit (walls and liquid 1, gas 0, interface clamp(phi, 0,
// 1)) and the arithmetic is that of the interface kernels, so their curvature
// and reconstruction come out as if they had computed the normals themselves.
//
// A warp whose 32 cells lie in one row of one domain (the usual case: rows
// start on multiples of 32 when nx is one) works on the row segment: the y / z
// offsets are common to the warp, each lane loads the 9 (dy, dz) rows at its
// own x and takes x - 1 and x + 1 from its neighbour lanes (the segment's end
// lanes load them, wrapping within the row), and the warp returns at once when
// no cell of the segment needs a normal.  Other warps take one cell per
// thread with the general stencil addressing.
template <typename T, bool ONE>
__global__ void __launch_bounds__(FSL_BLOCK) k_normals(StepArgs A) {
    using C = typename Form<T>::C;
    const long long g = (long long)blockIdx.x * FSL_BLOCK + threadIdx.x;   // stride: a multiple of the block
    const Dom& D = dom_at<ONE>(A, g);
    const C* __restrict__ ph;
    if constexpr (sizeof(C) == 8) ph = A.phit;
    else ph = A.phitf;
    const unsigned lane = threadIdx.x & 31u;
    const long long l0 = g - lane - D.off;   // the warp's first cell in its domain
    int x0, y, z;
    local_xyz(D, (int)(l0 < D.n ? l0 : 0), x0, y, z);
    if (l0 + 31 < D.n && x0 + 31 < D.nx) {
        const unsigned gi = (unsigned)g;
        const int sy = D.nx, sz = D.nx * D.ny;
        const int oy[3] = {y == 0 ? (D.ny - 1) * sy : -sy, 0, y == D.ny - 1 ? -(D.ny - 1) * sy : sy};
        const int oz[3] = {z == 0 ? (D.nz - 1) * sz : -sz, 0, z == D.nz - 1 ? -(D.nz - 1) * sz : sz};
        const int oxm = x0 == 0 ? D.nx - 1 : -1;          // lane 0: x - 1
        const int oxp = x0 + 32 == D.nx ? 1 - D.nx : 1;    // lane 31: x + 1
        const unsigned t = ctype(A.flag[gi]);
        const unsigned ty0 = ctype(A.flag[gi + oy[0]]), ty2 = ctype(A.flag[gi + oy[2]]);
        const unsigned tz0 = ctype(A.flag[gi + oz[0]]), tz2 = ctype(A.flag[gi + oz[2]]);
        const unsigned tl0 = lane == 0 ? ctype(A.flag[gi + oxm]) : 0u, tr0 = lane == 31 ? ctype(A.flag[gi + oxp]) : 0u;
        unsigned tl = __shfl_up_sync(0xffffffffu, t, 1), tr = __shfl_down_sync(0xffffffffu, t, 1);
        if (lane == 0) tl = tl0;
        if (lane == 31) tr = tr0;
        const bool need = (t == IFC) | (tl == IFC) | (tr == IFC) | (ty0 == IFC) | (ty2 == IFC) | (tz0 == IFC) |
                          (tz2 == IFC);
        if (!__any_sync(0xffffffffu, need)) return;
        C v[3][3][3];   // [dz + 1][dy + 1][dx + 1]
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const unsigned r = gi + (unsigned)(oy[dy + 1] + oz[dz + 1]);
                const C c = ph[r];
                const C e = lane == 0 ? ph[r + oxm] : (lane == 31 ? ph[r + oxp] : c);
                C l = __shfl_up_sync(0xffffffffu, c, 1), rr = __shfl_down_sync(0xffffffffu, c, 1);
                if (lane == 0) l = e;
                if (lane == 31) rr = e;
                v[dz + 1][dy + 1][0] = l;
                v[dz + 1][dy + 1][1] = c;
                v[dz + 1][dy + 1][2] = rr;
            }
        if (!need) return;
        C gx, gy, gz;
        pyg_of<C>([&](int dx, int dy, int dz) { return v[dz + 1][dy + 1][dx + 1]; }, gx, gy, gz);
        normal_out<C>(A, gi, t == IFC, gx, gy, gz);
        return;
    }
    if (g - D.off >= D.n) return;   // padding after the domain
    const Stencil st = make_stencil(D, g);
    // the seven types are loaded together (no load waits for another's result)
    const uint8_t t = ctype(A.flag[g]);
    const uint8_t t1 = ctype(A.flag[st.at(1, 0, 0)]), t2 = ctype(A.flag[st.at(-1, 0, 0)]);
    const uint8_t t3 = ctype(A.flag[st.at(0, 1, 0)]), t4 = ctype(A.flag[st.at(0, -1, 0)]);
    const uint8_t t5 = ctype(A.flag[st.at(0, 0, 1)]), t6 = ctype(A.flag[st.at(0, 0, -1)]);
    const int need = (t == IFC) | (t1 == IFC) | (t2 == IFC) | (t3 == IFC) | (t4 == IFC) | (t5 == IFC) | (t6 == IFC);
    if (!need) return;
    C gx, gy, gz;
    pyg_of<C>([&](int dx, int dy, int dz) { return ph[st.at(dx, dy, dz)]; }, gx, gy, gz);
    normal_out<C>(A, (unsigned)g, t == IFC, gx, gy, gz);
}

// The normals pass of a single-domain handle by 3D tiles: a block takes a
// tile of NT_X x NT_Y x NT_Z cells, loads the types and stencil values of the
// tile and its one-cell halo (wrapping periodically, as the stencil does)
// into shared memory with every load independent of the others, lists the
// tile's cells that need a normal and computes those one per thread from the
// shared copy.  The values and the arithmetic are those of k_normals.  Needs nx >= NT_X, ny >= NT_Y and
// nz >= NT_Z (a halo coordinate is then at most one domain length out).
constexpr int NT_X = 32, NT_Y = 8, NT_Z = 8;
constexpr int NH_X = NT_X + 2, NH_Y = NT_Y + 2, NH_Z = NT_Z + 2;
static_assert(NT_X == 32 && NT_Y == 8 && NT_Z <= 8, "the tile's cell list packs x, y, z into 5 + 3 + 3 bits");
template <typename T, bool ONE>
__global__ void __launch_bounds__(NT_X * NT_Y) k_normals_tiled(StepArgs A) {
    using C = typename Form<T>::C;
    __shared__ C vs[NH_Z][NH_Y][NH_X];
    __shared__ uint8_t ts[NH_Z][NH_Y][NH_X];
    __shared__ unsigned short clist[NT_X * NT_Y * NT_Z];
    __shared__ int nlist;
    if (threadIdx.x == 0) nlist = 0;
    // the block's tile: from its index in a single domain, from the tile
    // table in a batch
    int x0, y0, z0;
    const Dom* Dp;
    if constexpr (ONE) {
        Dp = &A.d0;
        const int ntx = (Dp->nx + NT_X - 1) / NT_X, nty = (Dp->ny + NT_Y - 1) / NT_Y;
        const int b = (int)blockIdx.x;
        x0 = (b % ntx) * NT_X; y0 = ((b / ntx) % nty) * NT_Y; z0 = (b / (ntx * nty)) * NT_Z;
    } else {
        const int4 t = A.ntiles[blockIdx.x];
        Dp = &get_dom(A, t.x);
        x0 = t.y; y0 = t.z; z0 = t.w;
    }
    const Dom& D = *Dp;
    const C* __restrict__ ph;
    if constexpr (sizeof(C) == 8) ph = A.phit;
    else ph = A.phitf;
    const unsigned off = (unsigned)D.off;
    // all loads of the thread first, then the shared stores (element i of the
    // halo tile is entry i of the flattened shared arrays)
    constexpr int NH = NH_X * NH_Y * NH_Z, NTH = NT_X * NT_Y, NIT = (NH + NTH - 1) / NTH;
    C lv[NIT];
    uint8_t lt[NIT];
#pragma unroll
    for (int k = 0; k < NIT; ++k) {
        const int i = (int)threadIdx.x + k * NTH;
        if (i < NH) {
            const int hx = i % NH_X, hy = (i / NH_X) % NH_Y, hz = i / (NH_X * NH_Y);
            int x = x0 + hx - 1, y = y0 + hy - 1, z = z0 + hz - 1;
            x = x < 0 ? x + D.nx : (x >= D.nx ? x - D.nx : x);
            y = y < 0 ? y + D.ny : (y >= D.ny ? y - D.ny : y);
            z = z < 0 ? z + D.nz : (z >= D.nz ? z - D.nz : z);
            const unsigned c = off + (unsigned)(x + D.nx * (y + D.ny * z));
            lv[k] = ph[c];
            lt[k] = ctype(A.flag[c]);
        }
    }
#pragma unroll
    for (int k = 0; k < NIT; ++k) {
        const int i = (int)threadIdx.x + k * NTH;
        if (i < NH) {
            (&vs[0][0][0])[i] = lv[k];
            (&ts[0][0][0])[i] = lt[k];
        }
    }
    __syncthreads();
    // the tile's cells that need a normal, listed (warp ballots), then taken
    // one per thread, so that no lane idles through a normal of its warp
    const int tx = threadIdx.x % NT_X, ty = threadIdx.x / NT_X;
    const unsigned lane = threadIdx.x & 31u;
    const bool col = x0 + tx < D.nx && y0 + ty < D.ny;
#pragma unroll 1
    for (int tz = 0; tz < NT_Z; ++tz) {
        const int hx = tx + 1, hy = ty + 1, hz = tz + 1;
        const bool nd = col && z0 + tz < D.nz &&
                        ((ts[hz][hy][hx] == IFC) | (ts[hz][hy][hx + 1] == IFC) | (ts[hz][hy][hx - 1] == IFC) |
                         (ts[hz][hy + 1][hx] == IFC) | (ts[hz][hy - 1][hx] == IFC) | (ts[hz + 1][hy][hx] == IFC) |
                         (ts[hz - 1][hy][hx] == IFC));
        const unsigned bal = __ballot_sync(0xffffffffu, nd);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(&nlist, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (nd) clist[base + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)(tx | (ty << 5) | (tz << 8));
    }
    __syncthreads();
    const int n = nlist;
    for (int i = threadIdx.x; i < n; i += NT_X * NT_Y) {
        const unsigned c = clist[i];
        const int cx_ = (int)(c & 31u), cy_ = (int)((c >> 5) & 7u), cz_ = (int)(c >> 8);
        const int hx = cx_ + 1, hy = cy_ + 1, hz = cz_ + 1;
        C gx, gy, gz;
        pyg_of<C>([&](int dx, int dy, int dz) { return vs[hz + dz][hy + dy][hx + dx]; }, gx, gy, gz);
        normal_out<C>(A, off + (unsigned)((x0 + cx_) + D.nx * ((y0 + cy_) + D.ny * (z0 + cz_))),
                      ts[hz][hy][hx] == IFC, gx, gy, gz);
    }
}

// One interface cell g by one thread, every direction unrolled: the same
// steps and the same arithmetic, operation by operation, as the shared
// interface pass (stream with bounce-back, Eq. 7; mass exchange over the 18
// links in direction order, Eq. 10; reconstruction from the bubble's gas
// density 3 (p_V + 2 sigma kappa), Eqs. 8, 11-15; collision, Eq. 6; filled /
// emptied marks).  The curvature and the normal test come from the normals
// pass (k_normals), run before this kernel in the same step.  Returns whether
// the cell was marked.
template <typename T, bool ONE>
__device__ __forceinline__ bool iface_one(const StepArgs& A, long long g) {
    using C = typename Form<T>::C;
    const Dom& D = dom_at<ONE>(A, g);
    const Par<C> R = par_of<C>(D);
    const Stencil st = make_stencil(D, g);
    const unsigned S = (unsigned)A.stride;
    const T* __restrict__ src = (const T*)A.fsrc;
    T* __restrict__ dst = (T*)A.fdst;
    const C* __restrict__ phic;
    if constexpr (sizeof(C) == 8) phic = A.phi;
    else phic = A.phif;
    // own PDFs, and per direction a the source x - c_a: its type, the PDF
    // streaming in and its fill level
    // (the 18 source types packed 3 bits each: ty(a) = (tym >> 3a) & 7)
    C fs[19], fy[19], phy[19];
    unsigned long long tym = 0;
    fs[0] = Form<T>::ld(src + (unsigned)g, 0);
#pragma unroll
    for (int a = 1; a < 19; ++a) {
        fs[a] = Form<T>::ld(src + ((unsigned)a * S + (unsigned)g), a);
        const unsigned y = st.at(-cx(a), -cy(a), -cz(a));
        tym |= (unsigned long long)ctype(A.flag[y]) << (3 * a);
        fy[a] = Form<T>::ld(src + ((unsigned)a * S + y), a);
        phy[a] = phic[y];
    }
    auto ty = [&](int a) { return (uint8_t)((tym >> (3 * a)) & 7u); };
    const C phx = phic[g];
    const double m0 = A.m[g];
    const C pv = ((const C*)A.pvc)[g];   // the bubble's pressure, from the normals pass
    // mass exchange (Eq. 10): link a reaches x + c_a = x - c_b, b = opp(a), whose
    // type, PDF f_b streaming in and fill level are the loads of direction b
    C dm = (C)0;
    bool has_gas = false, has_liq = false;
#pragma unroll
    for (int a = 1; a < 19; ++a) {
        const int b = opp(a);
        const uint8_t tz = ty(b);
        if (tz == LIQ || tz == IFC) {
            const C e = fy[b] - fs[a];
            dm = dm + (tz == IFC ? ((C)0.5 * (phx + phy[b])) * e : e);
        }
        has_gas |= tz == GAS;
        has_liq |= tz == LIQ;
    }
    // curvature (Eq. 15): half the divergence of the face neighbours' unit
    // normals by central differences; the normal test bits of the cell
    const C* __restrict__ nr = (const C*)A.nrm;
    const C dX = nr[st.at(1, 0, 0)] - nr[st.at(-1, 0, 0)];
    const C dY = nr[S + st.at(0, 1, 0)] - nr[S + st.at(0, -1, 0)];
    const C dZ = nr[2u * S + st.at(0, 0, 1)] - nr[2u * S + st.at(0, 0, -1)];
    const C kappa = (C)0.25 * ((dX + dY) + dZ);
    const unsigned nmk = A.nmask[g];
    // gas velocity: that of the cell's own post-collision PDFs
    C rs, jsx, jsy, jsz;
    moments<C>(fs, rs, jsx, jsy, jsz);
    const C ugx = jsx / rs, ugy = jsy / rs, ugz = jsz / rs;
    const C usg = ugx * ugx + ugy * ugy + ugz * ugz;
    const C rg = (C)3 * (pv + R.sigma2 * kappa);
    // stream with bounce-back and reconstruction
    C fin[19];
    fin[0] = fs[0];
#pragma unroll
    for (int a = 1; a < 19; ++a) {
        const C fsb = fs[opp(a)];
        const uint8_t tya = ty(a);
        if (tya == OBS) {
            fin[a] = fsb;
        } else if (tya == LID) {
            const C cuw = ((C)cx(a) * R.lid[0] + (C)cy(a) * R.lid[1]) + (C)cz(a) * R.lid[2];
            fin[a] = fsb + ((C)6 * weightc<C>(a)) * cuw;
        } else {
            C fp, fm;
            feq_pair<C>(a, rg, ugx, ugy, ugz, usg, fp, fm);
            const C fga = (a & 1) ? fp + fm : fp - fm;
            const C fgb = (a & 1) ? fp - fm : fp + fm;
            if (tya == GAS) {
                fin[a] = (fga + fgb) - fsb;
            } else {
                fin[a] = fy[a];
                if (D.normal_rule && ((nmk >> a) & 1u)) fin[a] = (fga + fgb) - fsb;
            }
        }
    }
    // collision (Eq. 6) and the outputs
    C rho;
    if (D.has_force) {
        const CollidePrep<C> P = collide_prep<C, true>(fin, R.g[0], R.g[1], R.g[2]);
        rho = P.rho;
#pragma unroll
        for (int a = 0; a < 19; ++a)
            Form<T>::st(dst + ((unsigned)a * S + (unsigned)g), a, collide_out<C, true>(a, fin, P, R.omp, R.omm));
    } else {
        const CollidePrep<C> P = collide_prep<C, false>(fin, (C)0, (C)0, (C)0);
        rho = P.rho;
#pragma unroll
        for (int a = 0; a < 19; ++a)
            Form<T>::st(dst + ((unsigned)a * S + (unsigned)g), a, collide_out<C, false>(a, fin, P, R.omp, R.omm));
    }
    if (!(rho == rho)) set_status(A.status, ST_NAN);
    // the cell mass accumulates in FP64 for every form; fill / empty marks
    const double mnew = m0 + (double)dm;
    A.m[g] = mnew;
    A.rhoi[g] = (double)rho;
    bool filled, emptied;
    if constexpr (sizeof(C) == 8) {
        filled = mnew > (1.0 + D.eps) * rho;
        emptied = mnew < (-D.eps) * rho;
    } else {
        const float mf = (float)mnew;
        filled = mf > (1.f + D.feps) * rho;
        emptied = mf < (-D.feps) * rho;
    }
    uint8_t mk = MK_NONE;
    if (filled) mk = MK_FILLED;
    else if (emptied) mk = MK_EMPTIED;
    else if (D.lonely_rule) {
        if (!has_gas) mk = MK_FILLED;
        else if (!has_liq) mk = MK_EMPTIED;
    }
    A.mark[g] = mk;
    return mk != MK_NONE;
}

// The interface cells of the list, one per thread, by a resident grid (block
// b takes list entries b IB .. b IB + IB - 1, then those a grid further).
template <typename T, bool ONE>
__global__ void __launch_bounds__(IfThreads<T>::n, sizeof(T) == 8 ? 4 : 5) k_iface(StepArgs A) {
    constexpr int IB = IfThreads<T>::n;
    pdl_trigger();   // the conversion kernel may be placed as blocks finish
    if (blockIdx.x == 0) step_counters(A);
    const int cnt = *A.icount;
    for (long long base = (long long)blockIdx.x * IB; base < cnt; base += (long long)gridDim.x * IB) {
        const long long i = base + threadIdx.x;
        bool mk = false;
        long long g = 0;
        if (i < cnt) {
            g = A.ilist[i];
            mk = iface_one<T, ONE>(A, g);
        }
        list_append(A.mlist, A.mcount, mk, (int)g);
    }
}

__device__ inline unsigned ifc_mask16(const uint8_t* flag, long long j);

// Tile-fused form: block b takes the TPB tiles of super-tile b.  It streams
// and collides their liquid cells, lists their interface cells in shared
// memory (ballot compaction), then processes those one per thread.  The
// interface cells' neighbour data is what the block has just read, and both
// kinds of stores to a 32-byte sector meet in L2 before it is written back.
template <typename T, bool ONE, int TPB>
__global__ void __launch_bounds__(FSL_BLOCK, 2) k_stream_tile(StepArgs A) {
    constexpr long long TILE = Form<T>::shifted ? 2 * FSL_BLOCK : FSL_BLOCK;
    constexpr int SUPER = (int)(TPB * TILE);
    __shared__ int il[SUPER];
    __shared__ int nil;
    pdl_trigger();   // the conversion kernel may be placed as blocks finish
    if (blockIdx.x == 0) step_counters(A);
    if (threadIdx.x == 0) nil = 0;
    __syncthreads();
    const long long c0 = (long long)blockIdx.x * SUPER;
#pragma unroll 1
    for (int k = 0; k < TPB; ++k) {
        const long long tile = (long long)blockIdx.x * TPB + k;
        if (tile * TILE >= A.stride) break;
        if constexpr (Form<T>::shifted) liquid_pairs<T, ONE>(A, tile);
        else liquid_single<T, ONE>(A, tile);
    }
    // the super-tile's interface cells (a 16-byte load of types per thread)
    const unsigned lane = threadIdx.x & 31u;
    for (long long j = c0 / 16 + threadIdx.x; j < (c0 + SUPER) / 16; j += FSL_BLOCK) {
        const unsigned m = j * 16 < A.stride ? ifc_mask16(A.flag, j) : 0u;
        const int n = __popc(m);
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (unsigned)o) incl += y;
        }
        int base = 0;
        if (lane == 31) base = atomicAdd(&nil, incl);
        base = __shfl_sync(0xffffffffu, base, 31);
        int pos = base + incl - n;
        for (unsigned b = m; b; b &= b - 1) il[pos++] = (int)(16 * j + (__ffs(b) - 1));
    }
    __syncthreads();
    const int ni = nil;
    for (int i0 = 0; i0 < ni; i0 += FSL_BLOCK) {
        const int i = i0 + threadIdx.x;
        bool mk = false;
        long long g = 0;
        if (i < ni) {
            g = il[i];
            mk = iface_one<T, ONE>(A, g);
        }
        list_append(A.mlist, A.mcount, mk, (int)g);
    }
}

// The liquid cells only (a tile per block), for the two-kernel form.
template <typename T, bool ONE>
__global__ void __launch_bounds__(FSL_BLOCK, 3) k_liquid(StepArgs A) {
    if constexpr (Form<T>::shifted) liquid_pairs<T, ONE>(A, (long long)blockIdx.x);
    else liquid_single<T, ONE>(A, (long long)blockIdx.x);
}

// The stream-collide step (Eqs. 6, 7, 10, 11) as one kernel: blocks
// [0, nif) take the interface cells from the list (they are launched first,
// so they are placed first), the other blocks the liquid cells.
template <typename T, bool ONE>
__global__ void __launch_bounds__(FSL_BLOCK, sizeof(T) == 8 ? 2 : FSL_STREAM_MINB) k_stream(StepArgs A, int nif) {
    __shared__ IfStage<T> sh;
    pdl_trigger();   // the conversion kernel may be placed as blocks finish
    if ((int)blockIdx.x < nif) {
        interface_cells<T, ONE>(A, (int)blockIdx.x, nif, sh);
    } else if constexpr (Form<T>::shifted) {
        liquid_pairs<T, ONE>(A, (long long)blockIdx.x - nif);
    } else {
        liquid_single<T, ONE>(A, (long long)blockIdx.x - nif);
    }
}

// Persistent form of the stream-collide kernel: a grid of resident blocks
// walks one sequence of work items in which the interface chunks (N list
// cells each) are spread evenly among the liquid items (LT tiles each): with
// nI chunks and nL liquid items, M = nI + nL, item w is chunk floor(w nI / M)
// when floor((w + 1) nI / M) > floor(w nI / M), else liquid item
// w - floor(w nI / M).  Block b takes items b, b + grid, b + 2 grid, ...  Every
// block does both kinds of work (the interface cells' latency chains overlap
// the liquid cells' streaming), and with the interface list in cell order the
// items in flight at any time lie close together in the lattice.  Results are
// those of the split form: every cell runs the same arithmetic.
template <typename T, bool ONE, int LT>
__global__ void __launch_bounds__(FSL_BLOCK, sizeof(T) == 8 ? 2 : FSL_STREAM_MINB) k_stream_pers(StepArgs A) {
    __shared__ IfStage<T> sh;
    pdl_trigger();   // the conversion kernel may be placed as blocks finish
    if (blockIdx.x == 0) step_counters(A);
    constexpr int N = IfCells<T>::n;
    constexpr long long TILE = Form<T>::shifted ? 2 * FSL_BLOCK : FSL_BLOCK;
    const int cnt = *A.icount;
    const long long nI = (cnt + N - 1) / N;
    const long long ntile = (A.stride + TILE - 1) / TILE;
    const long long nL = (ntile + LT - 1) / LT;
    const long long M = nI + nL;
    for (long long w = blockIdx.x; w < M; w += gridDim.x) {
        const long long c0 = (w * nI) / M, c1 = ((w + 1) * nI) / M;
        if (c1 > c0) {
            interface_chunk<T, ONE>(A, (int)(c0 * N), cnt, sh);
        } else {
            const long long t0 = (w - c0) * LT;
#pragma unroll 1
            for (int k = 0; k < LT; ++k) {
                const long long tile = t0 + k;
                if (tile >= ntile) break;
                if constexpr (Form<T>::shifted) liquid_pairs<T, ONE>(A, tile);
                else liquid_single<T, ONE>(A, tile);
            }
        }
    }
}

// First position in the (cell-ordered) interface list whose cell is >= cell.
__device__ inline int list_lower_bound(const int* list, int n, long long cell) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((long long)list[mid] < cell) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Slab form of the persistent stream-collide kernel (needs the interface list
// in cell order): block b owns the contiguous tiles [T b / grid, T (b + 1) /
// grid) and processes its liquid tiles and the interface cells that lie in
// them (a list range found by binary search), the two interleaved in
// proportion as in k_stream_pers.  A block works through one region of the
// lattice, so the neighbour data of its interface cells is mostly data its
// own liquid tiles and earlier chunks have just brought into its SM.
template <typename T, bool ONE>
__global__ void __launch_bounds__(FSL_BLOCK, sizeof(T) == 8 ? 2 : FSL_STREAM_MINB) k_stream_slab(StepArgs A) {
    __shared__ IfStage<T> sh;
    __shared__ int range[2];
    pdl_trigger();   // the conversion kernel may be placed as blocks finish
    if (blockIdx.x == 0) step_counters(A);
    constexpr int N = IfCells<T>::n;
    constexpr long long TILE = Form<T>::shifted ? 2 * FSL_BLOCK : FSL_BLOCK;
    const int cnt = *A.icount;
    const long long ntile = (A.stride + TILE - 1) / TILE;
    const long long t0 = ntile * blockIdx.x / gridDim.x, t1 = ntile * (blockIdx.x + 1) / gridDim.x;
    if (threadIdx.x < 2)
        range[threadIdx.x] = list_lower_bound(A.ilist, cnt, (threadIdx.x == 0 ? t0 : t1) * TILE);
    __syncthreads();
    const int l0 = range[0], l1 = range[1];
    const long long nI = (l1 - l0 + N - 1) / N;
    const long long nL = t1 - t0;
    const long long M = nI + nL;
    for (long long w = 0; w < M; ++w) {
        const long long c0 = (w * nI) / M, c1 = ((w + 1) * nI) / M;
        if (c1 > c0) {
            interface_chunk<T, ONE>(A, l0 + (int)(c0 * N), l1, sh);
        } else {
            const long long tile = t0 + (w - c0);
            if constexpr (Form<T>::shifted) liquid_pairs<T, ONE>(A, tile);
            else liquid_single<T, ONE>(A, tile);
        }
    }
}

// Stream-collide kernel forms (the autotuner picks one per workload): the split
// form (interface blocks first, then one block per liquid tile), the
// persistent form with 1, 2 or 4 tiles per liquid item, the slab form, the
// two-kernel form (liquid kernel, then one thread per interface cell), the
// tile-fused form with 2 or 4 tiles per block, and the two kernels run side by
// side on two streams.
enum { SC_SPLIT = 0, SC_PERS1 = 1, SC_PERS2 = 2, SC_PERS4 = 3, SC_SLAB = 4, SC_TWO = 5, SC_TILE2 = 6, SC_TILE4 = 7,
       SC_TWOC = 8, SC_FORMS = 9 };

// First neighbour of cell z (direction order) that is an interface cell
// carrying mark `want`, or -1.
//
// The neighbour scans below load all eighteen neighbours first and then test
// them (one memory latency, not one per neighbour): bit a of the mask is set
// when neighbour a (1-18) is an interface cell carrying mark `want`.
__device__ inline unsigned marked_mask(const StepArgs& A, const Cell& c, uint8_t want) {
    uint8_t fl[19], mk[19];
#pragma unroll
    for (int a = 1; a < 19; ++a) {
        const long long w = c.at(cx(a), cy(a), cz(a));
        fl[a] = A.flag[w];
        mk[a] = A.mark[w];
    }
    unsigned m = 0;
#pragma unroll
    for (int a = 1; a < 19; ++a) m |= (unsigned)(ctype(fl[a]) == IFC && mk[a] == want) << a;
    return m;
}
__device__ inline long long first_marked(const StepArgs& A, const Dom& D, long long z, uint8_t want) {
    const Cell c = make_cell(D, z);
    const unsigned m = marked_mask(A, c, want);
    if (m == 0) return -1;
    const int a = __ffs(m) - 1;
    return c.at(rcx(a), rcy(a), rcz(a));
}

// An interface cell carrying an emptied mark that phase A does not cancel (no
// filled neighbour).  Written as a test on the marks the interface kernel
// set, so it holds whether or not another thread has already cleared the
// cancelled mark.
__device__ inline bool still_emptied(const StepArgs& A, const Dom& D, long long w) {
    const uint8_t fw = A.flag[w], mw = A.mark[w];
    const unsigned filled = marked_mask(A, make_cell(D, w), MK_FILLED);   // loaded with w's own
    return ctype(fw) == IFC && mw == MK_EMPTIED && filled == 0;
}

// Conversion phases A and B (Sec. 2.2, cell conversion), one thread per
// (marked cell, direction).  A filled cell turns the gas neighbour in that
// direction into interface when it is that neighbour's first filled neighbour
// in direction order (so each new cell is claimed once) and initialises it
// with f = f_eq of the mean density and velocity of its liquid and
// non-emptied interface neighbours, m = 0; it also cancels an emptied mark
// there.  An emptied cell with no filled neighbour turns the liquid neighbour
// in that direction into interface when it is that neighbour's first such
// emptied neighbour: the new cell keeps its PDFs, takes m = rho and joins the
// emptied cell's bubble.
template <typename T>
__device__ inline void convert_ab_phase(const StepArgs& A) {
    using C = typename Form<T>::C;
    const int nm = *A.mcount;
    const int total = 18 * nm;
    const long long S = A.stride;
    T* f = (T*)A.fdst;
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < total; base += stride) {
        const int t = base + threadIdx.x;
        bool gclaim = false, lclaim = false;
        long long z = 0;
        if (t < total) {
            const long long p = A.mlist[t / 18];
            const int a = 1 + t % 18;
            const int d = block_dom(A, p);
            const Dom& D = get_dom(A, d);
            const uint8_t mp = A.mark[p];
            const Cell c = make_cell(D, p);
            z = c.at(rcx(a), rcy(a), rcz(a));
            const uint8_t tz = ctype(A.flag[z]);
            if (mp == MK_FILLED) {
                if (tz == GAS) {
                    if (first_marked(A, D, z, MK_FILLED) == p) {
                        gclaim = true;
                        // f = f_eq of the mean density and velocity of the liquid
                        // and non-emptied interface neighbours, in direction order
                        const Cell cz_ = make_cell(D, z);
                        // which neighbours enter the mean: types and marks of all
                        // eighteen first, the cancellation test only for the
                        // emptied ones
                        uint8_t fl[19], mk[19];
#pragma unroll
                        for (int q = 1; q < 19; ++q) {
                            const long long w = cz_.at(cx(q), cy(q), cz(q));
                            fl[q] = A.flag[w];
                            mk[q] = A.mark[w];
                        }
                        unsigned use = 0, emp = 0;
#pragma unroll
                        for (int q = 1; q < 19; ++q) {
                            const uint8_t tw = ctype(fl[q]);
                            use |= (unsigned)(tw == LIQ || (tw == IFC && mk[q] != MK_EMPTIED)) << q;
                            emp |= (unsigned)(tw == IFC && mk[q] == MK_EMPTIED) << q;
                        }
                        for (unsigned e = emp; e; e &= e - 1) {
                            const int q = __ffs(e) - 1;
                            if (!still_emptied(A, D, cz_.at(rcx(q), rcy(q), rcz(q)))) use |= 1u << q;
                        }
                        C sr = (C)0, sux = (C)0, suy = (C)0, suz = (C)0;
                        int cnt = 0;
                        for (int q = 1; q < 19; ++q) {
                            const long long w = cz_.at(rcx(q), rcy(q), rcz(q));
                            if ((use >> q) & 1u) {
                                C fo[19];
#pragma unroll
                                for (int r = 0; r < 19; ++r) fo[r] = Form<T>::ld(f + (long long)r * S + w, r);
                                C rr, jx, jy, jz;
                                moments<C>(fo, rr, jx, jy, jz);
                                sr = sr + rr;
                                sux = sux + jx / rr;
                                suy = suy + jy / rr;
                                suz = suz + jz / rr;
                                ++cnt;
                            }
                        }
                        const C rbar = sr / (C)cnt;
                        const C vx = sux / (C)cnt, vy = suy / (C)cnt, vz = suz / (C)cnt;
                        C fe[19];
                        feq_all<C>(rbar, vx, vy, vz, fe);
#pragma unroll
                        for (int r = 0; r < 19; ++r) Form<T>::st(f + (long long)r * S + z, r, fe[r]);
                        A.m[z] = 0.0;
                        A.rhoi[z] = (double)rbar;
                        A.mark[z] = MK_NEWG;
                        atomicAdd((unsigned long long*)&A.nif[d], 1ull);
                    }
                } else if (tz == IFC && A.mark[z] == MK_EMPTIED) {
                    A.mark[z] = MK_NONE;
                }
            } else if (mp == MK_EMPTIED && tz == LIQ && still_emptied(A, D, p)) {
                // is p the first emptied-and-not-cancelled neighbour of z?
                const Cell cz_ = make_cell(D, z);
                long long first = -1;
                for (unsigned e = marked_mask(A, cz_, MK_EMPTIED); e && first < 0; e &= e - 1) {
                    const int q = __ffs(e) - 1;
                    const long long w = cz_.at(rcx(q), rcy(q), rcz(q));
                    if (still_emptied(A, D, w)) first = w;
                }
                if (first == p) {
                    lclaim = true;
                    double r = (double)Form<T>::ld(f + z, 0);
                    for (int q = 1; q < 19; ++q) r = r + (double)Form<T>::ld(f + (long long)q * S + z, q);
                    A.mark[z] = MK_NEWL;
                    A.id[z] = A.id[p];
                    bbox_extend(A.bbox, A.id[p], cz_.x, cz_.y, cz_.z);
                    A.m[z] = r;
                    A.rhoi[z] = r;
                    atomicAdd((unsigned long long*)&A.nif[d], 1ull);
                }
            }
        }
        list_append(A.glist, A.gcount, gclaim, (int)z);
        list_append(A.llist, A.lcount, lclaim, (int)z);
    }
}

// Sum v over the lanes of the warp that share a key into base[key], one
// atomic per distinct key (the values are fixed point, so the order of the
// additions does not matter); key < 0 contributes nothing.  Every lane of the
// warp must call.
__device__ inline void warp_add(long long* base, int key, long long v) {
    const unsigned full = 0xffffffffu;
    const int k0 = __shfl_sync(full, key, 0);
    if (__all_sync(full, key == k0)) {
        if (k0 < 0) return;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(full, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0) atomicAdd((unsigned long long*)&base[k0], (unsigned long long)v);
        return;
    }
    const unsigned peers = __match_any_sync(full, key);
    long long sum = 0;
    for (unsigned m = peers; m; m &= m - 1) sum += __shfl_sync(peers, v, __ffs(m) - 1);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1 && key >= 0 && sum != 0)
        atomicAdd((unsigned long long*)&base[key], (unsigned long long)sum);
}

// 3x3x3 cube around a cell, bit k = (dx+1) + 3 (dy+1) + 9 (dz+1); bit 13 is the
// centre.  Face or edge neighbours of cube cell k inside the cube, the centre
// left out (a walk must not pass through the removed cell).
__host__ __device__ constexpr unsigned cube_adj18(int k) {
    const int kx = k % 3 - 1, ky = (k / 3) % 3 - 1, kz = k / 9 - 1;
    unsigned a = 0;
    for (int j = 0; j < 27; ++j) {
        const int ax = j % 3 - 1 - kx, ay = (j / 3) % 3 - 1 - ky, az = j / 9 - 1 - kz;
        if (ax < -1 || ax > 1 || ay < -1 || ay > 1 || az < -1 || az > 1) continue;
        const int dist = (ax != 0) + (ay != 0) + (az != 0);
        if (dist >= 1 && dist <= 2) a |= 1u << j;
    }
    return a & ~(1u << 13);
}
// the table, folded at compile time
__constant__ static const unsigned c_cube_adj18[27] = {
    cube_adj18(0),  cube_adj18(1),  cube_adj18(2),  cube_adj18(3),  cube_adj18(4),  cube_adj18(5),  cube_adj18(6),
    cube_adj18(7),  cube_adj18(8),  cube_adj18(9),  cube_adj18(10), cube_adj18(11), cube_adj18(12), cube_adj18(13),
    cube_adj18(14), cube_adj18(15), cube_adj18(16), cube_adj18(17), cube_adj18(18), cube_adj18(19), cube_adj18(20),
    cube_adj18(21), cube_adj18(22), cube_adj18(23), cube_adj18(24), cube_adj18(25), cube_adj18(26)};

// bits of the 18 face / edge neighbours of the centre
__host__ __device__ constexpr unsigned cube_mask18() {
    unsigned m = 0;
    for (int k = 0; k < 27; ++k) {
        const int dk = (k % 3 != 1) + ((k / 3) % 3 != 1) + (k / 9 != 1);
        if (dk >= 1 && dk <= 2) m |= 1u << k;
    }
    return m;
}

// Local test that removing the filled cell at the centre of the cube cannot
// split its bubble: the gas/interface cells among its 18 neighbours must stay
// connected inside the cube (18-connectivity) without the centre.
__device__ inline bool removal_is_local(unsigned fg) {
    constexpr unsigned kMask18 = cube_mask18();
    const unsigned targets = fg & kMask18;
    if (targets == 0) return true;
    unsigned reach = targets & (~targets + 1u);   // lowest target
    for (int it = 0; it < 27; ++it) {
        unsigned grow = reach;
        unsigned r = reach;
        while (r) {
            const int k = __ffs(r) - 1;
            r &= r - 1;
            grow |= c_cube_adj18[k];
        }
        grow &= fg;
        if (grow == reach) break;
        reach = grow;
    }
    return (targets & ~reach) == 0;
}

// ------------------------------------------- interface list in cell order
// On lattices much larger than the L2 cache the next step's interface list is
// rebuilt from the cell types after phase D, in increasing cell index, so that
// the stream-collide work items in flight at any time lie close together and
// share their neighbours' data in L2 (the list phase D appends is in the order
// its warps finish).  Block b of the conversion kernel owns 16-cell groups
// [G b / nb, G (b + 1) / nb), G = cells / 16 (the padded lattice is a multiple
// of 256 cells, the type array 256-byte aligned).

__device__ inline void order_range(const StepArgs& A, long long& lo, long long& hi) {
    const long long G = A.stride / 16, nb = gridDim.x;
    lo = G * blockIdx.x / nb;
    hi = G * (blockIdx.x + 1) / nb;
}

// Bit k set when cell 16 j + k is an interface cell (one 16-byte load).
__device__ inline unsigned ifc_mask16(const uint8_t* flag, long long j) {
    const uint4 v = ((const uint4*)flag)[j];
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
    unsigned m = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) m |= (unsigned)(((w[k >> 2] >> (8 * (k & 3))) & K_TYPE) == IFC) << k;
    return m;
}

// Exclusive prefix sum of v over the block (a multiple of 32 threads, at most
// 1024); *total receives the block's sum.  Every thread must call; ends with
// a barrier.
__device__ inline int block_exclusive_sum(int v, int* total) {
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) wsum[lane] = t;   // inclusive sums over the warps
    }
    __syncthreads();
    const int before = w > 0 ? wsum[w - 1] : 0;
    *total = wsum[nw - 1];
    __syncthreads();                      // wsum is reused by the next call
    return before + x - v;
}

// Each thread takes OU consecutive 16-cell words per pass, loaded before use.
constexpr int OU = 4;

// Pass 1: interface cells in each block's range.
__device__ inline void order_count_phase(const StepArgs& A) {
    long long lo, hi;
    order_range(A, lo, hi);
    int n = 0;
    for (long long j0 = lo + (long long)threadIdx.x * OU; j0 < hi; j0 += (long long)blockDim.x * OU) {
        unsigned m[OU];
#pragma unroll
        for (int u = 0; u < OU; ++u) m[u] = j0 + u < hi ? ifc_mask16(A.flag, j0 + u) : 0u;
#pragma unroll
        for (int u = 0; u < OU; ++u) n += __popc(m[u]);
    }
    int tot;
    block_exclusive_sum(n, &tot);
    if (threadIdx.x == 0) A.ocnt[blockIdx.x] = tot;
}

// Pass 2: each block writes its interface cells in order after those of the
// blocks before it; the last block stores the list length.
__device__ inline void order_write_phase(const StepArgs& A) {
    long long lo, hi;
    order_range(A, lo, hi);
    int part = 0;
    for (int k = threadIdx.x; k < (int)blockIdx.x; k += blockDim.x) part += A.ocnt[k];
    int off;
    block_exclusive_sum(part, &off);
    for (long long j0 = lo; j0 < hi; j0 += (long long)blockDim.x * OU) {
        // thread t takes words jt .. jt + OU - 1, after those of the threads before it
        const long long jt = j0 + (long long)threadIdx.x * OU;
        unsigned m[OU];
        int c = 0;
#pragma unroll
        for (int u = 0; u < OU; ++u) m[u] = jt + u < hi ? ifc_mask16(A.flag, jt + u) : 0u;
#pragma unroll
        for (int u = 0; u < OU; ++u) c += __popc(m[u]);
        int tot;
        int pos = off + block_exclusive_sum(c, &tot);
#pragma unroll
        for (int u = 0; u < OU; ++u)
            for (unsigned b = m[u]; b; b &= b - 1) A.ilist_next[pos++] = (int)(16 * (jt + u) + (__ffs(b) - 1));
        off += tot;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *A.icount_next = off;
}

// Scratch of the connected-component labelling and bubble-table rebuild.  A
// pass after initialisation labels only the cells of the bubbles that phase C
// marked (a merge or split may involve them); the other bubbles keep their
// slots and table rows.  Slots are recycled through a stack per domain.
struct CclArgs {
    int* lab;                    // union-find parent per cell (global index), -1 outside the pass
    int* aux;                    // new slot of each root cell
    unsigned long long* hkeys;   // (new slot << 32 | old slot) overlap keys, ~0 empty
    long long* hvals;            // overlap volumes V_{c,b}, fixed point
    long long hcap;              // power of two
    int* hused;                  // hash positions taken in this pass (emptied again at install)
    int* nhused;
    long long* nvfx;             // new table rows (slot-indexed, reset when a slot is handed out)
    long long* nvxfx;
    long long* nvsfx;
    long long* nncells;
    int* nconstp;
    int* croot;                  // root cell (global index) of each new slot
    long long* vtot;             // per old slot: total volume over all new components
    int* minc;                   // per old slot: lowest root among its components
    int* nused;                  // per domain: slots handed out so far (high-water mark)
    int* nfree;                  // per domain: slots on its free stack
    int* freelist;               // slot-indexed: domain d's stack at [slot_off, slot_off + cap)
    int* aff;                    // per slot: 1 while its bubble takes part in the pass, 2 when
                                 // handed out again in it, 0 otherwise
    int* afflist;                // slots marked 1 this step
    int* naff;
    int* plist;                  // cells taking part in the pass
    int* np;
    int* newslots;               // slots handed out in the pass
    int* nnew;
    long long* rowoff;           // per marked slot (afflist order): first box row of its scan
    long long* nrows;            // box rows over all marked slots
    const int* slot_dom;         // slot -> domain
    long long* runs;             // labelling passes run after initialisation, bubbles they took
    long long* vsfx;             // bubble tables written by the install phase
    int* constp;
    int initial;                 // 1: first labelling after initialisation (every bubble, V* = V)
    int max_iter;                // cap on union / find loops
};

// A merge or split may involve bubble b (slot) of domain d: b takes part in
// this step's labelling pass, which runs for the domain.
__device__ inline void mark_affected(const StepArgs& A, const CclArgs& K, int d, int b) {
    if (b >= 0 && atomicExch(&K.aff[b], 1) == 0) K.afflist[atomicAdd(K.naff, 1)] = b;
    atomicExch(&A.trig[1 + d], 1);
    atomicExch(A.trig, 1);
}

// Unit normal n = -g / |g| of the fill level at cell w (Parker-Youngs gradient
// g over the 3x3x3 stencil of the stencil fill levels), 0 where g = 0.
__device__ inline void unit_normal_at(const StepArgs& A, const Dom& D, long long w, float& nx, float& ny, float& nz) {
    const Cell c = make_cell(D, w);
    float v[27];
#pragma unroll
    for (int k = 0; k < 27; ++k) {
        const long long z = c.at(k % 3 - 1, (k / 3) % 3 - 1, k / 9 - 1);
        v[k] = A.phitf ? A.phitf[z] : (float)A.phit[z];
    }
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
#pragma unroll
        for (int a = -1; a <= 1; ++a) {
            const float W = (a == 0 && b == 0) ? 4.f : ((a == 0 || b == 0) ? 2.f : 1.f);
            gx += W * (v[2 + 3 * (a + 1) + 9 * (b + 1)] - v[0 + 3 * (a + 1) + 9 * (b + 1)]);
            gy += W * (v[(a + 1) + 3 * 2 + 9 * (b + 1)] - v[(a + 1) + 0 + 9 * (b + 1)]);
            gz += W * (v[(a + 1) + 3 * (b + 1) + 9 * 2] - v[(a + 1) + 3 * (b + 1) + 0]);
        }
    }
    const float q = gx * gx + gy * gy + gz * gz;
    const float il = q > 0.f ? -rsqrtf(q) : 0.f;
    nx = gx * il; ny = gy * il; nz = gz * il;
}

// The paper's split trigger (Sec. 2.3.2, Fig. "anti-parallel normals"): the
// cell g, which fills and becomes liquid, has two interface neighbours of its
// own bubble b (after this step's conversion) whose unit normals point in
// opposite directions (n_i . n_j < -1/2): a liquid film between two parts of
// one bubble, which may have cut it in two.
__device__ inline bool antiparallel_normals(const StepArgs& A, const Dom& D, const Cell& c, long long g, int b) {
    float nxs[18], nys[18], nzs[18];
    int k = 0;
    for (int a = 1; a < 19; ++a) {
        const long long w = c.at(rcx(a), rcy(a), rcz(a));
        if (new_type(ctype(A.flag[w]), A.mark[w]) != IFC || A.id[w] != b) continue;
        unit_normal_at(A, D, w, nxs[k], nys[k], nzs[k]);
        for (int j = 0; j < k; ++j)
            if (nxs[j] * nxs[k] + nys[j] * nys[k] + nzs[j] * nzs[k] < -0.5f) return true;
        ++k;
    }
    return false;
}

// Phase C, over the marked list and the new-from-liquid list: excess mass of
// converted cells (filled: m - rho, emptied: m) split equally among the
// neighbours that are interface after conversion, else pooled; merge / split
// triggers.  Taking the filled cells away one at a time in index order, each
// removal must pass the local test with the lower-index filled cells already
// gone and the higher-index ones still present, or the labelling runs.
__device__ inline void convert_c_phase(const StepArgs& A, const CclArgs& K) {
    const int nm = *A.mcount, nl = *A.lcount;
    const int total = nm + nl;
    const int step = *A.stepno;
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const long long g = i < nm ? A.mlist[i] : A.llist[i - nm];
        const int d = block_dom(A, g);
        const Dom& D = get_dom(A, d);
        const Cell c = make_cell(D, g);
        const uint8_t mk = A.mark[g];
        if (i < nm) {
            if (mk != MK_FILLED && mk != MK_EMPTIED) continue;   // emptied mark cancelled in phase A
            const double mex = (mk == MK_FILLED) ? A.m[g] - A.rhoi[g] : A.m[g];
            uint8_t fl[19], mz[19];
#pragma unroll
            for (int a = 1; a < 19; ++a) {
                const long long z = c.at(cx(a), cy(a), cz(a));
                fl[a] = A.flag[z];
                mz[a] = A.mark[z];
            }
            unsigned rcv = 0;
#pragma unroll
            for (int a = 1; a < 19; ++a) rcv |= (unsigned)(new_type(ctype(fl[a]), mz[a]) == IFC) << a;
            const int k = __popc(rcv);
            for (unsigned e = rcv; e; e &= e - 1) {
                const int a = __ffs(e) - 1;
                A.recv[c.at(rcx(a), rcy(a), rcz(a))] = step;   // pulls a share in phase D
            }
            if (k > 0) A.exs[g] = mex / (double)k;
            else atomicAdd((unsigned long long*)&A.pool[d], (unsigned long long)__double2ll_rn(mex * 1099511627776.0));
            if (mk == MK_FILLED) {
                unsigned fgm = 0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            if (dx == 0 && dy == 0 && dz == 0) continue;
                            const long long z = c.at(dx, dy, dz);
                            const uint8_t tz = ctype(A.flag[z]), mz = A.mark[z];
                            const uint8_t ntz = new_type(tz, mz);
                            const bool later_filled = (tz == IFC && (mz == MK_FILLED || mz == MK_CFILLED) && z > g);
                            if (ntz == GAS || ntz == IFC || later_filled)
                                fgm |= 1u << ((dx + 1) + 3 * (dy + 1) + 9 * (dz + 1));
                        }
                const bool may_split = D.split_trigger ? antiparallel_normals(A, D, c, g, A.id[g])
                                                       : !removal_is_local(fgm);
                if (may_split) mark_affected(A, K, d, A.id[g]);   // its bubble may split
            }
            A.cstep[g] = step;
            A.mark[g] = (mk == MK_FILLED) ? MK_CFILLED : MK_CEMPTIED;
            atomicAdd((unsigned long long*)&A.nif[d], (unsigned long long)-1LL);
            continue;
        }
        // new interface cell from liquid: a neighbour of another bubble merges
        const int b = A.id[g];
        uint8_t fl[19], mz[19];
        int iz[19];
#pragma unroll
        for (int a = 1; a < 19; ++a) {
            const long long z = c.at(cx(a), cy(a), cz(a));
            fl[a] = A.flag[z];
            mz[a] = A.mark[z];
            iz[a] = A.id[z];
        }
        bool merge = false;
        for (int a = 1; a < 19; ++a) {
            const uint8_t ntz = new_type(ctype(fl[a]), mz[a]);
            if ((ntz == GAS || ntz == IFC) && iz[a] != b) {
                merge = true;
                mark_affected(A, K, d, iz[a]);   // every bubble the new cell touches
            }
        }
        if (merge) mark_affected(A, K, d, b);
    }
}

// Phase D, over the interface list and the two new-interface lists: receivers
// pull the excess shares of converted neighbours in direction order and the
// pool share, phi = m / rho (Eq. 9); converted cells take their new type;
// bubble volumes change by exact fixed-point differences; the interface list
// of the next step; reservoir drain; the graph condition of the labelling.
__device__ inline void convert_d_phase(const StepArgs& A) {
    const int ni = *A.icount, ng = *A.gcount, nl = *A.lcount;
    const int total = ni + ng + nl;
    const int step = *A.stepno;
    const int stride = gridDim.x * blockDim.x;
    long long kept = 0;   // interface cells kept by this thread (one domain)
    for (int base = blockIdx.x * blockDim.x; base < total; base += stride) {
        const int i = base + threadIdx.x;
        const bool valid = i < total;
        long long g = 0;
        if (valid) g = i < ni ? A.ilist[i] : (i < ni + ng ? A.glist[i - ni] : A.llist[i - ni - ng]);
        const int d = valid ? block_dom(A, g) : 0;
        int key = -1;
        long long dv = 0;
        int ckey = -1;
        long long dc = 0;
        bool keep = false;
        if (valid) {
            // everything the cell needs, loaded together
            const uint8_t f = A.flag[g];
            const uint8_t mk = A.mark[g];
            key = A.id[g];
            const double m0 = A.m[g], rh = A.rhoi[g];
            // FP32-collide forms: fill levels and volume terms from the FP32 copies,
            // which are the only ones kept (the FP64 fill level and stencil level
            // belong to the FP64 form)
            const bool f32 = A.phif != nullptr;
            const double ph0 = f32 ? 0.0 : A.phi[g];
            const float ph0f = f32 ? A.phif[g] : 0.f;
            const int rs = A.recv[g];
            const long long nI = A.nif[d];
            const long long pool = A.pool[d];
            const uint8_t t = ctype(f);
            if (t == IFC && mk == MK_CFILLED) {
                dv = f32 ? -volume_term_f(IFC, ph0f) : -volume_term(IFC, ph0);
                ckey = key;
                dc = -1;
                A.flag[g] = (uint8_t)((f & ~K_TYPE) | LIQ);
                if (f32) { A.phif[g] = 1.f; A.phitf[g] = 1.f; }
                else { A.phi[g] = 1.0; A.phit[g] = 1.0; }
                A.id[g] = -1;
                A.mark[g] = MK_NONE;
            } else if (t == IFC && mk == MK_CEMPTIED) {
                dv = FSL_VOL_ONE - (f32 ? volume_term_f(IFC, ph0f) : volume_term(IFC, ph0));
                A.flag[g] = (uint8_t)((f & ~K_TYPE) | GAS);
                if (f32) { A.phif[g] = 0.f; A.phitf[g] = 0.f; }
                else { A.phi[g] = 0.0; A.phit[g] = 0.0; }
                A.m[g] = 0.0;
                A.mark[g] = MK_NONE;
            } else {
                double sm = m0;
                if (rs == step) {
                    // a converted neighbour listed this cell among its receivers:
                    // all eighteen step stamps first, then the shares of the
                    // converted ones, added in direction order
                    const Dom& D = get_dom(A, d);
                    const Cell c = make_cell(D, g);
                    int cs[19];
#pragma unroll
                    for (int a = 1; a < 19; ++a) cs[a] = A.cstep[c.at(cx(a), cy(a), cz(a))];
                    double ex[19];
#pragma unroll
                    for (int a = 1; a < 19; ++a) ex[a] = cs[a] == step ? A.exs[c.at(cx(a), cy(a), cz(a))] : 0.0;
#pragma unroll
                    for (int a = 1; a < 19; ++a)
                        if (cs[a] == step) sm = sm + ex[a];
                }
                if (nI > 0 && pool != 0) {
                    const double share = ((double)pool * 9.094947017729282379150390625e-13) / (double)nI;
                    sm = sm + share;
                }
                A.m[g] = sm;
                if (f32) {
                    // phi = m / rho in FP32 (Eq. 9); three conversions are the
                    // only FP64-pipe work of the cell
                    const float phf = (float)sm / (float)rh;
                    A.phif[g] = phf;
                    A.phitf[g] = fminf(fmaxf(phf, 0.f), 1.f);
                    dv = volume_term_f(IFC, phf) - volume_term_f(t, ph0f);
                } else {
                    const double phn = sm / rh;
                    const long long told = volume_term(t, ph0);
                    A.phi[g] = phn;
                    A.phit[g] = phn < 0.0 ? 0.0 : (phn > 1.0 ? 1.0 : phn);
                    dv = volume_term(IFC, phn) - told;
                }
                if (t != IFC) A.flag[g] = (uint8_t)((f & ~K_TYPE) | IFC);
                if (t == LIQ) { ckey = key; dc = 1; }
                keep = true;
            }
        }
        warp_add(A.vfx, dv != 0 ? key : -1, dv);
        warp_add(A.ncells, ckey, dc);
        if (A.ndom == 1) kept += keep ? 1 : 0;
        else warp_add(A.icnt, keep ? d : -1, 1);
        if (!A.order) list_append(A.ilist_next, A.icount_next, keep, (int)g);
    }
    if (A.ndom == 1) {
        // one domain: the interface count by one atomic per warp
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) kept += __shfl_down_sync(0xffffffffu, kept, o);
        if ((threadIdx.x & 31) == 0 && kept) atomicAdd((unsigned long long*)&A.icnt[0], (unsigned long long)kept);
    }
    if (blockIdx.x == 0) {
        // reservoir drain of every domain whose seed cell is still gas or
        // interface (types read through the marks, which stay consistent
        // while other threads update the flags), one thread per domain
        for (int d = threadIdx.x; d < A.ndom; d += blockDim.x) {
            const Dom& D = get_dom(A, d);
            if (D.seed < 0) continue;
            const long long gs = D.off + D.seed;
            const uint8_t nt = new_type(ctype(A.flag[gs]), A.mark[gs]);
            const int b = A.id[gs];
            if ((nt == GAS || nt == IFC) && b >= 0)
                atomicAdd((unsigned long long*)&A.vxfx[b], (unsigned long long)(-D.rate_fx));
        }
        if (threadIdx.x == 0) *A.mcount = 0;
    }
}



// --------------------------------------------- connected-component labelling
// Bubbles are the 18-connected components of gas + interface cells (Sec. 2.3);
// the paper's serial flood fill and its colour unification across processes
// (Sec. 2.4.1) become one lock-free union-find over the whole lattice whose
// roots are the minimum cell index of each component.  Each phase below walks
// the tiles (256 cells) of the domains taking part, one cell per thread of a
// 256-thread block (a tile lies in one domain), or a table with a
// thread-stride loop, so that it runs both as a kernel of its own and inside
// the conversion kernel.

__device__ inline bool is_fg(uint8_t f) { return ctype(f) == GAS || ctype(f) == IFC; }

// Root of a; halves the path on the way (each cell is pointed at its
// grandparent).  Only the hook phase uses it: there a cell's parent changes
// only from itself (a root) to a smaller root, so every ancestor a thread has
// read stays an ancestor and a halving store, however late, keeps the cell in
// its tree.
__device__ inline int find_root(int* L, int a, int cap, bool& ok) {
    for (int it = 0; it < cap; ++it) {
        const int p = L[a];
        if (p == a) return a;
        const int gp = L[p];
        if (gp != p) L[a] = gp;
        a = gp;
    }
    ok = false;
    return a;
}

// Root of a without writing (parents have smaller indices, so the walk ends).
// The compress phase uses this one: a halving store there could land after
// the cell's own thread has stored the root, and leave an inner node behind.
__device__ inline int find_root_ro(const int* L, int a, int cap, bool& ok) {
    for (int it = 0; it < cap; ++it) {
        const int p = L[a];
        if (p == a) return a;
        a = p;
    }
    ok = false;
    return a;
}

// Lock-free union: hook the larger root under the smaller one by a
// compare-and-swap that succeeds only while it is still a root (a non-root's
// parent is never rewritten), so the final root of every component is its
// minimum cell index.
__device__ inline bool unite(int* L, int a, int b, int cap) {
    bool ok = true;
    for (int it = 0; it < cap && ok; ++it) {
        a = find_root(L, a, cap, ok);
        b = find_root(L, b, cap, ok);
        if (!ok) return false;
        if (a == b) return true;
        if (a < b) { const int tt = a; a = b; b = tt; }
        if (atomicCAS(&L[a], a, b) == a) return true;
        // a was hooked by another thread meanwhile: find both roots again
    }
    return false;
}

// First tile and tile count of domain d (read field by field).
__device__ inline long long dom_tile0(const StepArgs& A, int d) {
    return (A.ndom == 1 ? A.d0.off : A.doms[d].off) / FSL_BLOCK;
}
__device__ inline long long dom_ntiles(const StepArgs& A, int d) {
    return ((long long)(A.ndom == 1 ? A.d0.n : A.doms[d].n) + FSL_BLOCK - 1) / FSL_BLOCK;
}

// Grid-stride loop over a device-counted list: every lane of a warp runs the
// same iterations (i >= n on the lanes past the end), so warp collectives may
// be used in the body.
#define FSL_LIST_LOOP(i, n)                                                                                  \
    for (long long base_ = (long long)blockIdx.x * blockDim.x, i = base_ + threadIdx.x; base_ < (n);      \
         base_ += (long long)gridDim.x * blockDim.x, i = base_ + threadIdx.x)

// Phase 0 (passes after the initial one): block 0 lays the box rows of the
// marked bubbles end to end, rowoff[k] = rows of the boxes of afflist[0 .. k).
__device__ inline void ccl_rows_phase(const StepArgs& A, const CclArgs& K) {
    if (blockIdx.x != 0) return;
    const int na = *K.naff;
    long long base = 0;
    for (int k0 = 0; k0 < na; k0 += blockDim.x) {
        const int k = k0 + (int)threadIdx.x;
        long long rows = 0;
        if (k < na) {
            const int* q = A.bbox + 6 * (long long)K.afflist[k];
            if (q[3] >= q[0]) rows = (long long)(q[4] - q[1] + 1) * (long long)(q[5] - q[2] + 1);
        }
        // block-wide exclusive sum of the row counts (64-bit, warp shuffles
        // and one shared word per warp)
        __shared__ long long ws[32];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        long long x = rows;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[w] = x;
        __syncthreads();
        long long before = 0, tot = 0;
        for (int v = 0; v < nw; ++v) {
            if (v < w) before += ws[v];
            tot += ws[v];
        }
        if (k < na) K.rowoff[k] = base + before + x - rows;
        base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *K.nrows = base;
}

// Phase 1: the cells taking part start as their own roots and are listed.  In
// the initial pass that is every gas / interface cell (a scan of the whole
// lattice, one cell per thread of a 256-thread block, which also writes -1
// into the labels of the other cells).  Afterwards it is the cells of the
// bubbles phase C marked, found by scanning only their boxes, a warp per box
// row (a cell is listed by the box of its own bubble, so at most once); the
// labels of all other cells are -1 already (each pass resets those it set),
// and the marked slots go onto their domains' free stacks.  A marked bubble's
// cells touch no gas or interface cell outside the pass: two bubbles become
// adjacent only through a new interface cell from liquid, and phase C marks
// every bubble around such a cell.
__device__ inline void ccl_init_phase(const StepArgs& A, const CclArgs& K) {
    if (K.initial) {
        for (long long tile = blockIdx.x; tile < A.stride / FSL_BLOCK; tile += gridDim.x) {
            const long long g = tile * FSL_BLOCK + threadIdx.x;
            const bool part = is_fg(A.flag[g]);
            K.lab[g] = part ? (int)g : -1;
            list_append(K.plist, K.np, part, (int)g);
        }
        return;
    }
    const int na = *K.naff;
    const long long nrows = *K.nrows;
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < nrows; r += nwarps) {
        // the marked slot whose rows hold r: the last k with rowoff[k] <= r
        int lo = 0, hi = na - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (K.rowoff[mid] <= r) lo = mid;
            else hi = mid - 1;
        }
        const int b = K.afflist[lo];
        const int* q = A.bbox + 6 * (long long)b;
        const long long ri = r - K.rowoff[lo];
        const int nyb = q[4] - q[1] + 1;
        const int y = q[1] + (int)(ri % nyb), z = q[2] + (int)(ri / nyb);
        const Dom& D = get_dom(A, K.slot_dom[b]);
        const long long row = D.off + (long long)D.nx * ((long long)y + (long long)D.ny * z);
        for (int x0 = q[0]; x0 <= q[3]; x0 += 32) {
            const int x = x0 + lane;
            const long long g = row + x;
            bool part = false;
            if (x <= q[3] && is_fg(A.flag[g])) part = A.id[g] == b;
            if (part) K.lab[g] = (int)g;
            list_append(K.plist, K.np, part, (int)g);
        }
    }
    FSL_LIST_LOOP(i, na) {
        if (i >= na) continue;
        const int b = K.afflist[i];
        const Dom& D = get_dom(A, K.slot_dom[b]);
        K.freelist[D.slot_off + atomicAdd(&K.nfree[K.slot_dom[b]], 1)] = b;
        K.vtot[b] = 0;
        K.minc[b] = INT_MAX;
    }
}

// Phase 2: unions over the 18-neighbourhood (the nine directions 1, 3, ...,
// 17 cover each neighbour pair once).
__device__ inline void ccl_hook_phase(const StepArgs& A, const CclArgs& K) {
    const int np = *K.np;
    FSL_LIST_LOOP(i, np) {
        if (i >= np) continue;
        const long long g = K.plist[i];
        const Dom& D = get_dom(A, block_dom(A, g));
        const Cell c = make_cell(D, g);
        for (int a = 1; a < 19; a += 2) {
            const long long h = c.at(rcx(a), rcy(a), rcz(a));
            if (K.lab[h] >= 0 && !unite(K.lab, (int)g, (int)h, K.max_iter)) {
                set_status(A.status, ST_CCL);
                break;
            }
        }
    }
}

// Phase 3: every cell onto its root; each root takes a slot (from its
// domain's free stack, else a fresh one) and resets that slot's new row.
__device__ inline void ccl_compress_phase(const StepArgs& A, const CclArgs& K) {
    const int np = *K.np;
    FSL_LIST_LOOP(i, np) {
        if (i >= np) continue;
        const long long g = K.plist[i];
        bool ok = true;
        const int r = find_root_ro(K.lab, (int)g, K.max_iter, ok);
        if (!ok) { set_status(A.status, ST_CCL); continue; }
        K.lab[g] = r;
        if (r != (int)g) continue;
        const int d = block_dom(A, g);
        const Dom& D = get_dom(A, d);
        int sl = -1;
        const int k = K.initial ? -1 : atomicSub(&K.nfree[d], 1) - 1;
        if (k >= 0) {
            sl = K.freelist[D.slot_off + k];
        } else {
            const int j = atomicAdd(&K.nused[d], 1);
            if (j < D.slot_cap) sl = D.slot_off + j;
            else set_status(A.status, ST_TABLE_FULL);
        }
        K.aux[g] = sl;
        if (sl < 0) continue;
        K.aff[sl] = 2;
        K.croot[sl] = r;
        int* q = A.bbox + 6 * (long long)sl;
        q[0] = INT_MAX; q[1] = INT_MAX; q[2] = INT_MAX; q[3] = INT_MIN; q[4] = INT_MIN; q[5] = INT_MIN;
        K.nvfx[sl] = 0; K.nvxfx[sl] = 0; K.nvsfx[sl] = 0; K.nncells[sl] = 0; K.nconstp[sl] = 0;
        K.newslots[atomicAdd(K.nnew, 1)] = sl;
    }
}

// Grow the box of slot c by cell g, every lane of the warp calling (c < 0:
// nothing): the lanes with the same slot reduce their coordinates first, so a
// warp of one bubble's cells costs six atomics.
__device__ inline void warp_bbox(const StepArgs& A, long long g, int c) {
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    int x = 0, y = 0, z = 0;
    if (c >= 0) {
        const Dom& D = get_dom(A, block_dom(A, g));
        local_xyz(D, (int)(g - D.off), x, y, z);
    }
    const int mnx = __reduce_min_sync(peers, x), mny = __reduce_min_sync(peers, y), mnz = __reduce_min_sync(peers, z);
    const int mxx = __reduce_max_sync(peers, x), mxy = __reduce_max_sync(peers, y), mxz = __reduce_max_sync(peers, z);
    if (c >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
        int* q = A.bbox + 6 * (long long)c;
        atomicMin(q + 0, mnx); atomicMin(q + 1, mny); atomicMin(q + 2, mnz);
        atomicMax(q + 3, mxx); atomicMax(q + 4, mxy); atomicMax(q + 5, mxz);
    }
}

__device__ inline void hash_add(const CclArgs& K, unsigned long long key, long long v, int* status) {
    unsigned long long h = key * 0x9E3779B97F4A7C15ull;
    long long pos = (long long)(h >> 20) & (K.hcap - 1);
    for (long long probe = 0; probe < K.hcap; ++probe) {
        const unsigned long long prev = atomicCAS(&K.hkeys[pos], ~0ull, key);
        if (prev == ~0ull || prev == key) {
            if (prev == ~0ull) K.hused[atomicAdd(K.nhused, 1)] = (int)pos;
            atomicAdd((unsigned long long*)&K.hvals[pos], (unsigned long long)v);
            return;
        }
        pos = (pos + 1) & (K.hcap - 1);
    }
    set_status(status, ST_TABLE_FULL);
}

// Phase 4: new volumes and cell counts per component, overlap volumes V_{c,b}
// of new component c with old bubble b, new slots into the id field.
__device__ inline void ccl_pairs_phase(const StepArgs& A, const CclArgs& K) {
    const int np = *K.np;
    FSL_LIST_LOOP(i, np) {
        const bool valid = i < np;
        const long long g = valid ? K.plist[i] : 0;
        int c = -1;
        long long term = 0;
        if (valid) {
            // the slot of the cell's root; -1 when a find gave up at its
            // iteration cap (the pass has then latched ST_CCL and r may be an
            // inner node whose aux entry was never written)
            const int r = K.lab[g];
            c = (r >= 0 && K.lab[r] == r) ? K.aux[r] : -1;
            const uint8_t ty = ctype(A.flag[g]);
            term = A.phif ? volume_term_f(ty, A.phif[g]) : volume_term(ty, A.phi[g]);
        }
        warp_add(K.nvfx, c, term);
        warp_add(K.nncells, c, c >= 0 ? 1 : 0);
        warp_bbox(A, valid ? g : -1, c);
        if (c < 0) continue;
        if (!K.initial && A.id[g] >= 0) {
            const int b = A.id[g];
            const unsigned long long key = ((unsigned long long)(unsigned)c << 32) | (unsigned)b;
            hash_add(K, key, term, A.status);
            atomicAdd((unsigned long long*)&K.vtot[b], (unsigned long long)term);
            atomicMin(&K.minc[b], K.lab[g]);
            const Dom& D = get_dom(A, block_dom(A, g));
            if (D.seed >= 0 && g - D.off == D.seed) {
                const long long x = A.vxfx[b];
                hash_add(K, key, x, A.status);
                atomicAdd((unsigned long long*)&K.vtot[b], (unsigned long long)x);
                K.nvxfx[c] = x;
            }
        }
        A.id[g] = c;
    }
}

// Phase 5: V*_c = sum over b of V*_b V_{c,b} / V_b, V*_b copied when c holds
// all of b (Secs. 2.3.1, 2.3.2); a component touching a constant-pressure
// bubble stays constant-pressure.
__device__ inline void ccl_table_phase(const StepArgs& A, const CclArgs& K) {
    const int nh = *K.nhused;
    FSL_LIST_LOOP(i, nh) {
        if (i >= nh) continue;
        const long long h = K.hused[i];
        const unsigned long long key = K.hkeys[h];
        const int c = (int)(key >> 32);
        const int b = (int)(key & 0xffffffffu);
        const long long vcb = K.hvals[h];
        const long long vt = K.vtot[b];
        const long long vs = A.vsfx[b];
        long long contrib;
        if (vt == 0) contrib = (K.croot[c] == K.minc[b]) ? vs : 0;
        else if (vcb == vt) contrib = vs;
        else {
            const double r = (double)vcb / (double)vt;
            contrib = __double2ll_rn((double)vs * r);
        }
        atomicAdd((unsigned long long*)&K.nvsfx[c], (unsigned long long)contrib);
        if (A.constp[b]) K.nconstp[c] = 1;
    }
}

// Phase 6: the new rows replace the old; slots of marked bubbles that were
// not handed out again are emptied (they stay on the free stack); the hash
// positions taken are emptied; the marks are cleared.
__device__ inline void ccl_install_phase(const StepArgs& A, const CclArgs& K) {
    if (!K.initial && blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd((unsigned long long*)K.runs, 1ull);
        atomicAdd((unsigned long long*)K.runs + 1, (unsigned long long)*K.naff);
    }
    // the labels this pass set go back to -1 (the next pass scans boxes only)
    const int np = *K.np;
    FSL_LIST_LOOP(i, np) {
        if (i < np) K.lab[K.plist[i]] = -1;
    }
    const int nn = *K.nnew;
    FSL_LIST_LOOP(i, nn) {
        if (i >= nn) continue;
        const int sl = K.newslots[i];
        A.vfx[sl] = K.nvfx[sl];
        A.vxfx[sl] = K.nvxfx[sl];
        K.vsfx[sl] = K.initial ? K.nvfx[sl] + K.nvxfx[sl] : K.nvsfx[sl];
        A.ncells[sl] = K.nncells[sl];
        K.constp[sl] = K.nconstp[sl];
        K.aff[sl] = 0;
    }
    if (K.initial) return;
    const int na = *K.naff;
    FSL_LIST_LOOP(i, na) {
        if (i >= na) continue;
        const int b = K.afflist[i];
        if (K.aff[b] == 1) {   // not handed out again (a reused slot reads 2, or 0 once rewritten)
            A.vfx[b] = 0; A.vxfx[b] = 0; K.vsfx[b] = 0; A.ncells[b] = 0; K.constp[b] = 0;
            K.aff[b] = 0;
        }
    }
    const int nh = *K.nhused;
    FSL_LIST_LOOP(i, nh) {
        if (i >= nh) continue;
        K.hkeys[K.hused[i]] = ~0ull;
        K.hvals[K.hused[i]] = 0;
    }
    for (long long dd = (long long)blockIdx.x * blockDim.x + threadIdx.x; dd < A.ndom;
         dd += (long long)gridDim.x * blockDim.x)
        if (K.nfree[dd] < 0) K.nfree[dd] = 0;
}

// Barrier over all blocks of a cooperative launch (all of them resident).  The
// last block to arrive resets the count and advances the generation; the others
// wait for the generation to move, at most A.spins polls, after which they
// record ST_SYNC and report failure (the caller returns).  The arrival is an
// acquire-release atomic and the release of the generation and its polls are
// release / acquire at GPU scope, so every write before the barrier is
// visible to every read after it.
__device__ inline bool grid_barrier(const StepArgs& A) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned* count = A.bar;
        unsigned* gen = A.bar + 1;
        unsigned g0, old, gnow;
        ok = 1;
        asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(g0) : "l"(gen) : "memory");
        // arrive: release this block's writes (ordered before by the block
        // barrier), acquire those of the blocks that arrived before
        asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(count) : "memory");
        if (old == gridDim.x - 1 + (unsigned)A.bar_extra) {
            asm volatile("st.relaxed.gpu.u32 [%0], 0;" ::"l"(count) : "memory");
            asm volatile("red.release.gpu.add.u32 [%0], 1;" ::"l"(gen) : "memory");
        } else {
            int it = 0;
            do {
                asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(gnow) : "l"(gen) : "memory");
            } while (gnow == g0 && ++it < A.spins);
            if (gnow == g0) {
                set_status(A.status, ST_SYNC);
                ok = 0;
            }
        }
    }
    __syncthreads();
    return ok != 0;
}

// Conversion (Sec. 2.2) in one cooperative launch: phases A+B, C and D
// separated by grid barriers, then, when phase C set a merge / split trigger,
// the labelling of the triggered domains (Secs. 2.3.1, 2.3.2).
template <typename T>
__global__ void __launch_bounds__(FSL_CONV_THREADS, 3) k_convert(StepArgs A, CclArgs K) {
    pdl_wait();   // the stream-collide kernel has finished and its writes are visible
    if (blockIdx.x == 0) {
        for (int d = threadIdx.x; d < A.ndom; d += blockDim.x) A.icnt[d] = 0;
        if (threadIdx.x == 0) {
            *A.icount_next = 0;
            // list counters of this step's labelling (used after phase C at the earliest)
            *K.naff = 0; *K.np = 0; *K.nnew = 0; *K.nhused = 0;
        }
    }
    convert_ab_phase<T>(A);
    if (!grid_barrier(A)) return;
    convert_c_phase(A, K);
    if (!grid_barrier(A)) return;
    const bool relabel = *(volatile int*)A.trig != 0;   // final after phase C
    convert_d_phase(A);
    if (A.order) {
        if (!grid_barrier(A)) return;
        order_count_phase(A);
        if (!grid_barrier(A)) return;
        order_write_phase(A);
    }
    if (!relabel) return;
    if (!grid_barrier(A)) return;
    ccl_rows_phase(A, K);
    if (!grid_barrier(A)) return;
    ccl_init_phase(A, K);
    if (!grid_barrier(A)) return;
    ccl_hook_phase(A, K);
    if (!grid_barrier(A)) return;
    ccl_compress_phase(A, K);
    if (!grid_barrier(A)) return;
    ccl_pairs_phase(A, K);
    if (!grid_barrier(A)) return;
    ccl_table_phase(A, K);
    if (!grid_barrier(A)) return;
    ccl_install_phase(A, K);
}

// Initial state: validate the closed interface layer, f = f_eq(rho, u),
// m = phi rho on interface cells (Eq. 9).
template <typename T>
__global__ void __launch_bounds__(FSL_BLOCK) k_init_state(StepArgs A, int d, const uint8_t* flags_in,
                                                         const double* fill, const double* rho, const double* u) {
    using C = typename Form<T>::C;
    const Dom& D = get_dom(A, d);
    const long long l = (long long)blockIdx.x * FSL_BLOCK + threadIdx.x;
    if (l >= D.n) return;
    const long long g = D.off + l;
    const long long S = A.stride;
    const uint8_t t = flags_in[l];
    const Cell c = make_cell(D, g);
    if (t > LID) { set_status(A.status, -1); return; }
    bool wall = false;
    for (int a = 1; a < 19; ++a) {
        // neighbours are read from the input (the device flag array is being
        // written by other threads)
        const long long z = c.at(cx(a), cy(a), cz(a)) - D.off;
        if (t == LIQ && flags_in[z] == GAS) set_status(A.status, ST_GEOMETRY);
        if (flags_in[z] == OBS || flags_in[z] == LID) wall = true;
    }
    A.flag[g] = (uint8_t)(t | (wall ? K_WALL : 0));
    A.mark[g] = MK_NONE;
    A.id[g] = -1;
    A.exs[g] = 0.0;
    double ph = (t == LIQ) ? 1.0 : (t == IFC ? fill[l] : 0.0);
    A.phi[g] = ph;
    const double pht = (t == LIQ || t == OBS || t == LID) ? 1.0 : (t == GAS ? 0.0 : (ph < 0.0 ? 0.0 : (ph > 1.0 ? 1.0 : ph)));
    A.phit[g] = pht;
    if (A.phif) { A.phif[g] = (float)ph; A.phitf[g] = (float)pht; }
    T* f = (T*)A.fdst;
    if (t == LIQ || t == IFC) {
        C fe[19];
        feq_all<C>((C)rho[l], (C)u[l], (C)u[D.n + l], (C)u[2 * (long long)D.n + l], fe);
        for (int a = 0; a < 19; ++a) Form<T>::st(f + (long long)a * S + g, a, fe[a]);
        A.rhoi[g] = rho[l];
        A.m[g] = (t == IFC) ? fill[l] * rho[l] : rho[l];
    } else {
        for (int a = 0; a < 19; ++a) Form<T>::st(f + (long long)a * S + g, a, (C)weight(a));
        A.rhoi[g] = 0.0;
        A.m[g] = 0.0;
    }
}

// Export of the PDFs (unshifted, double) and of their density and velocity.
template <typename T>
__global__ void k_export_pdf(const T* f, long long S, long long off, int n, double* pdf, double* rho, double* u) {
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const long long g = off + l;
    double fo[19];
    for (int a = 0; a < 19; ++a) {
        fo[a] = (double)Form<T>::ld(f + (long long)a * S + g, a);
        if (pdf) pdf[(long long)a * n + l] = fo[a];
    }
    if (rho || u) {
        double r, jx, jy, jz;
        moments<double>(fo, r, jx, jy, jz);
        if (rho) rho[l] = r;
        if (u) {
            u[l] = r != 0.0 ? jx / r : 0.0;
            u[n + l] = r != 0.0 ? jy / r : 0.0;
            u[2LL * n + l] = r != 0.0 ? jz / r : 0.0;
        }
    }
}

// Liquid mass of one domain, deterministically: per block the sum, in a fixed
// tree order, of rho (sum of the stored PDFs, Eq. 4) over liquid cells and of m
// over interface cells; the host adds the block sums in block order.
template <typename T>
__global__ void __launch_bounds__(FSL_BLOCK) k_mass_partials(const T* f, const uint8_t* flag, const double* m,
                                                             long long S, long long off, int n, double* part) {
    const long long l = (long long)blockIdx.x * FSL_BLOCK + threadIdx.x;
    double v = 0.0;
    if (l < n) {
        const long long g = off + l;
        const uint8_t t = ctype(flag[g]);
        if (t == LIQ) {
            double r = (double)Form<T>::ld(f + g, 0);
            for (int a = 1; a < 19; ++a) r += (double)Form<T>::ld(f + (long long)a * S + g, a);
            v = r;
        } else if (t == IFC) {
            v = m[g];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __shared__ double ws[FSL_BLOCK / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < FSL_BLOCK / 32; ++w) t += ws[w];
        part[blockIdx.x] = t;
    }
}

// The normals pass ahead of the forms that take interface cells one per
// thread: by tiles when every domain is at least one tile in size (a batch
// through its tile table), else one thread per cell.
template <typename T>
inline void launch_normals(const StepArgs& A, long long nb, cudaStream_t s) {
    const Dom& D = A.d0;
    if (A.ndom == 1 && D.nx >= NT_X && D.ny >= NT_Y && D.nz >= NT_Z) {
        const unsigned nt = (unsigned)(((D.nx + NT_X - 1) / NT_X) * ((D.ny + NT_Y - 1) / NT_Y) *
                                       ((D.nz + NT_Z - 1) / NT_Z));
        k_normals_tiled<T, true><<<nt, NT_X * NT_Y, 0, s>>>(A);
    } else if (A.ndom > 1 && A.ntiles) {
        k_normals_tiled<T, false><<<(unsigned)A.nntiles, NT_X * NT_Y, 0, s>>>(A);
    } else if (A.ndom == 1) {
        k_normals<T, true><<<(unsigned)nb, FSL_BLOCK, 0, s>>>(A);
    } else {
        k_normals<T, false><<<(unsigned)nb, FSL_BLOCK, 0, s>>>(A);
    }
}

// Launch helpers instantiated once per storage form.
template <typename T> void launch_stream(const StepArgs& A, long long nblocks, int ifblocks, int form, int pgrid,
                                         cudaStream_t s, cudaEvent_t el, cudaEvent_t ei, cudaStream_t s2,
                                         cudaEvent_t efork, cudaEvent_t ejoin);
template <typename T> int stream_blocks_per_sm(int form, bool one);
template <typename T> cudaError_t launch_convert(const StepArgs& A, const CclArgs& K, int nblocks, cudaStream_t s,
                                                 bool pdl);
template <typename T> int convert_blocks_per_sm();
template <typename T> void launch_init_state(const StepArgs& A, int d, int n, const uint8_t* fl, const double* fill,
                                             const double* rho, const double* u, cudaStream_t s);
template <typename T> void launch_export_pdf(const void* f, long long S, long long off, int n, double* pdf,
                                             double* rho, double* u, cudaStream_t s);
template <typename T> void launch_mass_partials(const void* f, const uint8_t* flag, const double* m, long long S,
                                                long long off, int n, double* part, cudaStream_t s);

#define FSL_INSTANTIATE_FORM(T)                                                                              \
    template <> void launch_stream<T>(const StepArgs& A, long long nb, int ifb, int form, int pgrid,          \
                                      cudaStream_t s, cudaEvent_t el, cudaEvent_t ei, cudaStream_t s2,       \
                                      cudaEvent_t efork, cudaEvent_t ejoin) {                                \
        /* split form: interface blocks first, then one block per liquid tile; */                          \
        /* persistent forms: pgrid resident blocks; el / ei (optional) both */                              \
        /* mark the kernel's end */                                                                          \
        const unsigned pg = (unsigned)(pgrid > 0 ? pgrid : 1);                                               \
        if (form == SC_SPLIT) {                                                                              \
            const int nif = FSL_IF_GRID * ifb / 2;                                                           \
            const long long nliq = Form<T>::shifted ? (nb + 1) / 2 : nb;                                     \
            if (A.ndom == 1)                                                                                 \
                k_stream<T, true><<<(unsigned)(nif + nliq), FSL_BLOCK, 0, s>>>(A, nif);                      \
            else                                                                                             \
                k_stream<T, false><<<(unsigned)(nif + nliq), FSL_BLOCK, 0, s>>>(A, nif);                     \
        } else if (form == SC_TILE2 || form == SC_TILE4) {                                                  \
            const long long tile = Form<T>::shifted ? 2LL * FSL_BLOCK : (long long)FSL_BLOCK;                \
            const int tpb = form == SC_TILE2 ? 2 : 4;                                                       \
            const unsigned nsup = (unsigned)((A.stride + tpb * tile - 1) / (tpb * tile));                    \
            if (A.ndom == 1) {                                                                               \
                launch_normals<T>(A, nb, s);                                                                 \
                if (tpb == 2) k_stream_tile<T, true, 2><<<nsup, FSL_BLOCK, 0, s>>>(A);                       \
                else k_stream_tile<T, true, 4><<<nsup, FSL_BLOCK, 0, s>>>(A);                                \
            } else {                                                                                         \
                launch_normals<T>(A, nb, s);                                                                 \
                if (tpb == 2) k_stream_tile<T, false, 2><<<nsup, FSL_BLOCK, 0, s>>>(A);                      \
                else k_stream_tile<T, false, 4><<<nsup, FSL_BLOCK, 0, s>>>(A);                               \
            }                                                                                                \
        } else if (form == SC_TWOC) {                                                                        \
            /* the interface kernel on a second stream, beside the liquid kernel */                          \
            const long long nliq = Form<T>::shifted ? (nb + 1) / 2 : nb;                                     \
            launch_normals<T>(A, nb, s);                                                                     \
            cudaEventRecord(efork, s);                                                                       \
            cudaStreamWaitEvent(s2, efork, 0);                                                               \
            if (A.ndom == 1) k_iface<T, true><<<pg, IfThreads<T>::n, 0, s2>>>(A);                            \
            else k_iface<T, false><<<pg, IfThreads<T>::n, 0, s2>>>(A);                                       \
            cudaEventRecord(ejoin, s2);                                                                      \
            if (A.ndom == 1) k_liquid<T, true><<<(unsigned)nliq, FSL_BLOCK, 0, s>>>(A);                      \
            else k_liquid<T, false><<<(unsigned)nliq, FSL_BLOCK, 0, s>>>(A);                                 \
            cudaStreamWaitEvent(s, ejoin, 0);                                                                \
        } else if (form == SC_TWO) {                                                                         \
            const long long nliq = Form<T>::shifted ? (nb + 1) / 2 : nb;                                     \
            if (A.ndom == 1) {                                                                               \
                launch_normals<T>(A, nb, s);                                                                 \
                k_liquid<T, true><<<(unsigned)nliq, FSL_BLOCK, 0, s>>>(A);                                   \
                k_iface<T, true><<<pg, IfThreads<T>::n, 0, s>>>(A);                                          \
            } else {                                                                                         \
                launch_normals<T>(A, nb, s);                                                                 \
                k_liquid<T, false><<<(unsigned)nliq, FSL_BLOCK, 0, s>>>(A);                                  \
                k_iface<T, false><<<pg, IfThreads<T>::n, 0, s>>>(A);                                         \
            }                                                                                                \
        } else if (form == SC_SLAB) {                                                                        \
            if (A.ndom == 1) k_stream_slab<T, true><<<pg, FSL_BLOCK, 0, s>>>(A);                             \
            else k_stream_slab<T, false><<<pg, FSL_BLOCK, 0, s>>>(A);                                        \
        } else if (A.ndom == 1) {                                                                            \
            if (form == SC_PERS1) k_stream_pers<T, true, 1><<<pg, FSL_BLOCK, 0, s>>>(A);                    \
            else if (form == SC_PERS2) k_stream_pers<T, true, 2><<<pg, FSL_BLOCK, 0, s>>>(A);               \
            else k_stream_pers<T, true, 4><<<pg, FSL_BLOCK, 0, s>>>(A);                                      \
        } else {                                                                                             \
            if (form == SC_PERS1) k_stream_pers<T, false, 1><<<pg, FSL_BLOCK, 0, s>>>(A);                   \
            else if (form == SC_PERS2) k_stream_pers<T, false, 2><<<pg, FSL_BLOCK, 0, s>>>(A);              \
            else k_stream_pers<T, false, 4><<<pg, FSL_BLOCK, 0, s>>>(A);                                     \
        }                                                                                                    \
        if (ei) cudaEventRecord(ei, s);                                                                      \
        if (el) cudaEventRecord(el, s);                                                                      \
    }                                                                                                        \
    template <> int stream_blocks_per_sm<T>(int form, bool one) {                                            \
        int nb = 0;                                                                                          \
        if (form == SC_SPLIT) nb = 1;                                                                        \
        else if (form == SC_TILE2 || form == SC_TILE4) {                                                     \
            if (one) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream_tile<T, true, 2>, FSL_BLOCK, 0); \
            else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream_tile<T, false, 2>, FSL_BLOCK, 0); \
        }                                                                                                    \
        else if (form == SC_TWOC && one)                                                                     \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_iface<T, true>, IfThreads<T>::n, 0);        \
        else if (form == SC_TWOC)                                                                            \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_iface<T, false>, IfThreads<T>::n, 0);       \
        else if (form == SC_TWO && one)                                                                      \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_iface<T, true>, IfThreads<T>::n, 0);        \
        else if (form == SC_TWO)                                                                             \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_iface<T, false>, IfThreads<T>::n, 0);       \
        else if (form == SC_SLAB && one)                                                                     \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream_slab<T, true>, FSL_BLOCK, 0);        \
        else if (form == SC_SLAB)                                                                            \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream_slab<T, false>, FSL_BLOCK, 0);       \
        else if (one && form == SC_PERS1)                                                                    \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream_pers<T, true, 1>, FSL_BLOCK, 0);     \
        else if (one && form == SC_PERS2)                                                                    \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream_pers<T, true, 2>, FSL_BLOCK, 0);     \
        else if (one)                                                                                        \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream_pers<T, true, 4>, FSL_BLOCK, 0);     \
        else if (form == SC_PERS1)                                                                           \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream_pers<T, false, 1>, FSL_BLOCK, 0);    \
        else if (form == SC_PERS2)                                                                           \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream_pers<T, false, 2>, FSL_BLOCK, 0);    \
        else                                                                                                 \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream_pers<T, false, 4>, FSL_BLOCK, 0);    \
        return nb;                                                                                           \
    }                                                                                                        \
    template <> cudaError_t launch_convert<T>(const StepArgs& A, const CclArgs& K, int nb, cudaStream_t s,  \
                                              bool pdl) {                                                    \
        cudaLaunchConfig_t cfg = {};                                                                         \
        cfg.gridDim = dim3((unsigned)nb);                                                                    \
        cfg.blockDim = dim3(FSL_CONV_THREADS);                                                               \
        cfg.stream = s;                                                                                      \
        cudaLaunchAttribute at[2];                                                                           \
        at[0].id = cudaLaunchAttributeCooperative;                                                           \
        at[0].val.cooperative = 1;                                                                           \
        at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;                                       \
        at[1].val.programmaticStreamSerializationAllowed = 1;                                                \
        cfg.attrs = at;                                                                                      \
        cfg.numAttrs = pdl ? 2 : 1;   /* after a join of two streams: a plain dependency */               \
        return cudaLaunchKernelEx(&cfg, k_convert<T>, A, K);                                                 \
    }                                                                                                        \
    template <> int convert_blocks_per_sm<T>() {                                                             \
        int nb = 0;                                                                                          \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_convert<T>, FSL_CONV_THREADS, 0);               \
        return nb;                                                                                           \
    }                                                                                                        \
    template <> void launch_init_state<T>(const StepArgs& A, int d, int n, const uint8_t* fl,                \
                                          const double* fill, const double* rho, const double* u,            \
                                          cudaStream_t s) {                                                  \
        k_init_state<T><<<(unsigned)((n + FSL_BLOCK - 1) / FSL_BLOCK), FSL_BLOCK, 0, s>>>(A, d, fl, fill,   \
                                                                                          rho, u);           \
    }                                                                                                        \
    template <> void launch_mass_partials<T>(const void* f, const uint8_t* flag, const double* m,            \
                                             long long S, long long off, int n, double* part,               \
                                             cudaStream_t s) {                                              \
        k_mass_partials<T><<<(unsigned)((n + FSL_BLOCK - 1) / FSL_BLOCK), FSL_BLOCK, 0, s>>>(                 \
            (const T*)f, flag, m, S, off, n, part);                                                          \
    }                                                                                                        \
    template <> void launch_export_pdf<T>(const void* f, long long S, long long off, int n, double* pdf,     \
                                          double* rho, double* u, cudaStream_t s) {                          \
        k_export_pdf<T><<<(unsigned)((n + 127) / 128), 128, 0, s>>>((const T*)f, S, off, n, pdf, rho, u);   \
    }

}  // namespace fsl
