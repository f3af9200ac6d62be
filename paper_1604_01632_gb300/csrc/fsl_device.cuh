// fsl_device.cuh -- device-side definitions of the GB300 FSLBM library:
// lattice constants, cell/mark codes, per-domain descriptors, PDF storage
// forms and the templated per-cell kernels (stream-collide and the second
// conversion phase) that exist once per storage precision.
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
#include <stdint.h>

#define FSL_BLOCK 256

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
enum { ST_GEOMETRY = -2, ST_NAN = -4, ST_CCL = -5, ST_TABLE_FULL = -6 };

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
    int* ilist_next;            // interface cells after this step's conversion (C4)
    int* icount_next;
    int* mlist;                 // interface cells marked filled / emptied (K1I)
    int* mcount;
    int* glist;                 // gas cells that become interface (phase A)
    int* gcount;
    int* llist;                 // liquid cells that become interface (phase B)
    int* lcount;
    int* cstep;                 // step number at which each cell was last converted
    int* recv;                  // step number at which each cell last received excess mass
    int* stepno;                // device step counter
    long long* icnt;            // per-domain interface count at the end of the step
    unsigned long long cond;    // graph conditional handle set to the trigger (0: none)
    Dom d0;                     // domain 0, read from the parameter space when ndom == 1
};

// Domain descriptor and domain of a cell: a handle with one domain reads
// them from the kernel parameters, a batch from its device tables.
__device__ inline Dom get_dom(const StepArgs& A, int d) { return A.ndom == 1 ? A.d0 : A.doms[d]; }
__device__ inline int block_dom(const StepArgs& A, long long g) { return A.ndom == 1 ? 0 : A.blk_dom[g / FSL_BLOCK]; }

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
    __device__ static inline void st_dev(__half* p, float v) { *p = __float2half_rn(v); }
    __device__ static inline float ld(const __half* p, int a) { return weightc<float>(a) + __half2float(*p); }
    __device__ static inline void st(__half* p, int a, float v) { *p = __float2half_rn(v - weightc<float>(a)); }
};
template <> struct Form<__nv_bfloat16> {
    using C = float;
    static constexpr bool shifted = true;
    __device__ static inline float ld_dev(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    __device__ static inline void st_dev(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
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

// K1L: stream with half-way bounce-back (Eq. 7) and collide (Eq. 6) for
// liquid cells.  Only cells flagged as touching a wall read the types of
// their neighbours; a liquid cell never touches gas (closed interface layer).
template <typename T>
__global__ void __launch_bounds__(FSL_BLOCK, 5) k_stream_liquid(StepArgs A) {
    using C = typename Form<T>::C;
    const long long g = (long long)blockIdx.x * FSL_BLOCK + threadIdx.x;
    const uint8_t f = A.flag[g];
    if (ctype(f) != LIQ) return;
    const Dom D = get_dom(A, block_dom(A, g));
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
#pragma unroll
            for (int a = 1; a < 19; ++a) {
                const int ab = opp(a);
                const unsigned y = (unsigned)(gi + P.ox[1 - cx(a)] + P.oy[1 - cy(a)] + P.oz[1 - cz(a)]);
                const uint8_t ty = ctype(A.flag[y]);
                if (ty == OBS) {
                    d[a] = Form<T>::ld_dev(src + ab * S + gi);   // w_a = w_abar
                } else if (ty == LID) {
                    const float cuw = cdot<float>(a, R.lid[0], R.lid[1], R.lid[2]);
                    d[a] = Form<T>::ld_dev(src + ab * S + gi) + (6.f * weightc<float>(a)) * cuw;
                } else {
                    d[a] = Form<T>::ld_dev(src + a * S + y);
                }
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
#pragma unroll
            for (int a = 1; a < 19; ++a) {
                const int ab = opp(a);
                const unsigned y = (unsigned)(gi + P.ox[1 - cx(a)] + P.oy[1 - cy(a)] + P.oz[1 - cz(a)]);
                const uint8_t ty = ctype(A.flag[y]);
                if (ty == OBS) {
                    fin[a] = Form<T>::ld(src + ab * S + gi, ab);
                } else if (ty == LID) {
                    C cuw = cdot<C>(a, R.lid[0], R.lid[1], R.lid[2]);
                    fin[a] = Form<T>::ld(src + ab * S + gi, ab) + ((C)6 * weightc<C>(a)) * cuw;
                } else {
                    fin[a] = Form<T>::ld(src + a * S + y, a);
                }
            }
        }
        C fout[19];
        C rho = collide_any<C>(D.has_force, fin, fout, R.omp, R.omm, R.g[0], R.g[1], R.g[2]);
        if (!(rho == rho)) set_status(A.status, ST_NAN);
#pragma unroll
        for (int a = 0; a < 19; ++a) Form<T>::st(dst + a * S + gi, a, fout[a]);
    }
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

struct Stencil {
    int x, y, z, nx, ny, nz;
    long long off, g;
    bool inner;   // two cells from every face: no wrap needed
    __device__ inline long long at(int dx, int dy, int dz) const {
        if (inner) return g + dx + (long long)nx * (dy + (long long)ny * dz);
        return off + wrap2(x + dx, nx) + (long long)nx * (wrap2(y + dy, ny) + (long long)ny * wrap2(z + dz, nz));
    }
};

__device__ inline Stencil make_stencil(const Dom& D, long long g) {
    Stencil s;
    local_xyz(D, (int)(g - D.off), s.x, s.y, s.z);
    s.nx = D.nx; s.ny = D.ny; s.nz = D.nz;
    s.off = D.off;
    s.g = g;
    s.inner = s.x >= 2 && s.x < D.nx - 2 && s.y >= 2 && s.y < D.ny - 2 && s.z >= 2 && s.z < D.nz - 2;
    return s;
}


// K1I: interface cells, from the list of interface cells built at the end of
// the previous step.  A block of 128 threads takes FSL_IFC cells per pass.
// Load phase, four threads per cell: the 5x5x5 box of fill levels around the
// cell (rows along x), and for the directions q, q+4, ... the cell's PDFs, the
// PDF streaming in, the neighbour types and the mass-exchange terms.
// Gradient phase, four threads per cell: Parker-Youngs gradients at the cell
// and at its six face neighbours (unit normals there).  Compute phase, one
// thread per cell, in the oracle's order: stream with bounce-back (Eq. 7),
// mass exchange over the 18 links (Eq. 10), reconstruction of the PDFs coming
// from the gas side with the gas density 3 (p_V + 2 sigma kappa) of the
// cell's bubble (Eqs. 8, 11-15, kappa = 1/2 div n_hat by central differences
// of the face normals), collision (Eq. 6), then the filled / emptied marks.
// The FP32-collide forms do all of this in FP32 except the cell mass, which
// accumulates in FP64.
#define FSL_IF_THREADS 128
template <typename T> struct IfCells {
    static constexpr int n = sizeof(typename Form<T>::C) == 8 ? 16 : 32;
};
template <typename T>
struct IfStage {
    using C = typename Form<T>::C;
    static constexpr int N = IfCells<T>::n;
    C ph[N][125];      // fill levels, 5x5x5 box around the cell
    C fs[N][19];       // own post-collision PDFs of the previous step
    C fy[N][19];       // PDF streaming in from the source cell
    C ex[N][19];       // mass-exchange term of each link (Eq. 10)
    C nrm[N][7][3];    // gradient at the cell, unit normals at the face neighbours
    C pv[N];           // bubble pressure (Eq. 13)
    double m[N];       // mass
    uint8_t ty[N][19];
    uint8_t tz[N][19];
};

__device__ inline int ph_index(int dx, int dy, int dz) { return (dx + 2) + 5 * (dy + 2) + 25 * (dz + 2); }

template <typename T>
__global__ void __launch_bounds__(FSL_IF_THREADS) k_stream_interface(StepArgs A) {
    using C = typename Form<T>::C;
    constexpr int N = IfCells<T>::n;
    constexpr int TPC = FSL_IF_THREADS / N;   // threads per cell in the load and gradient phases
    __shared__ IfStage<T> sh;
    if (blockIdx.x == 0) {
        // per-step counters; the previous step's kernels are done with them
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
    const int cnt = *A.icount;
    const long long S = A.stride;
    const T* __restrict__ src = (const T*)A.fsrc;
    T* __restrict__ dst = (T*)A.fdst;
    // fill levels in the arithmetic type (FP32 copies for the FP32-collide forms)
    const C* __restrict__ phic;
    const C* __restrict__ phtc;
    if constexpr (sizeof(C) == 8) { phic = A.phi; phtc = A.phit; }
    else { phic = A.phif; phtc = A.phitf; }
    const int c = threadIdx.x / TPC;      // cell of this thread in the load and gradient phases
    const int q = threadIdx.x % TPC;
    for (int i0 = blockIdx.x * N; i0 < cnt; i0 += gridDim.x * N) {
        // ---------------- load phase
        if (i0 + c < cnt) {
            const long long g = A.ilist[i0 + c];
            const Dom D = get_dom(A, block_dom(A, g));
            const Stencil st = make_stencil(D, g);
            // rows (dy, dz) of the box, five cells along x each
            for (int r = q; r < 25; r += TPC) {
                const int dy = r % 5 - 2, dz = r / 5 - 2;
                C* row = &sh.ph[c][5 * r];
                if (st.x >= 2 && st.x < st.nx - 2) {
                    const long long b = st.at(0, dy, dz);
#pragma unroll
                    for (int k = 0; k < 5; ++k) row[k] = phtc[b + (k - 2)];
                } else {
#pragma unroll
                    for (int k = 0; k < 5; ++k) row[k] = phtc[st.at(k - 2, dy, dz)];
                }
            }
            if (q == TPC - 1) {
                sh.m[c] = A.m[g];
                const int bub = A.id[g];
                if constexpr (sizeof(C) == 8)
                    sh.pv[c] = bub >= 0 ? bubble_pressure(A.vfx[bub], A.vxfx[bub], A.vsfx[bub], A.constp[bub]) : 1.0 / 3.0;
                else
                    sh.pv[c] = bub >= 0 ? bubble_pressure_f(A.vfx[bub], A.vxfx[bub], A.vsfx[bub], A.constp[bub])
                                        : (float)(1.0 / 3.0);
            }
            const C phx = phic[g];
            for (int a = q; a < 19; a += TPC) {
                const C fsa = Form<T>::ld(src + (long long)a * S + g, a);
                sh.fs[c][a] = fsa;
                if (a == 0) continue;
                const int ab = opp(a);
                const int ax = rcx(a), ay = rcy(a), az = rcz(a);
                const long long y = st.at(-ax, -ay, -az);
                sh.ty[c][a] = ctype(A.flag[y]);
                sh.fy[c][a] = Form<T>::ld(src + (long long)a * S + y, a);
                const long long z = st.at(ax, ay, az);
                const uint8_t tz = ctype(A.flag[z]);
                sh.tz[c][a] = tz;
                if (tz == LIQ || tz == IFC) {
                    const C e = Form<T>::ld(src + (long long)ab * S + z, ab) - fsa;
                    sh.ex[c][a] = tz == IFC ? ((C)0.5 * (phx + phic[z])) * e : e;
                }
            }
        }
        __syncthreads();
        // ---------------- gradient phase: point j (the cell, then its +x, -x,
        // +y, -y, +z, -z neighbours) for j = q, q + TPC, ...
        if (i0 + c < cnt) {
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
        // ---------------- compute phase, one thread per cell
        if (threadIdx.x < 32) {
            const int cc = threadIdx.x;
            uint8_t mk = MK_NONE;
            long long g = 0;
            if (cc < N && i0 + cc < cnt) {
                g = A.ilist[i0 + cc];
                const Dom D = get_dom(A, block_dom(A, g));
                const Par<C> R = par_of<C>(D);
                C fs[19];
#pragma unroll
                for (int a = 0; a < 19; ++a) fs[a] = sh.fs[cc][a];
                C rs, jsx, jsy, jsz;
                moments<C>(fs, rs, jsx, jsy, jsz);
                const C ugx = jsx / rs, ugy = jsy / rs, ugz = jsz / rs;
                const C dX = sh.nrm[cc][1][0] - sh.nrm[cc][2][0];
                const C dY = sh.nrm[cc][3][1] - sh.nrm[cc][4][1];
                const C dZ = sh.nrm[cc][5][2] - sh.nrm[cc][6][2];
                const C kappa = (C)0.25 * ((dX + dY) + dZ);
                const C gx = sh.nrm[cc][0][0], gy = sh.nrm[cc][0][1], gz = sh.nrm[cc][0][2];
                const C pg = sh.pv[cc] + R.sigma2 * kappa;
                const C rg = (C)3 * pg;
                C fg[19];
                feq_all<C>(rg, ugx, ugy, ugz, fg);
                C fin[19];
                fin[0] = fs[0];
#pragma unroll
                for (int a = 1; a < 19; ++a) {
                    const int ab = opp(a);
                    const uint8_t ty = sh.ty[cc][a];
                    if (ty == OBS) {
                        fin[a] = fs[ab];
                    } else if (ty == LID) {
                        const C cuw = cdot<C>(a, R.lid[0], R.lid[1], R.lid[2]);
                        fin[a] = fs[ab] + ((C)6 * weightc<C>(a)) * cuw;
                    } else if (ty == GAS) {
                        fin[a] = (fg[a] + fg[ab]) - fs[ab];
                    } else {
                        fin[a] = sh.fy[cc][a];
                        if (D.normal_rule && cdot<C>(a, gx, gy, gz) > (C)0) fin[a] = (fg[a] + fg[ab]) - fs[ab];
                    }
                }
                // mass exchange, summed in direction order (Eq. 10); the cell
                // mass itself accumulates in FP64 for every form
                C dm = (C)0;
                bool has_gas = false, has_liq = false;
#pragma unroll
                for (int a = 1; a < 19; ++a) {
                    const uint8_t tz = sh.tz[cc][a];
                    if (tz == LIQ || tz == IFC) dm = dm + sh.ex[cc][a];
                    has_gas |= tz == GAS;
                    has_liq |= tz == LIQ;
                }
                const double mnew = sh.m[cc] + (double)dm;
                C fout[19];
                const C rho = collide_any<C>(D.has_force, fin, fout, R.omp, R.omm, R.g[0], R.g[1], R.g[2]);
                if (!(rho == rho)) set_status(A.status, ST_NAN);
#pragma unroll
                for (int a = 0; a < 19; ++a) Form<T>::st(dst + (long long)a * S + g, a, fout[a]);
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
            list_append(A.mlist, A.mcount, mk != MK_NONE, (int)g);
        }
        __syncthreads();
    }
}

// First neighbour of cell z (direction order) that is an interface cell
// carrying mark `want`, or -1.
__device__ inline long long first_marked(const StepArgs& A, const Dom& D, long long z, uint8_t want) {
    const Cell c = make_cell(D, z);
    for (int a = 1; a < 19; ++a) {
        const long long w = c.at(cx(a), cy(a), cz(a));
        if (ctype(A.flag[w]) == IFC && A.mark[w] == want) return w;
    }
    return -1;
}

// An interface cell carrying an emptied mark that phase A does not cancel (no
// filled neighbour).  Written as a test on the marks K1I set, so it holds
// whether or not another thread has already cleared the cancelled mark.
__device__ inline bool still_emptied(const StepArgs& A, const Dom& D, long long w) {
    if (ctype(A.flag[w]) != IFC || A.mark[w] != MK_EMPTIED) return false;
    const Cell c = make_cell(D, w);
    for (int a = 1; a < 19; ++a) {
        const long long v = c.at(cx(a), cy(a), cz(a));
        if (ctype(A.flag[v]) == IFC && A.mark[v] == MK_FILLED) return false;
    }
    return true;
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
__global__ void __launch_bounds__(128) k_convert_ab(StepArgs A) {
    using C = typename Form<T>::C;
    if (blockIdx.x == 0) {
        for (int d = threadIdx.x; d < A.ndom; d += blockDim.x) A.icnt[d] = 0;
        if (threadIdx.x == 0) *A.icount_next = 0;
    }
    pdl_trigger();
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
            const Dom D = get_dom(A, d);
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
                        C sr = (C)0, sux = (C)0, suy = (C)0, suz = (C)0;
                        int cnt = 0;
                        for (int q = 1; q < 19; ++q) {
                            const long long w = cz_.at(cx(q), cy(q), cz(q));
                            const uint8_t tw = ctype(A.flag[w]);
                            if (tw == LIQ || (tw == IFC && !still_emptied(A, D, w))) {
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
                for (int q = 1; q < 19 && first < 0; ++q) {
                    const long long w = cz_.at(cx(q), cy(q), cz(q));
                    if (still_emptied(A, D, w)) first = w;
                }
                if (first == p) {
                    lclaim = true;
                    double r = (double)Form<T>::ld(f + z, 0);
                    for (int q = 1; q < 19; ++q) r = r + (double)Form<T>::ld(f + (long long)q * S + z, q);
                    A.mark[z] = MK_NEWL;
                    A.id[z] = A.id[p];
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

// Initial state: validate the closed interface layer, f = f_eq(rho, u),
// m = phi rho on interface cells (Eq. 9).
template <typename T>
__global__ void __launch_bounds__(FSL_BLOCK) k_init_state(StepArgs A, int d, const uint8_t* flags_in,
                                                         const double* fill, const double* rho, const double* u) {
    using C = typename Form<T>::C;
    const Dom D = get_dom(A, d);
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

// Launch helpers instantiated once per storage form.
template <typename T> void launch_stream(const StepArgs& A, long long nblocks, int ifblocks, cudaStream_t s,
                                         cudaStream_t s2, cudaEvent_t fork, cudaEvent_t join, cudaEvent_t el,
                                         cudaEvent_t ei);
template <typename T> void launch_convert_ab(const StepArgs& A, long long nblocks, cudaStream_t s);
template <typename T> void launch_init_state(const StepArgs& A, int d, int n, const uint8_t* fl, const double* fill,
                                             const double* rho, const double* u, cudaStream_t s);
template <typename T> void launch_export_pdf(const void* f, long long S, long long off, int n, double* pdf,
                                             double* rho, double* u, cudaStream_t s);

#define FSL_INSTANTIATE_FORM(T)                                                                              \
    template <> void launch_stream<T>(const StepArgs& A, long long nb, int ifb, cudaStream_t s,               \
                                      cudaStream_t s2, cudaEvent_t fork, cudaEvent_t join, cudaEvent_t el,   \
                                      cudaEvent_t ei) {                                                      \
        /* liquid cells on s, interface cells on s2 at the same time (disjoint outputs); */                 \
        /* el / ei (optional) mark the end of each kernel */                                                \
        cudaEventRecord(fork, s);                                                                            \
        cudaStreamWaitEvent(s2, fork, 0);                                                                    \
        k_stream_interface<T><<<(unsigned)(2 * ifb), FSL_IF_THREADS, 0, s2>>>(A);                           \
        if (ei) cudaEventRecord(ei, s2);                                                                     \
        k_stream_liquid<T><<<(unsigned)nb, FSL_BLOCK, 0, s>>>(A);                                           \
        if (el) cudaEventRecord(el, s);                                                                      \
        cudaEventRecord(join, s2);                                                                           \
        cudaStreamWaitEvent(s, join, 0);                                                                     \
    }                                                                                                        \
    template <> void launch_convert_ab<T>(const StepArgs& A, long long nb, cudaStream_t s) {                 \
        k_convert_ab<T><<<(unsigned)nb, 128, 0, s>>>(A);                                                    \
    }                                                                                                        \
    template <> void launch_init_state<T>(const StepArgs& A, int d, int n, const uint8_t* fl,                \
                                          const double* fill, const double* rho, const double* u,            \
                                          cudaStream_t s) {                                                  \
        k_init_state<T><<<(unsigned)((n + FSL_BLOCK - 1) / FSL_BLOCK), FSL_BLOCK, 0, s>>>(A, d, fl, fill,   \
                                                                                          rho, u);           \
    }                                                                                                        \
    template <> void launch_export_pdf<T>(const void* f, long long S, long long off, int n, double* pdf,     \
                                          double* rho, double* u, cudaStream_t s) {                          \
        k_export_pdf<T><<<(unsigned)((n + 127) / 128), 128, 0, s>>>((const T*)f, S, off, n, pdf, rho, u);   \
    }

}  // namespace fsl
