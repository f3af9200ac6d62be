// fsl_core.cu -- precision-independent step kernels of the GB300 FSLBM
// library (conversion phases A, C, D; connected-component labelling of the
// bubbles; bubble-table rebuild; exports) and the FP64 instantiation of the
// per-precision kernels.  Compiled without FMA contraction (-fmad=false) so
// that every FP64 operation rounds where it is written, as in the oracle.
//
// Method: Anderl et al., arXiv:1604.01632, Sec. 2.2 (cell conversion, closed
// interface layer), Sec. 2.3 (bubble volume per step, Eq. 13), Sec. 2.3.1
// (merge: V* and V add), Sec. 2.3.2 (split: flood-fill colouring, daughters
// keep the old pressure).  The paper's serial flood fill and its colour
// unification across processes (Sec. 2.4.1) become one lock-free union-find
// over the whole GPU lattice whose roots are the minimum cell index of each
// component.
#include <cuda_runtime.h>
#include <limits.h>

#include "fsl_device.cuh"
#include "fsl_internal.h"

namespace fsl {

// 3x3x3 cube around a cell, bit k = (dx+1) + 3 (dy+1) + 9 (dz+1); bit 13 is the
// centre.  c_adj18[k] = cells of the cube that are face or edge neighbours of
// cell k (built on the host at load time).
__constant__ unsigned c_adj18[27];
__constant__ unsigned c_mask18;   // the 18 face/edge neighbours of the centre

FSL_INSTANTIATE_FORM(double)

// Sum v over the warp into base[key] with one atomic when every lane has the
// same key; key < 0 contributes nothing.  Every lane of the warp must call.
__device__ inline void warp_add(long long* base, int key, long long v) {
    const unsigned full = 0xffffffffu;
    const int k0 = __shfl_sync(full, key, 0);
    if (__all_sync(full, key == k0)) {
        if (k0 < 0) return;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(full, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0) atomicAdd((unsigned long long*)&base[k0], (unsigned long long)v);
    } else if (key >= 0 && v != 0) {
        atomicAdd((unsigned long long*)&base[key], (unsigned long long)v);
    }
}

// ------------------------------------------------------ conversion phases
// All four phases work on compact lists (marked cells, new interface cells,
// interface cells), so their cost follows the interface, not the lattice.

// Local test that removing the filled cell at the centre of the cube cannot
// split its bubble: the gas/interface cells among its 18 neighbours must stay
// connected inside the cube (18-connectivity) without the centre.
__device__ inline bool removal_is_local(unsigned fg) {
    const unsigned targets = fg & c_mask18;
    if (targets == 0) return true;
    unsigned reach = targets & (~targets + 1u);   // lowest target
    for (int it = 0; it < 27; ++it) {
        unsigned grow = reach;
        unsigned r = reach;
        while (r) {
            const int k = __ffs(r) - 1;
            r &= r - 1;
            grow |= c_adj18[k];
        }
        grow &= fg;
        if (grow == reach) break;
        reach = grow;
    }
    return (targets & ~reach) == 0;
}

// C3, over the marked list and the new-from-liquid list: excess mass of
// converted cells (filled: m - rho, emptied: m) split equally among the
// neighbours that are interface after conversion, else pooled; merge / split
// triggers.  Taking the filled cells away one at a time in index order, each
// removal must pass the local test with the lower-index filled cells already
// gone and the higher-index ones still present, or the labelling runs.
__global__ void __launch_bounds__(128) k_convert_c(StepArgs A) {
    pdl_wait();
    pdl_trigger();
    const int nm = *A.mcount, nl = *A.lcount;
    const int total = nm + nl;
    const int step = *A.stepno;
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const long long g = i < nm ? A.mlist[i] : A.llist[i - nm];
        const int d = block_dom(A, g);
        const Dom D = get_dom(A, d);
        const Cell c = make_cell(D, g);
        const uint8_t mk = A.mark[g];
        if (i < nm) {
            if (mk != MK_FILLED && mk != MK_EMPTIED) continue;   // emptied mark cancelled in phase A
            const double mex = (mk == MK_FILLED) ? A.m[g] - A.rhoi[g] : A.m[g];
            int k = 0;
            for (int a = 1; a < 19; ++a) {
                const long long z = c.at(cx(a), cy(a), cz(a));
                if (new_type(ctype(A.flag[z]), A.mark[z]) == IFC) {
                    ++k;
                    A.recv[z] = step;   // z pulls a share in the update phase
                }
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
                if (!removal_is_local(fgm)) {
                    atomicExch(&A.trig[1 + d], 1);
                    atomicExch(A.trig, 1);
                }
            }
            A.cstep[g] = step;
            A.mark[g] = (mk == MK_FILLED) ? MK_CFILLED : MK_CEMPTIED;
            atomicAdd((unsigned long long*)&A.nif[d], (unsigned long long)-1LL);
            continue;
        }
        // new interface cell from liquid: a neighbour of another bubble merges
        const int b = A.id[g];
        for (int a = 1; a < 19; ++a) {
            const long long z = c.at(cx(a), cy(a), cz(a));
            const uint8_t ntz = new_type(ctype(A.flag[z]), A.mark[z]);
            if ((ntz == GAS || ntz == IFC) && A.id[z] != b) {
                atomicExch(&A.trig[1 + d], 1);
                atomicExch(A.trig, 1);
                break;
            }
        }
    }
}

// C4, over the interface list and the two new-interface lists: receivers pull
// the excess shares of converted neighbours in direction order and the pool
// share, phi = m / rho (Eq. 9); converted cells take their new type; bubble
// volumes change by exact fixed-point differences; the interface list of the
// next step; reservoir drain; the graph condition of the labelling.
__global__ void __launch_bounds__(128) k_convert_d(StepArgs A) {
    pdl_wait();
    const int ni = *A.icount, ng = *A.gcount, nl = *A.lcount;
    const int total = ni + ng + nl;
    const int step = *A.stepno;
    const int stride = gridDim.x * blockDim.x;
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
            const double m0 = A.m[g], rh = A.rhoi[g], ph0 = A.phi[g];
            const int rs = A.recv[g];
            const long long nI = A.nif[d];
            const long long pool = A.pool[d];
            const uint8_t t = ctype(f);
            if (t == IFC && mk == MK_CFILLED) {
                dv = -volume_term(IFC, ph0);
                ckey = key;
                dc = -1;
                A.flag[g] = (uint8_t)((f & ~K_TYPE) | LIQ);
                A.phi[g] = 1.0;
                A.phit[g] = 1.0;
                if (A.phif) { A.phif[g] = 1.f; A.phitf[g] = 1.f; }
                A.id[g] = -1;
                A.mark[g] = MK_NONE;
            } else if (t == IFC && mk == MK_CEMPTIED) {
                dv = FSL_VOL_ONE - volume_term(IFC, ph0);
                A.flag[g] = (uint8_t)((f & ~K_TYPE) | GAS);
                A.phi[g] = 0.0;
                A.phit[g] = 0.0;
                if (A.phif) { A.phif[g] = 0.f; A.phitf[g] = 0.f; }
                A.m[g] = 0.0;
                A.mark[g] = MK_NONE;
            } else {
                double s = m0;
                if (rs == step) {
                    // a converted neighbour listed this cell among its receivers
                    const Dom D = get_dom(A, d);
                    const Cell c = make_cell(D, g);
                    for (int a = 1; a < 19; ++a) {
                        const long long z = c.at(cx(a), cy(a), cz(a));
                        if (A.cstep[z] == step) s = s + A.exs[z];
                    }
                }
                if (nI > 0) {
                    const double share = ((double)pool * 9.094947017729282379150390625e-13) / (double)nI;
                    s = s + share;
                }
                const double phn = s / rh;
                const long long told = volume_term(t, ph0);
                A.m[g] = s;
                A.phi[g] = phn;
                const double pht = phn < 0.0 ? 0.0 : (phn > 1.0 ? 1.0 : phn);
                A.phit[g] = pht;
                if (A.phif) { A.phif[g] = (float)phn; A.phitf[g] = (float)pht; }
                if (t != IFC) A.flag[g] = (uint8_t)((f & ~K_TYPE) | IFC);
                dv = volume_term(IFC, phn) - told;
                if (t == LIQ) { ckey = key; dc = 1; }
                keep = true;
            }
        }
        warp_add(A.vfx, dv != 0 ? key : -1, dv);
        warp_add(A.ncells, ckey, dc);
        warp_add(A.icnt, keep ? d : -1, 1);
        list_append(A.ilist_next, A.icount_next, keep, (int)g);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // reservoir drain of every domain whose seed cell is still gas or
        // interface (types read through the marks, which stay consistent
        // while other threads update the flags)
        for (int d = 0; d < A.ndom; ++d) {
            const Dom D = get_dom(A, d);
            if (D.seed < 0) continue;
            const long long gs = D.off + D.seed;
            const uint8_t nt = new_type(ctype(A.flag[gs]), A.mark[gs]);
            const int b = A.id[gs];
            if ((nt == GAS || nt == IFC) && b >= 0)
                atomicAdd((unsigned long long*)&A.vxfx[b], (unsigned long long)(-D.rate_fx));
        }
        *A.mcount = 0;
        if (A.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)A.cond, *A.trig ? 1u : 0u);
    }
}

// Interface list and per-domain interface counts of the initial state.
__global__ void __launch_bounds__(FSL_BLOCK) k_build_ilist(StepArgs A) {
    const long long g = (long long)blockIdx.x * FSL_BLOCK + threadIdx.x;
    const int d = block_dom(A, (long long)blockIdx.x * FSL_BLOCK);
    const bool itf = ctype(A.flag[g]) == IFC;
    warp_add(A.icnt, itf ? d : -1, 1);
    list_append(A.ilist, A.icount, itf, (int)g);
}

// --------------------------------------------- connected-component labelling

__device__ inline bool is_fg(uint8_t f) { return ctype(f) == GAS || ctype(f) == IFC; }

// Root of a; halves the path on the way (each cell is pointed at its
// grandparent, still one of its ancestors, so the trees keep their roots).
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

// Lock-free union: always hook the larger root under the smaller one, so the
// final root of every component is its minimum cell index.
__device__ inline bool unite(int* L, int a, int b, int cap) {
    bool ok = true;
    for (int it = 0; it < cap && ok; ++it) {
        a = find_root(L, a, cap, ok);
        b = find_root(L, b, cap, ok);
        if (!ok) return false;
        if (a == b) return true;
        if (a < b) { const int tt = a; a = b; b = tt; }
        const int old = atomicMin(&L[a], b);
        if (old == a) return true;
        a = old;
    }
    return false;
}

// Domain of a block taking part in this labelling pass (every domain after
// initialisation, else the domains whose step set the trigger).
__device__ inline bool ccl_active(const StepArgs& A, const CclArgs& K, int d) {
    return K.initial || A.trig[1 + d] != 0;
}

__global__ void __launch_bounds__(FSL_BLOCK) k_ccl_init(StepArgs A, CclArgs K) {
    if (!K.initial && *A.trig == 0) return;
    const long long g = (long long)blockIdx.x * FSL_BLOCK + threadIdx.x;
    if (ccl_active(A, K, block_dom(A, g))) K.lab[g] = is_fg(A.flag[g]) ? (int)g : -1;
    const long long nth = (long long)gridDim.x * FSL_BLOCK;
    for (long long h = g; h < K.hcap; h += nth) {
        K.hkeys[h] = ~0ull;
        K.hvals[h] = 0;
    }
    for (long long s = g; s < K.nslots_total; s += nth) {
        K.nvfx[s] = 0; K.nvxfx[s] = 0; K.nvsfx[s] = 0; K.nncells[s] = 0; K.nconstp[s] = 0;
        K.croot[s] = -1;
        K.vtot[s] = 0;
        K.minc[s] = INT_MAX;
    }
    for (long long dd = g; dd < A.ndom; dd += nth)
        if (ccl_active(A, K, (int)dd)) K.nslot[dd] = 0;
}

__global__ void __launch_bounds__(FSL_BLOCK) k_ccl_hook(StepArgs A, CclArgs K) {
    if (!K.initial && *A.trig == 0) return;
    const long long g = (long long)blockIdx.x * FSL_BLOCK + threadIdx.x;
    if (!ccl_active(A, K, block_dom(A, g)) || !is_fg(A.flag[g])) return;
    const Dom D = get_dom(A, block_dom(A, (long long)blockIdx.x * FSL_BLOCK));
    const Cell c = make_cell(D, g);
    // the nine directions 1, 3, ..., 17 cover each neighbour pair once
    for (int a = 1; a < 19; a += 2) {
        const long long h = c.at(cx(a), cy(a), cz(a));
        if (is_fg(A.flag[h])) {
            if (!unite(K.lab, (int)g, (int)h, K.max_iter)) {
                set_status(A.status, ST_CCL);
                return;
            }
        }
    }
}

// Compress every cell onto its root; roots take a new bubble-table slot.
__global__ void __launch_bounds__(FSL_BLOCK) k_ccl_compress(StepArgs A, CclArgs K) {
    if (!K.initial && *A.trig == 0) return;
    const long long g = (long long)blockIdx.x * FSL_BLOCK + threadIdx.x;
    if (!ccl_active(A, K, block_dom(A, g)) || !is_fg(A.flag[g])) return;
    bool ok = true;
    const int r = find_root(K.lab, (int)g, K.max_iter, ok);
    if (!ok) { set_status(A.status, ST_CCL); return; }
    K.lab[g] = r;
    if (r == (int)g) {
        const int d = block_dom(A, (long long)blockIdx.x * FSL_BLOCK);
        const Dom D = get_dom(A, d);
        const int k = atomicAdd(&K.nslot[d], 1);
        if (k >= D.slot_cap) { set_status(A.status, ST_TABLE_FULL); K.aux[g] = -1; return; }
        K.aux[g] = D.slot_off + k;
        K.croot[D.slot_off + k] = r;
    }
}

__device__ inline void hash_add(const CclArgs& K, unsigned long long key, long long v, int* status) {
    unsigned long long h = key * 0x9E3779B97F4A7C15ull;
    long long pos = (long long)(h >> 20) & (K.hcap - 1);
    for (long long probe = 0; probe < K.hcap; ++probe) {
        const unsigned long long prev = atomicCAS(&K.hkeys[pos], ~0ull, key);
        if (prev == ~0ull || prev == key) {
            atomicAdd((unsigned long long*)&K.hvals[pos], (unsigned long long)v);
            return;
        }
        pos = (pos + 1) & (K.hcap - 1);
    }
    set_status(status, ST_TABLE_FULL);
}

// New volumes and cell counts per component, overlap volumes V_{c,b} of new
// component c with old bubble b, new ids.
__global__ void __launch_bounds__(FSL_BLOCK) k_ccl_pairs(StepArgs A, CclArgs K) {
    if (!K.initial && *A.trig == 0) return;
    const long long g = (long long)blockIdx.x * FSL_BLOCK + threadIdx.x;
    if (!ccl_active(A, K, block_dom(A, g))) return;   // whole block: one domain
    const uint8_t t = ctype(A.flag[g]);
    int c = -1;
    long long term = 0;
    if (t == GAS || t == IFC) {
        const int r = K.lab[g];
        c = K.aux[r];
        term = volume_term(t, A.phi[g]);
    }
    warp_add(K.nvfx, c, term);
    warp_add(K.nncells, c, c >= 0 ? 1 : 0);
    if (c < 0) return;
    if (!K.initial && A.id[g] >= 0) {
        const int b = A.id[g];
        const unsigned long long key = ((unsigned long long)(unsigned)c << 32) | (unsigned)b;
        hash_add(K, key, term, A.status);
        atomicAdd((unsigned long long*)&K.vtot[b], (unsigned long long)term);
        atomicMin(&K.minc[b], K.lab[g]);
        const Dom D = get_dom(A, block_dom(A, (long long)blockIdx.x * FSL_BLOCK));
        if (D.seed >= 0 && g - D.off == D.seed) {
            const long long x = A.vxfx[b];
            hash_add(K, key, x, A.status);
            atomicAdd((unsigned long long*)&K.vtot[b], (unsigned long long)x);
            K.nvxfx[c] = x;
        }
    }
    A.id[g] = c;
}

// V*_c = sum over b of V*_b V_{c,b} / V_b, V*_b copied when c holds all of b
// (Secs. 2.3.1, 2.3.2); a component touching a constant-pressure bubble
// stays constant-pressure.
__global__ void k_ccl_table(StepArgs A, CclArgs K) {
    if (K.initial || *A.trig == 0) return;
    const long long nth = (long long)gridDim.x * blockDim.x;
    for (long long h = (long long)blockIdx.x * blockDim.x + threadIdx.x; h < K.hcap; h += nth) {
        const unsigned long long key = K.hkeys[h];
        if (key == ~0ull) continue;
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

__global__ void k_ccl_install(StepArgs A, CclArgs K, long long* vsfx, int* constp) {
    if (!K.initial && *A.trig == 0) return;
    if (!K.initial && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd((unsigned long long*)K.runs, 1ull);
    const long long nth = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < K.nslots_total; s += nth) {
        const int d = K.slot_dom[s];
        if (!ccl_active(A, K, d)) continue;   // untouched domains keep their table
        const Dom D = get_dom(A, d);
        const int k = (int)(s - D.slot_off);
        if (k < K.nslot[d]) {
            A.vfx[s] = K.nvfx[s];
            A.vxfx[s] = K.nvxfx[s];
            vsfx[s] = K.initial ? K.nvfx[s] + K.nvxfx[s] : K.nvsfx[s];
            A.ncells[s] = K.nncells[s];
            constp[s] = K.nconstp[s];
        } else {
            A.vfx[s] = 0; A.vxfx[s] = 0; vsfx[s] = 0; A.ncells[s] = 0; constp[s] = 0;
        }
    }
}

// ------------------------------------------------------------------ exports

__global__ void k_export_minid(const int* id, long long off, int n, int* minidx) {
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int b = id[off + l];
    if (b >= 0) atomicMin(&minidx[b], (int)l);
}

__global__ void k_export_cells(const uint8_t* flag, const double* phi, const double* m, const int* id,
                               const int* minidx, long long off, int n, uint8_t* oflag, double* ophi, double* om,
                               long long* oid, long long* counts) {
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (counts) {
        const int t = l < n ? (int)ctype(flag[off + l]) : -1;
        for (int k = 0; k < 5; ++k) {
            const unsigned m5 = __ballot_sync(0xffffffffu, t == k);
            if ((threadIdx.x & 31) == 0 && m5) atomicAdd((unsigned long long*)&counts[k], (unsigned long long)__popc(m5));
        }
        return;
    }
    if (l >= n) return;
    const long long g = off + l;
    if (oflag) oflag[l] = ctype(flag[g]);
    if (ophi) ophi[l] = phi[g];
    if (om) om[l] = m[g];
    if (oid) {
        const int b = id[g];
        oid[l] = b >= 0 ? (long long)minidx[b] : -1;
    }
}

// ------------------------------------------------------------ host launches

void launch_convert_c(const StepArgs& A, long long nb, cudaStream_t s) { launch_pdl(k_convert_c, (unsigned)nb, 128u, s, A); }
void launch_convert_d(const StepArgs& A, long long nb, cudaStream_t s) { launch_pdl(k_convert_d, (unsigned)nb, 128u, s, A); }
void launch_build_ilist(const StepArgs& A, long long nb, cudaStream_t s) { k_build_ilist<<<(unsigned)nb, FSL_BLOCK, 0, s>>>(A); }

int launch_ccl(const StepArgs& A, const CclArgs& K, long long nb, long long* vsfx, int* constp, cudaStream_t s) {
    k_ccl_init<<<(unsigned)nb, FSL_BLOCK, 0, s>>>(A, K);
    k_ccl_hook<<<(unsigned)nb, FSL_BLOCK, 0, s>>>(A, K);
    k_ccl_compress<<<(unsigned)nb, FSL_BLOCK, 0, s>>>(A, K);
    k_ccl_pairs<<<(unsigned)nb, FSL_BLOCK, 0, s>>>(A, K);
    const unsigned tb = (unsigned)((K.hcap + 255) / 256);
    k_ccl_table<<<tb > 0 ? tb : 1, 256, 0, s>>>(A, K);
    const unsigned ib = (unsigned)((K.nslots_total + 255) / 256);
    k_ccl_install<<<ib > 0 ? ib : 1, 256, 0, s>>>(A, K, vsfx, constp);
    return 6;
}

void launch_export_minid(const int* id, long long off, int n, int* minidx, cudaStream_t s) {
    k_export_minid<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(id, off, n, minidx);
}

void launch_export_cells(const uint8_t* flag, const double* phi, const double* m, const int* id, const int* minidx,
                         long long off, int n, uint8_t* oflag, double* ophi, double* om, long long* oid,
                         long long* counts, cudaStream_t s) {
    k_export_cells<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(flag, phi, m, id, minidx, off, n, oflag, ophi, om,
                                                              oid, counts);
}

cudaError_t upload_tables() {
    unsigned adj[27];
    unsigned m18 = 0;
    for (int k = 0; k < 27; ++k) {
        const int kx = k % 3 - 1, ky = (k / 3) % 3 - 1, kz = k / 9 - 1;
        const int dk = (kx != 0) + (ky != 0) + (kz != 0);
        if (dk >= 1 && dk <= 2) m18 |= 1u << k;
        unsigned a = 0;
        for (int j = 0; j < 27; ++j) {
            const int jx = j % 3 - 1, jy = (j / 3) % 3 - 1, jz = j / 9 - 1;
            const int ax = jx - kx, ay = jy - ky, az = jz - kz;
            const int dist = (ax != 0) + (ay != 0) + (az != 0);
            if (ax < -1 || ax > 1 || ay < -1 || ay > 1 || az < -1 || az > 1) continue;
            if (dist >= 1 && dist <= 2) a |= 1u << j;
        }
        adj[k] = a & ~(1u << 13);   // never walk through the removed centre
    }
    cudaError_t e = cudaMemcpyToSymbol(c_adj18, adj, sizeof(adj));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_mask18, &m18, sizeof(m18));
}

}  // namespace fsl
