// fsl_core.cu -- precision-independent step kernels of the GB300 FSLBM
// library (connected-component labelling of the bubbles; bubble-table
// rebuild; exports) and the FP64 instantiation of the per-precision kernels.  Compiled without FMA contraction (-fmad=false) so
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

FSL_INSTANTIATE_FORM(double)

// Interface list and per-domain interface counts of the initial state.
__global__ void __launch_bounds__(FSL_BLOCK) k_build_ilist(StepArgs A) {
    const long long g = (long long)blockIdx.x * FSL_BLOCK + threadIdx.x;
    const int d = block_dom(A, (long long)blockIdx.x * FSL_BLOCK);
    const bool itf = ctype(A.flag[g]) == IFC;
    warp_add(A.icnt, itf ? d : -1, 1);
    list_append(A.ilist, A.icount, itf, (int)g);
}

// --------------------------------------------- connected-component labelling

// The labelling phases of the initial pass (every bubble), one kernel each.
__global__ void __launch_bounds__(FSL_BLOCK) k_ccl_init(StepArgs A, CclArgs K) { ccl_init_phase(A, K); }
__global__ void __launch_bounds__(FSL_BLOCK) k_ccl_hook(StepArgs A, CclArgs K) { ccl_hook_phase(A, K); }
__global__ void __launch_bounds__(FSL_BLOCK) k_ccl_compress(StepArgs A, CclArgs K) { ccl_compress_phase(A, K); }
__global__ void __launch_bounds__(FSL_BLOCK) k_ccl_pairs(StepArgs A, CclArgs K) { ccl_pairs_phase(A, K); }
__global__ void __launch_bounds__(FSL_BLOCK) k_ccl_install(StepArgs A, CclArgs K) { ccl_install_phase(A, K); }

// ------------------------------------------------------------------ exports

// Lowest cell index of every bubble slot (its canonical id).  The lanes of a
// warp hold consecutive cells, so among the lanes with the same slot the
// lowest lane has the lowest index: one atomic per slot and warp.
__global__ void k_export_minid(const int* id, long long off, int n, int* minidx) {
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = l < n ? id[off + l] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    if (b >= 0 && (int)(threadIdx.x & 31u) == __ffs(peers) - 1) atomicMin(&minidx[b], (int)l);
}

// Cell export; phif (the FP32-collide forms' fill level, null in FP64) takes the
// place of phi where given.
__global__ void k_export_cells(const uint8_t* flag, const double* phi, const float* phif, const double* m, const int* id,
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
    if (ophi) ophi[l] = phif ? (double)phif[g] : phi[g];
    if (om) om[l] = m[g];
    if (oid) {
        const int b = id[g];
        oid[l] = b >= 0 ? (long long)minidx[b] : -1;
    }
}

// ------------------------------------------------------------ host launches

void launch_build_ilist(const StepArgs& A, long long nb, cudaStream_t s) { k_build_ilist<<<(unsigned)nb, FSL_BLOCK, 0, s>>>(A); }

// Initial labelling (K.initial = 1): the list phases run over a grid of one
// thread per cell, which covers the participant list whatever its length.
int launch_ccl(const StepArgs& A, const CclArgs& K, long long nb, cudaStream_t s) {
    k_ccl_init<<<(unsigned)nb, FSL_BLOCK, 0, s>>>(A, K);
    k_ccl_hook<<<(unsigned)nb, FSL_BLOCK, 0, s>>>(A, K);
    k_ccl_compress<<<(unsigned)nb, FSL_BLOCK, 0, s>>>(A, K);
    k_ccl_pairs<<<(unsigned)nb, FSL_BLOCK, 0, s>>>(A, K);
    k_ccl_install<<<(unsigned)nb, FSL_BLOCK, 0, s>>>(A, K);
    return 5;
}

void launch_export_minid(const int* id, long long off, int n, int* minidx, cudaStream_t s) {
    k_export_minid<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(id, off, n, minidx);
}

void launch_export_cells(const uint8_t* flag, const double* phi, const float* phif, const double* m, const int* id,
                         const int* minidx, long long off, int n, uint8_t* oflag, double* ophi, double* om,
                         long long* oid, long long* counts, cudaStream_t s) {
    k_export_cells<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(flag, phi, phif, m, id, minidx, off, n, oflag, ophi,
                                                              om, oid, counts);
}

}  // namespace fsl
