// fsl_internal.h -- declarations shared by the translation units of the
// library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fsl {

struct StepArgs;
struct Dom;

// Scratch of the connected-component labelling and bubble-table rebuild.
struct CclArgs {
    int* lab;                    // union-find parent per cell (global index), -1 background
    int* aux;                    // new slot of each root cell
    unsigned long long* hkeys;   // (new slot << 32 | old slot) overlap keys, ~0 empty
    long long* hvals;            // overlap volumes V_{c,b}, fixed point
    long long hcap;              // power of two
    long long* nvfx;             // new table (slot-indexed)
    long long* nvxfx;
    long long* nvsfx;
    long long* nncells;
    int* nconstp;
    int* croot;                  // root cell (global index) of each new slot
    long long* vtot;             // per old slot: total volume over all new components
    int* minc;                   // per old slot: lowest root among its components
    int* nslot;                  // per domain: slots in use
    const int* slot_dom;         // slot -> domain
    long long nslots_total;
    long long* runs;             // labelling passes run after initialisation
    int initial;                 // 1: first labelling after initialisation (V* = V)
    int max_iter;                // cap on union / find loops
};

void launch_convert_c(const StepArgs& A, long long nb, cudaStream_t s);
void launch_convert_d(const StepArgs& A, long long nb, cudaStream_t s);
void launch_build_ilist(const StepArgs& A, long long nb, cudaStream_t s);
int launch_ccl(const StepArgs& A, const CclArgs& K, long long nb, long long* vsfx, int* constp, cudaStream_t s);
void launch_export_minid(const int* id, long long off, int n, int* minidx, cudaStream_t s);
void launch_export_cells(const uint8_t* flag, const double* phi, const double* m, const int* id, const int* minidx,
                         long long off, int n, uint8_t* oflag, double* ophi, double* om, long long* oid,
                         long long* counts, cudaStream_t s);
cudaError_t upload_tables();

}  // namespace fsl
