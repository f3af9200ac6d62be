// fsl_internal.h -- declarations shared by the translation units of the
// library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fsl_device.cuh"

namespace fsl {

void launch_build_ilist(const StepArgs& A, long long nb, cudaStream_t s);
int launch_ccl(const StepArgs& A, const CclArgs& K, long long nb, cudaStream_t s);
void launch_export_minid(const int* id, long long off, int n, int* minidx, cudaStream_t s);
void launch_export_cells(const uint8_t* flag, const double* phi, const float* phif, const double* m, const int* id,
                         const int* minidx,
                         long long off, int n, uint8_t* oflag, double* ophi, double* om, long long* oid,
                         long long* counts, cudaStream_t s);

}  // namespace fsl
