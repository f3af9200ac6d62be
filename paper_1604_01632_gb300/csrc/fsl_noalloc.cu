// fsl_noalloc.cu -- bubble labelling for callers that cannot allocate device
// memory.
//
// Some callers cannot call cudaMalloc: latency-critical loops in which an
// allocation may synchronise the device, deployments that hand all device
// memory to their own pool up front, and host frameworks that own the device
// memory budget and forbid libraries to allocate behind their back.
// fsl_label_bubbles_static gives them the library's
// bubble labelling (connected components of gas + interface cells under the
// 18-neighbourhood, label = minimum linear index, the same labels that
// fsl_fields(FSL_F_ID) reports after fsl_init_geometry) using only the
// caller's input and output buffers plus a fixed scratch array compiled into
// the library.
//
// The scratch is a file-scope static __device__ array of FSL_STATIC_MAX_CELLS
// int32 labels (8 MiB); every GPU that loads the library holds it until the
// process exits.  In host code the array's name is only a host-side stand-in,
// not a device address, so its device address is looked up once per device
// with cudaGetSymbolAddress (with that device current) and cached.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "../../include/fsl.h"

#define FSL_STATIC_MAX_CELLS (1 << 21)
#define FSL_STATIC_MAX_DEVICES 64

namespace {

static __device__ __align__(256) int g_label_scratch[FSL_STATIC_MAX_CELLS];

// device address of the scratch per device ordinal, looked up once per device
// (under the mutex; later calls read the atomic slot without locking)
std::atomic<void*> g_scratch_ptr[FSL_STATIC_MAX_DEVICES];
std::mutex g_scratch_mutex;

__host__ __device__ inline bool is_bubble_cell(uint8_t f) {
    const uint8_t t = (uint8_t)(f & 7);
    return t == FSL_GAS || t == FSL_INTERFACE;
}

__device__ inline int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__global__ void k_static_init(const uint8_t* flags, int n, int* lab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) lab[i] = is_bubble_cell(flags[i]) ? i : -1;   // every call starts from scratch
}

__device__ inline int static_root(const int* L, int a) {
    // labels only decrease along a chain, so this walk ends within a steps
    for (int it = 0; it < FSL_STATIC_MAX_CELLS; ++it) {
        const int p = L[a];
        if (p == a) return a;
        a = p;
    }
    return a;
}

__global__ void k_static_hook(const uint8_t* flags, int nx, int ny, int nz, int* lab) {
    const int n = nx * ny * nz;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !is_bubble_cell(flags[i])) return;
    const int x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
    // one direction of each of the nine neighbour pairs of the 18-neighbourhood
    const int d[9][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, -1, 0},
                         {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1}};
    for (int k = 0; k < 9; ++k) {
        const int j = wrap1(x + d[k][0], nx) + nx * (wrap1(y + d[k][1], ny) + ny * wrap1(z + d[k][2], nz));
        if (!is_bubble_cell(flags[j])) continue;
        int a = i, b = j;
        // union: hook the larger root under the smaller; a retry follows a link
        // another thread made, so the loop ends
        for (int it = 0; it < FSL_STATIC_MAX_CELLS; ++it) {
            a = static_root(lab, a);
            b = static_root(lab, b);
            if (a == b) break;
            if (a < b) { const int t = a; a = b; b = t; }
            const int old = atomicMin(&lab[a], b);
            if (old == a) break;
            a = old;
        }
    }
}

__global__ void k_static_out(const uint8_t* flags, int n, const int* lab, int64_t* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = is_bubble_cell(flags[i]) ? (int64_t)static_root(lab, i) : -1;
}

}  // namespace

extern "C" fsl_status fsl_label_bubbles_static(const uint8_t* flags, int32_t nx, int32_t ny, int32_t nz,
                                               int64_t* labels, void* cuda_stream) {
    if (!flags || !labels || nx <= 0 || ny <= 0 || nz <= 0) return FSL_ERR_ARG;
    const long long n = (long long)nx * ny * nz;
    if (n > FSL_STATIC_MAX_CELLS) return FSL_ERR_ARG;   // larger lattices need fsl_create
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= FSL_STATIC_MAX_DEVICES) return FSL_ERR_CUDA;
    void* lab_ptr = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!lab_ptr) {
        // first call on this device: look up the device address of the scratch
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        lab_ptr = g_scratch_ptr[dev].load(std::memory_order_relaxed);
        if (!lab_ptr) {
            if (cudaGetSymbolAddress(&lab_ptr, g_label_scratch) != cudaSuccess || !lab_ptr) return FSL_ERR_CUDA;
            g_scratch_ptr[dev].store(lab_ptr, std::memory_order_release);
        }
    }
    int* lab = (int*)lab_ptr;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nb = (int)((n + 255) / 256);
    k_static_init<<<nb, 256, 0, s>>>(flags, (int)n, lab);
    k_static_hook<<<nb, 256, 0, s>>>(flags, nx, ny, nz, lab);
    k_static_out<<<nb, 256, 0, s>>>(flags, (int)n, lab, labels);
    return cudaGetLastError() == cudaSuccess ? FSL_OK : FSL_ERR_CUDA;
}
