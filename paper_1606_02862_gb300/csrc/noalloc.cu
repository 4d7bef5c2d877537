// noalloc.cu -- FP64 field-energy reduction that allocates no device memory.
//
// pic_diagnostics sums the field energy through the context's scratch
// buffers.  This entry point computes the same quantity,
//   W = sum over cells of (E^2 + B^2) / 2 * cell_volume,
// from device arrays the caller owns, and keeps its per-block partial sums
// in the file-scope array g_partials below instead of allocating them.  It
// serves callers that cannot call cudaMalloc when they need the number:
// hosts that give a library only memory they reserved up front, and code
// running where the host's rules forbid a device allocation at that point.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Each call writes every partial it later reads, so nothing has to
// start at zero, but calls whose work overlaps on the GPU (two streams, or
// two host threads) race on it: order them on one stream.  Its device
// address is looked up once per device and kept for the life of the process;
// a device reset (cudaDeviceReset) makes that address stale and is not
// supported between calls.
#include "pic.h"

#include <cuda_runtime.h>
#include <mutex>

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 32;                    // values per thread
constexpr int kMaxBlocks = 16384;                 // partials in g_partials (128 KB)
constexpr int64_t kSpan = (int64_t)kThreads * kPerThread;   // values per block
// E and B hold 3 values per cell each; one partial per kSpan values
constexpr int64_t kMaxCells = (int64_t)kMaxBlocks * kSpan / 3;  // 44,739,242 cells
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_partials[kMaxBlocks];

// Host-side device addresses of g_partials, one per device (the symbol name
// in host code is only a stand-in, not a device address).
double* g_partials_addr[kMaxDevices] = {};
std::mutex g_setup_mutex;

__global__ void __launch_bounds__(kThreads) k_energy_partials(const double* __restrict__ E,
                                                               const double* __restrict__ B,
                                                               int64_t n3, double* partials)
{
    // block b sums the contiguous range [b * kSpan, (b + 1) * kSpan)
    const int64_t lo = (int64_t)blockIdx.x * kSpan;
    double acc = 0.0;
    for (int k = 0; k < kPerThread; ++k) {
        const int64_t i = lo + (int64_t)k * kThreads + threadIdx.x;
        if (i < n3) {
            const double e = E[i], b = B[i];
            acc += e * e + b * b;
        }
    }
    __shared__ double s[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0)
        s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w)
            t += s[w];
        partials[blockIdx.x] = t;  // every partial the final pass reads is written here
    }
}

__global__ void __launch_bounds__(1024) k_energy_final(const double* partials, int nblk, double half_vol,
                                                       double* out)
{
    __shared__ double s[32];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
        acc += partials[b];
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0)
        s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w)
            t += s[w];
        *out = t * half_vol;
    }
}

// Device address of g_partials on the current device, looked up once.
pic_status partials_address(double** addr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PIC_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices)
        return PIC_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) {
            cudaGetLastError();
            return PIC_ERR_CUDA;
        }
        g_partials_addr[dev] = static_cast<double*>(p);
    }
    *addr = g_partials_addr[dev];
    return PIC_OK;
}

}  // namespace

extern "C" pic_status pic_field_energy_noalloc(const double* E, const double* B, int64_t ncells,
                                               double cell_volume, double* out, void* stream)
{
    if (!E || !B || !out || ncells < 0 || !(cell_volume > 0.0))
        return PIC_ERR_ARG;
    if (ncells > kMaxCells)
        return PIC_ERR_ARG;  // more cells than g_partials has partial sums for
    double* partials = nullptr;
    pic_status st = partials_address(&partials);
    if (st != PIC_OK)
        return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n3 = 3 * ncells;
    const int nblk = (int)((n3 + kSpan - 1) / kSpan);  // <= kMaxBlocks for ncells <= kMaxCells
    // each launch is judged by its own return code: an error that earlier,
    // unrelated calls left pending is neither reported here nor cleared
    if (nblk > 0) {
        void* args[] = {(void*)&E, (void*)&B, (void*)&n3, (void*)&partials};
        if (cudaLaunchKernel((const void*)k_energy_partials, dim3(nblk), dim3(kThreads), args, 0, s) !=
            cudaSuccess)
            return PIC_ERR_CUDA;
    }
    const double half_vol = 0.5 * cell_volume;
    void* fargs[] = {(void*)&partials, (void*)&nblk, (void*)&half_vol, (void*)&out};
    if (cudaLaunchKernel((const void*)k_energy_final, dim3(1), dim3(1024), fargs, 0, s) != cudaSuccess)
        return PIC_ERR_CUDA;
    return PIC_OK;
}
