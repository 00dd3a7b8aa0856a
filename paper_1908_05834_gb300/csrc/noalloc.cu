// bchar_mass_noalloc: the porous mass sum_K |K|_phi c_K of the update stage,
// for callers that must not allocate device memory.
//
// Some callers cannot allocate at the point where they need this value: a
// time-stepping loop that owns a fixed device-memory budget (an allocation
// could fail or evict), a framework that hands out memory only from its own
// pool, or code that must not trigger the implicit device synchronisation
// of cudaMalloc/cudaFree in the middle of a step.  This entry point needs no
// buffer from them beyond the inputs and the output: the per-block partial
// sums live in a fixed array in the library's own device memory.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it until the process exits.  Host code only knows a host-side
// stand-in for it, so its device address is looked up once per device with
// cudaGetSymbolAddress (on the first call made on that device, with that
// device current) and passed to the kernels.
#include <mutex>

#include "device.cuh"

namespace bchar {

constexpr int kNoAllocBlocks = 1024;    // partial sums held in the scratch array
constexpr int kNoAllocPerThread = 64;   // elements per thread of one block
constexpr int64_t kNoAllocMaxN = static_cast<int64_t>(kNoAllocBlocks) * kThreads * kNoAllocPerThread;  // 2^24

// Scratch shared by every call (the last call's partials stay in it).
static __device__ __align__(256) double g_noalloc_partials[kNoAllocBlocks];

// Block b sums volphi_i c_i over its contiguous chunk, in a fixed order.
template <class T>
__global__ void k_mass_partials(int64_t n, const double *volphi, const T *c, double *partials) {
    const int64_t chunk = static_cast<int64_t>(kThreads) * kNoAllocPerThread;
    const int64_t base = blockIdx.x * chunk;
    double s = 0.0;
    for (int k = 0; k < kNoAllocPerThread; ++k) {
        const int64_t i = base + static_cast<int64_t>(k) * kThreads + threadIdx.x;
        if (i < n) s += volphi[i] * static_cast<double>(c[i]);
    }
    s = block_sum(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_mass_total(const double *partials, int nblocks, double *out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) s += partials[i];
    s = block_sum(s);
    if (threadIdx.x == 0) *out = s;
}

// Device address of the scratch array, looked up once per device.
static bchar_status scratch_address(double **out) {
    static std::mutex lock;
    static double *addr[256] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return BCHAR_ERR_CUDA;
    }
    std::lock_guard<std::mutex> guard(lock);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) {
            cudaGetLastError();
            return BCHAR_ERR_CUDA;
        }
        addr[dev] = static_cast<double *>(p);
    }
    *out = addr[dev];
    return BCHAR_OK;
}

}  // namespace bchar

using namespace bchar;

extern "C" bchar_status bchar_mass_noalloc(const double *volphi, const void *c, int c_dtype, int64_t n,
                                           double *mass_out, void *stream) {
    if (!volphi || !c || !mass_out || n < 1 || (c_dtype != BCHAR_C_F64 && c_dtype != BCHAR_C_F32))
        return BCHAR_ERR_INVALID_ARG;
    if (n > kNoAllocMaxN) return BCHAR_ERR_CAPACITY;
    double *partials = nullptr;
    bchar_status st = scratch_address(&partials);
    if (st != BCHAR_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t chunk = static_cast<int64_t>(kThreads) * kNoAllocPerThread;
    const int nblocks = static_cast<int>((n + chunk - 1) / chunk);
    if (c_dtype == BCHAR_C_F32)
        k_mass_partials<float><<<nblocks, kThreads, 0, s>>>(n, volphi, static_cast<const float *>(c), partials);
    else
        k_mass_partials<double><<<nblocks, kThreads, 0, s>>>(n, volphi, static_cast<const double *>(c), partials);
    k_mass_total<<<1, 1024, 0, s>>>(partials, nblocks, mass_out);
    if (cudaGetLastError() != cudaSuccess) return BCHAR_ERR_CUDA;
    return BCHAR_OK;
}
