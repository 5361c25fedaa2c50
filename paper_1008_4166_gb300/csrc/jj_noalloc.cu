// Pivot Gram by fp16 digit products on the tensor cores, for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside a host
// callback or a driver hook where allocation calls are forbidden, code that
// must not touch an allocator that is already being used in another thread,
// or a strict real-time loop that promised never to allocate after start-up.
// jjk_gram allocates its scratch (the int128 accumulators and the column
// exponents) from the stream-ordered allocator; jjk_gram_noalloc takes the
// same scratch from one fixed array in device memory that is part of the
// library image instead.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it (kNoAllocBytes, about 8.3 MiB) until the process exits.
// Host code cannot use the variable's name as a device address (on the host it
// names a shadow object), so the address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and cached.
#include <mutex>

#include "jj_common.cuh"

namespace jj {
namespace {

constexpr size_t kNoAllocAccBytes = size_t(8) << 20;  // int128 Gram accumulators
constexpr int64_t kNoAllocMaxCols = 65536;            // column exponents (int32)
constexpr size_t kNoAllocBytes = kNoAllocAccBytes + kNoAllocMaxCols * sizeof(int32_t);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices];

// Device address of the scratch array on the current device (looked up once).
cudaError_t noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace jj

using namespace jj;

extern "C" int jjk_gram_noalloc(int32_t dtype, const void *G, int64_t ld, int64_t m,
                                const int32_t *pairs, int32_t npairs, double *A, int32_t kmax,
                                int64_t ncols, void *stream) {
    if ((dtype != JJ_F64 && dtype != JJ_C128) || !G || !pairs || !A || ld < m || m < 1 ||
        kmax < 1 || npairs < 0 || ncols < 1)
        return JJ_INVALID_ARG;
    const bool cplx = dtype == JJ_C128;
    if (!ozaki_supported(cplx, kmax)) return JJ_INVALID_ARG;
    if (ozaki_gram_workspace_bytes(npairs, kmax, cplx) > kNoAllocAccBytes ||
        ncols > kNoAllocMaxCols)
        return JJ_INVALID_ARG;
    if (npairs == 0) return JJ_OK;
    void *base = nullptr;
    if (noalloc_scratch(&base) != cudaSuccess) return JJ_CUDA_ERROR;
    unsigned long long *acc = static_cast<unsigned long long *>(base);
    int32_t *cexp = reinterpret_cast<int32_t *>(static_cast<unsigned char *>(base) + kNoAllocAccBytes);
    cudaStream_t st = (cudaStream_t)stream;
    // launch_gram_ozaki clears the accumulators before use (the array keeps the
    // previous call's contents).
    if (launch_colexp(cplx, (const double *)G, ld, m, ncols, cexp, st) != cudaSuccess)
        return JJ_CUDA_ERROR;
    if (launch_gram_ozaki(cplx, (const double *)G, ld, m, ncols, pairs, npairs, A, kmax, 0, cexp, acc,
                          ozaki_default_slices(true), nullptr, st) != cudaSuccess)
        return JJ_CUDA_ERROR;
    return JJ_OK;
}
