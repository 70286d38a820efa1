// Allocation-free compensated sum: the variant of the library's reduction
// kernels for callers that cannot allocate device memory.
//
// Who needs it: code embedded in a host application that owns the device
// memory budget through its own pool (a solver framework, a plugin host) and
// forbids growing it, and loops with latency limits where cudaMalloc's
// possible device-wide synchronisation and unbounded cost are not acceptable.
// tf_lbm_mass needs a handle, whose creation allocates; this entry point sums
// a caller-owned device array instead and touches no allocator.
//
// The block partial sums live in one file-scope device array of fixed size,
// which every GPU that loads the library holds until the process exits.  Host
// code cannot use that array's name as an address (it is a host-side stand-in
// for the symbol): the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// the device.  That first call should therefore come before any stream
// capture begins.  All calls share the array and it keeps the last call's
// contents: every partial a call reads was written by that same call, so
// nothing has to be cleared, but two calls whose kernels overlap on the GPU
// (different streams, no ordering between them) race on the array and give
// wrong sums.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>
#include <string>

#include "../../include/tflbm.h"

namespace tflbm {
void set_thread_error(const std::string& msg);  // defined in tflbm_api.cu
}

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 4096;
constexpr long long kPerBlock = 16384;                 // elements summed by one block
constexpr long long kMaxElems = kMaxBlocks * kPerBlock;  // 67,108,864
constexpr int kMaxDevices = 64;

static_assert(kMaxElems == TF_LBM_NOALLOC_MAX_ELEMS, "header limit out of date");

// (sum, compensation) of each block, then the final result: 64 KB per device.
static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxBlocks];

struct Pair {
    double s, c;  // value s + c (Neumaier)
};

__device__ __forceinline__ void add(Pair& a, double v)
{
    const double t = a.s + v;
    if (fabs(a.s) >= fabs(v)) a.c += (a.s - t) + v;
    else a.c += (v - t) + a.s;
    a.s = t;
}

__device__ __forceinline__ Pair warp_sum(Pair a)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Pair b;
        b.s = __shfl_down_sync(0xffffffffu, a.s, off);
        b.c = __shfl_down_sync(0xffffffffu, a.c, off);
        add(a, b.s);
        a.c += b.c;
    }
    return a;
}

__device__ __forceinline__ Pair block_sum(Pair a)
{
    __shared__ Pair sm[kThreads / 32];
    a = warp_sum(a);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = a;
    __syncthreads();
    Pair b{0.0, 0.0};
    if (wid == 0) {
        if (lane < kThreads / 32) b = sm[lane];
        b = warp_sum(b);
    }
    return b;  // valid in thread 0
}

// Block b sums x[b * kPerBlock, min((b + 1) * kPerBlock, n)).
__global__ void __launch_bounds__(kThreads) k_noalloc_partial(const double* __restrict__ x, long long n,
                                                              double* part)
{
    const long long beg = blockIdx.x * kPerBlock;
    const long long end = beg + kPerBlock < n ? beg + kPerBlock : n;
    Pair a{0.0, 0.0};
    for (long long i = beg + threadIdx.x; i < end; i += kThreads) add(a, x[i]);
    a = block_sum(a);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a.s;
        part[2 * blockIdx.x + 1] = a.c;
    }
}

__global__ void __launch_bounds__(kThreads) k_noalloc_final(const double* part, int nb, double* out)
{
    Pair a{0.0, 0.0};
    for (int i = threadIdx.x; i < nb; i += kThreads) {
        add(a, part[2 * i]);
        a.c += part[2 * i + 1];
    }
    a = block_sum(a);
    if (threadIdx.x == 0) *out = a.s + a.c;
}

std::mutex g_mu;
double* g_scratch[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
int scratch_address(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        tflbm::set_thread_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return TF_LBM_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        tflbm::set_thread_error("tf_lbm_sum_noalloc: device ordinal beyond 63");
        return TF_LBM_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
        double* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            tflbm::set_thread_error(std::string("cudaGetSymbolAddress of the sum scratch: ") +
                                    cudaGetErrorString(e));
            return TF_LBM_ERR_CUDA;
        }
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return TF_LBM_OK;
}

int device_pointer(const void* p, const char* name)
{
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        tflbm::set_thread_error(std::string(name) + " is not a CUDA pointer");
        return TF_LBM_ERR_ARG;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) {
        tflbm::set_thread_error(std::string(name) + " must be device or managed memory");
        return TF_LBM_ERR_ARG;
    }
    // memory of another GPU would be read (or written) from this one, which
    // without peer access is an illegal address, not an argument error
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        tflbm::set_thread_error("cudaGetDevice failed");
        return TF_LBM_ERR_CUDA;
    }
    if (a.type == cudaMemoryTypeDevice && a.device != dev) {
        tflbm::set_thread_error(std::string(name) + " lives on device " + std::to_string(a.device) +
                                ", not on the current device " + std::to_string(dev));
        return TF_LBM_ERR_ARG;
    }
    return TF_LBM_OK;
}

}  // namespace

extern "C" int tf_lbm_sum_noalloc(const double* x, int64_t n, double* out, void* stream)
{
    if (n < 0 || n > kMaxElems) {
        tflbm::set_thread_error("tf_lbm_sum_noalloc: n = " + std::to_string((long long)n) +
                                " is outside [0, " + std::to_string(kMaxElems) +
                                "], the most its fixed scratch array can reduce");
        return TF_LBM_ERR_ARG;
    }
    if (!out || (n > 0 && !x)) {
        tflbm::set_thread_error("tf_lbm_sum_noalloc: out (and x when n > 0) must not be NULL");
        return TF_LBM_ERR_ARG;
    }
    int rc;
    if ((rc = device_pointer(out, "out"))) return rc;
    if (n > 0 && (rc = device_pointer(x, "x"))) return rc;
    double* scratch = nullptr;
    if ((rc = scratch_address(&scratch))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (int)((n + kPerBlock - 1) / kPerBlock);
    if (nb > 0) k_noalloc_partial<<<nb, kThreads, 0, st>>>(x, (long long)n, scratch);
    k_noalloc_final<<<1, kThreads, 0, st>>>(scratch, nb, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        tflbm::set_thread_error(std::string("tf_lbm_sum_noalloc kernels: ") + cudaGetErrorString(e));
        return TF_LBM_ERR_CUDA;
    }
    return TF_LBM_OK;
}
