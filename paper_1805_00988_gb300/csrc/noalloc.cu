// noalloc.cu -- the FP64 norm of a caller's state buffer without any device
// allocation.
//
// sim_norm needs a handle, and a handle allocates (the state unless wrapped,
// the reduction scratch, a status word).  Some callers cannot allocate device
// memory at the moment they need a norm: for example code running while
// another allocator (a framework's caching allocator, or a memory pool sized
// to the whole GPU) holds all free device memory, or code that must not enter
// the device allocator because an allocation can synchronise the device.
// sim_norm_noalloc serves them: the caller passes the state and receives the
// result, and the only scratch is a fixed array compiled into the library.
//
// The scratch array lives in every GPU that loads the library, for the life of
// the process.  All calls share it, so calls that overlap on the GPU (two
// streams, two threads) race and must be serialised by the caller.  Each call
// overwrites every scratch slot it later reads (one partial per block of a
// fixed grid, then the total), so nothing has to start at zero and a call
// never sees the previous call's values.
//
// In host code the array's name is only a host-side stand-in for the device
// symbol: the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device.
#include <mutex>

#include "internal.cuh"

namespace qsim {

namespace {

constexpr int kNaBlocks = 1216;            // fixed grid: 152 SMs x 8 blocks
constexpr int kNaThreads = 256;
constexpr int kNaSlots = kNaBlocks + 1;    // block partials + the total
constexpr int kNaMaxDevices = 64;

// 1217 doubles = 9,736 bytes of scratch, the whole working memory of a call
static __device__ __align__(256) double g_norm_scratch[kNaSlots];

std::mutex g_lock;
double *g_scratch_ptr[kNaMaxDevices] = {nullptr};

// FP64 sum of |a|^2 over a contiguous range per block, squares taken in FP64
template <typename R>
__global__ void __launch_bounds__(kNaThreads) k_norm_partial(const R *__restrict__ st, uint64_t n_amp, uint64_t per,
                                                             double *__restrict__ scratch)
{
    __shared__ double sh[kNaThreads / 32];
    const uint64_t lo = (uint64_t)blockIdx.x * per;
    const uint64_t hi = min(n_amp, lo + per);
    double a = 0.0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += kNaThreads) {
        const double re = (double)st[2 * i], im = (double)st[2 * i + 1];
        a += re * re + im * im;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kNaThreads / 32; ++w) s += sh[w];
        scratch[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kNaThreads) k_norm_total(double *__restrict__ scratch)
{
    __shared__ double sh[kNaThreads];
    double a = 0.0;
    for (int i = threadIdx.x; i < kNaBlocks; i += kNaThreads) a += scratch[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = kNaThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) scratch[kNaBlocks] = sh[0];
}

// device address of the scratch array on the current device (set up once)
int scratch_for_current_device(double **out)
{
    int dev = 0;
    QSIM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) return fail(SIM_EUNSUPPORTED, "sim_norm_noalloc: device index too large");
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_norm_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "sim_norm_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = (double *)p;
    }
    *out = g_scratch_ptr[dev];
    return SIM_OK;
}

}  // namespace

}  // namespace qsim

using namespace qsim;

extern "C" int sim_norm_noalloc(const void *dev_state, int n, int dtype, void *stream, double *out)
{
    set_error("");
    if (!dev_state || !out) return fail(SIM_EINVAL, "sim_norm_noalloc: dev_state and out must be non-NULL");
    if (n < 1 || n > 34)
        return fail(SIM_EINVAL, "sim_norm_noalloc: n must be in [1, 34] (the scratch holds one partial per block of "
                                "a fixed 1216-block grid; states above 2^34 amplitudes are beyond its stated maximum)");
    if (dtype != SIM_C64 && dtype != SIM_C128) return fail(SIM_EINVAL, "sim_norm_noalloc: unknown dtype");
    if ((uintptr_t)dev_state & 15) return fail(SIM_EINVAL, "sim_norm_noalloc: dev_state must be 16-byte aligned");
    double *scratch = nullptr;
    if (int rc = scratch_for_current_device(&scratch)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t n_amp = 1ull << n;
    const uint64_t per = (n_amp + kNaBlocks - 1) / kNaBlocks;
    if (dtype == SIM_C128)
        k_norm_partial<double><<<kNaBlocks, kNaThreads, 0, s>>>((const double *)dev_state, n_amp, per, scratch);
    else
        k_norm_partial<float><<<kNaBlocks, kNaThreads, 0, s>>>((const float *)dev_state, n_amp, per, scratch);
    QSIM_CUDA(cudaGetLastError());
    k_norm_total<<<1, kNaThreads, 0, s>>>(scratch);
    QSIM_CUDA(cudaGetLastError());
    QSIM_CUDA(cudaMemcpyAsync(out, scratch + kNaBlocks, sizeof(double), cudaMemcpyDeviceToHost, s));
    QSIM_CUDA(cudaStreamSynchronize(s));
    return SIM_OK;
}
