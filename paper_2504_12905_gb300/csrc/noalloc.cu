// lmrs_step_size_noalloc: the step-size reduction without any device
// allocation, for callers that cannot call cudaMalloc (see include/lmrs.h).
//
// Its scratch is a fixed file-scope device array instead of scene-owned or
// cudaMalloc'd memory.  Every GPU that loads the library holds this array
// (16,512 bytes) until the process exits.  All calls on a device share it:
// calls that overlap on the GPU race on it.  Each call clears the words that
// must start at zero before it launches.
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "reduce.cuh"

namespace lmrs {
namespace {

constexpr int kNaBlock = 256;
constexpr int kNaItems = 8;                         // Gaussians per thread
constexpr int kNaPerBlock = kNaBlock * kNaItems;    // Gaussians per block
constexpr int kNaMaxBlocks = 4096;                  // one partial maximum per block
constexpr long long kNaMaxGauss = (long long)kNaMaxBlocks * kNaPerBlock;  // 8,388,608
constexpr int kNaCounter = kNaMaxBlocks;            // word index of the arrival counter
constexpr int kNaResult = kNaMaxBlocks + 1;         // word index of the result
constexpr int kNaWords = kNaMaxBlocks + 32;

// Partial maxima, arrival counter and result.  In host code this name is a
// host-side stand-in, not a device address: host code uses the address
// obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned int g_noalloc_scratch[kNaWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned int* g_scratch_ptr[kMaxDevices] = {};

// Per-device set-up: done by the first call on each device, with that device
// current.
cudaError_t scratch_address(int dev, unsigned int** out) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<unsigned int*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// max |x| over the SH degree-0 entries (as k_max_dc), with fixed work per
// block: every block stores its partial maximum in the scratch array and the
// last block to arrive reduces the partials into the result word.
__global__ void __launch_bounds__(kNaBlock) k_max_dc_noalloc(const float* x, long long G, int K,
                                                             unsigned int* scratch) {
    __shared__ float s_w[kNaBlock / kWarp];
    __shared__ bool s_last;
    float m = 0.f;
    const long long base = (long long)blockIdx.x * kNaPerBlock;
#pragma unroll
    for (int it = 0; it < kNaItems; ++it) {
        const long long g = base + (long long)it * kNaBlock + threadIdx.x;
        if (g < G) {
            const float* e = x + 11ll * G + g * K * 3;
            m = fmaxf(m, fmaxf(fabsf(e[0]), fmaxf(fabsf(e[1]), fabsf(e[2]))));
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s_w[w] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float bm = 0.f;
        for (int i = 0; i < kNaBlock / kWarp; ++i) bm = fmaxf(bm, s_w[i]);
        scratch[blockIdx.x] = __float_as_uint(bm);  // non-negative: bits order as values
        __threadfence();
        const unsigned int t = atomicAdd(&scratch[kNaCounter], 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    unsigned int r = 0u;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kNaBlock) r = max(r, ((volatile unsigned int*)scratch)[i]);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) r = max(r, __shfl_xor_sync(kFull, r, o));
    __shared__ unsigned int s_r[kNaBlock / kWarp];
    if (lane == 0) s_r[w] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int tot = 0u;
        for (int i = 0; i < kNaBlock / kWarp; ++i) tot = max(tot, s_r[i]);
        scratch[kNaResult] = tot;
        scratch[kNaCounter] = 0u;
    }
}

}  // namespace
}  // namespace lmrs

extern "C" lmrs_status lmrs_step_size_noalloc(const float* x_dev, int64_t n_gauss, int32_t sh_degree,
                                              int64_t lm_step, double lr_warm, double lr_cap, double color_bound,
                                              int32_t warm_iters, void* cuda_stream, double* eta_host) {
    using namespace lmrs;
    if (!x_dev || !eta_host || n_gauss <= 0 || sh_degree < 0 || sh_degree > 3) return LMRS_ERR_INVALID_ARG;
    if (n_gauss > kNaMaxGauss) return LMRS_ERR_BUDGET;  // the fixed scratch holds 4096 block partials
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return LMRS_ERR_CUDA;
    }
    unsigned int* scratch = nullptr;
    if (scratch_address(dev, &scratch) != cudaSuccess) {
        cudaGetLastError();
        return LMRS_ERR_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int K = (sh_degree + 1) * (sh_degree + 1);
    const int blocks = (int)((n_gauss + kNaPerBlock - 1) / kNaPerBlock);
    // the arrival counter and the result must start at zero
    if (cudaMemsetAsync(scratch + kNaCounter, 0, 2 * sizeof(unsigned int), st) != cudaSuccess) {
        cudaGetLastError();
        return LMRS_ERR_CUDA;
    }
    LMRS_LAUNCH(k_max_dc_noalloc, blocks, kNaBlock, 0, st, x_dev, (long long)n_gauss, K, scratch);
    unsigned int bits = 0u;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, scratch + kNaResult, sizeof(bits), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LMRS_ERR_CUDA;
    float m;
    std::memcpy(&m, &bits, sizeof(m));
    if (lm_step < warm_iters) *eta_host = lr_warm;
    else if (m == 0.f) *eta_host = lr_cap;
    else *eta_host = std::fmin(lr_cap, color_bound / (double)m);
    return LMRS_OK;
}
