// lmrs_measure_peaks: microbenchmarks of the rates the roofline of the hot
// path divides by.  The HBM copy rate and the tensor rate come from outside
// the library; the kernels here time the other units the raster kernels lean
// on: FP32 and FP64 fused multiply-adds, the special-function unit's 2^x,
// and float atomic adds into L2 (scalar and 4-wide, to scattered slots as
// the back-scatter issues them, and 32 lanes on one address).
//
// Every kernel runs a fixed amount of work from registers (the arithmetic
// ones: independent dependency chains per thread, enough warps to fill every
// SM) or into a 64 MB scratch buffer that the call allocates and frees (the
// atomic ones), and is timed with CUDA events on the caller's stream after one
// untimed launch.
#include <cstdint>

#include "common.cuh"

namespace lmrs {
namespace {

constexpr int kPkBlock = 256;
constexpr int kPkChains = 8;  // independent chains per thread
constexpr int kPkUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(kPkBlock) k_peak_fma(T* out, int iters, T a, T b) {
    T x[kPkChains];
#pragma unroll
    for (int k = 0; k < kPkChains; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kPkUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kPkChains; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kPkChains; ++k) s += x[k];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x -> 2^(-x) stays in (0.5, 1) for x in (0, 1): no overflow, no denormals.
__global__ void __launch_bounds__(kPkBlock) k_peak_ex2(float* out, int iters) {
    float x[kPkChains];
#pragma unroll
    for (int k = 0; k < kPkChains; ++k) x[k] = 0.25f + 1e-4f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kPkUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kPkChains; ++k) x[k] = ex2_approx(-x[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kPkChains; ++k) s += x[k];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ void red_v4(float* addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// Slot (64 bytes) of update k of thread t: a multiplicative hash over the
// nslots slots (a power of two), so the lanes of a warp hit unrelated lines.
__device__ __forceinline__ unsigned long long slot_of(unsigned long long t, int k, unsigned long long mask) {
    return ((t * 0x9E3779B97F4A7C15ull + (unsigned long long)k * 0xD1B54A32D192ED03ull) >> 20) & mask;
}

// mode 0: one scalar add per update, scattered slots; 1: one 4-wide add per
// update, scattered slots; 2: scalar adds, the 32 lanes of a warp on one
// address (warps scattered).
template <int kMode>
__global__ void __launch_bounds__(kPkBlock) k_peak_atomic(float* buf, unsigned long long mask, int iters) {
    const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long w = t >> 5;
    for (int k = 0; k < iters; ++k) {
        if (kMode == 0) {
            atomicAdd(buf + slot_of(t, k, mask) * 16, 1.f);
        } else if (kMode == 1) {
            red_v4(buf + slot_of(t, k, mask) * 16, 1.f, 1.f, 1.f, 1.f);
        } else {
            atomicAdd(buf + slot_of(w, k, mask) * 16, 1.f);
        }
    }
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// Runs launch() once untimed and once timed; returns seconds (< 0 on error).
template <typename F>
double time_launch(F launch, cudaStream_t st) {
    Timer t;
    launch();
    if (cudaEventRecord(t.a, st) != cudaSuccess) return -1.0;
    launch();
    if (cudaEventRecord(t.b, st) != cudaSuccess || cudaEventSynchronize(t.b) != cudaSuccess) return -1.0;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess || cudaGetLastError() != cudaSuccess) return -1.0;
    return ms * 1e-3;
}

}  // namespace
}  // namespace lmrs

using namespace lmrs;

extern "C" lmrs_status lmrs_measure_peaks(void* cuda_stream, lmrs_peaks* out) {
    if (!out) return LMRS_ERR_INVALID_ARG;
    *out = lmrs_peaks{};
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0, clk_khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LMRS_ERR_CUDA;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    out->sm_count = sms;
    out->sm_clock_max_mhz = clk_khz / 1000.0;
    const int grid = sms * 8;  // 64 warps per SM
    const long long threads = (long long)grid * kPkBlock;
    float* f32 = nullptr;
    double* f64 = nullptr;
    float* buf = nullptr;
    const unsigned long long nslots = 1ull << 20;  // 64-byte slots: 64 MB, resident in L2
    lmrs_status rc = LMRS_OK;
    if (cudaMalloc(&f32, sizeof(float) * threads) != cudaSuccess ||
        cudaMalloc(&f64, sizeof(double) * threads) != cudaSuccess ||
        cudaMalloc(&buf, 64 * nslots) != cudaSuccess) {
        rc = LMRS_ERR_OOM;
    }
    if (rc == LMRS_OK && cudaMemsetAsync(buf, 0, 64 * nslots, st) != cudaSuccess) rc = LMRS_ERR_CUDA;
    const double fma_per_iter = (double)threads * kPkUnroll * kPkChains;
    if (rc == LMRS_OK) {
        const int it = 512;
        const double s = time_launch([&] { k_peak_fma<float><<<grid, kPkBlock, 0, st>>>(f32, it, 0.999999f, 1e-7f); }, st);
        if (s <= 0) rc = LMRS_ERR_CUDA;
        else out->fp32_tflops = 2.0 * fma_per_iter * it / s * 1e-12;
    }
    if (rc == LMRS_OK) {
        const int it = 16;
        const double s = time_launch([&] { k_peak_fma<double><<<grid, kPkBlock, 0, st>>>(f64, it, 0.999999, 1e-7); }, st);
        if (s <= 0) rc = LMRS_ERR_CUDA;
        else out->fp64_tflops = 2.0 * fma_per_iter * it / s * 1e-12;
    }
    if (rc == LMRS_OK) {
        const int it = 64;
        const double s = time_launch([&] { k_peak_ex2<<<grid, kPkBlock, 0, st>>>(f32, it); }, st);
        if (s <= 0) rc = LMRS_ERR_CUDA;
        else out->ex2_gops = fma_per_iter * it / s * 1e-9;
    }
    const int ait = 64;
    const double n_upd = (double)threads * ait;
    if (rc == LMRS_OK) {
        const double s = time_launch([&] { k_peak_atomic<0><<<grid, kPkBlock, 0, st>>>(buf, nslots - 1, ait); }, st);
        if (s <= 0) rc = LMRS_ERR_CUDA;
        else out->atomic_scattered_gops = n_upd / s * 1e-9;
    }
    if (rc == LMRS_OK) {
        const double s = time_launch([&] { k_peak_atomic<1><<<grid, kPkBlock, 0, st>>>(buf, nslots - 1, ait); }, st);
        if (s <= 0) rc = LMRS_ERR_CUDA;
        else out->red_v4_scattered_gops = n_upd / s * 1e-9;
    }
    if (rc == LMRS_OK) {
        const double s = time_launch([&] { k_peak_atomic<2><<<grid, kPkBlock, 0, st>>>(buf, nslots - 1, ait); }, st);
        if (s <= 0) rc = LMRS_ERR_CUDA;
        else out->atomic_same_address_gops = n_upd / s * 1e-9;
    }
    if (f32) cudaFree(f32);
    if (f64) cudaFree(f64);
    if (buf) cudaFree(buf);
    if (rc != LMRS_OK) cudaGetLastError();
    return rc;
}
