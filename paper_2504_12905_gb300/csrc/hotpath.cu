// The preprocessing, raster and PCG kernels of the hot path in one
// translation unit, so that one persistent launch can run every phase of the
// batched PCG (kb_pcg below) for all the scenes of a batch.
#include "preprocess.cu"
#include "raster.cu"
#include "cg.cu"

namespace lmrs {

// ---- grid-wide barrier ------------------------------------------------------
// An arrival counter, a generation word and an error word in device memory,
// zeroed by the host before the launch.  Thread 0 of each block arrives; the
// last of `expected` arrivals resets the counter and advances the generation;
// the others wait for the generation to move, at most timeout_ns by
// %globaltimer, then set the error word.  Every block reads the error word
// after the barrier, so a barrier that cannot complete ends the kernel
// (every block returns) instead of hanging it.  The kernel must be launched
// cooperatively: that launch guarantees every block is resident, the
// condition for blocks to wait on one another.
struct GridBar {
    unsigned int arrive;
    unsigned int gen;
    int err;  // 0, or 1: a wait ran out
    int pad;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool grid_barrier(GridBar* b, unsigned expected, unsigned long long timeout_ns) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = &b->gen;
        volatile int* verr = &b->err;
        const unsigned int g = *vgen;
        __threadfence();  // the block's writes before the barrier, before its arrival
        if (atomicAdd(&b->arrive, 1u) == expected - 1) {
            atomicExch(&b->arrive, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*vgen == g && *verr == 0) {
                if (global_ns() - t0 > timeout_ns) {
                    atomicExch(&b->err, 1);
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
    }
    __syncthreads();
    // every thread orders its later loads after the barrier (the other
    // blocks' writes of the previous phase are then the ones it sees)
    __threadfence();
    return *((volatile int*)&b->err) == 0;
}

// ---- the batched PCG in one persistent launch ---------------------------------
// The phases of the graph of per-phase launches (kb_precond_init, then per
// iteration kb_direction, kb_prep_jvp, kb_jtj, kb_prep_vjp, kb_update, then
// kb_max_dc and kb_lm_update), each a grid-stride loop over its chunk table,
// separated by grid barriers.  The per-scene FP64 scalars are those of the
// per-phase form, so both give the same result.  The kernel waits mostly on
// memory (ncu on the SH0 batch: long-scoreboard stalls first, 31% of DRAM
// throughput at 5 blocks per SM), so at SH0 it is held to 80 registers for 6
// resident blocks per SM (44 B of spills); the SH >= 1 forms keep 3.
template <int DEG>
__global__ void __launch_bounds__(kBatchBlock, DEG == 0 ? 6 : 3)
    kb_pcg(BatchTables t, int iters, GridBar* bar, unsigned long long timeout_ns) {
    __shared__ WarpSmem s_warp[kRasterWarps];
    const unsigned int n = gridDim.x;
    b_precond_init(t);
    if (!grid_barrier(bar, n, timeout_ns)) return;
    for (int it = 0; it < iters; ++it) {
        b_direction(t, it);
        if (!grid_barrier(bar, n, timeout_ns)) return;
        b_prep_jvp<DEG>(t);
        if (!grid_barrier(bar, n, timeout_ns)) return;
        b_jtj(t, s_warp);
        if (!grid_barrier(bar, n, timeout_ns)) return;
        b_prep_vjp<DEG>(t, it);
        if (!grid_barrier(bar, n, timeout_ns)) return;
        b_update(t, it);
        if (!grid_barrier(bar, n, timeout_ns)) return;
    }
    b_max_dc(t);
    if (!grid_barrier(bar, n, timeout_ns)) return;
    b_lm_update(t);
}

// One barrier expecting `missing` more blocks than the grid has: with
// missing > 0 no block can pass, every wait runs out and err is set.
__global__ void k_barrier_selftest(GridBar* bar, unsigned int missing, unsigned long long timeout_ns) {
    grid_barrier(bar, gridDim.x + missing, timeout_ns);
}

namespace {

template <typename K>
cudaError_t cooperative_grid(K kernel, int block, int* grid) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    *grid = per_sm * sms;
    return e;
}

template <int DEG>
cudaError_t pcg_deg(const BatchTables& t, int iters, GridBar* bar, unsigned long long timeout_ns, cudaStream_t st) {
    int grid = 0;
    cudaError_t e = cooperative_grid(kb_pcg<DEG>, kBatchBlock, &grid);
    if (e != cudaSuccess) return e;
    BatchTables ta = t;
    void* args[] = {&ta, &iters, &bar, &timeout_ns};
    note_launch();
    LaunchTimer* tm = active_timer();
    const int rec = tm ? timer_start(tm, "kb_pcg", st) : -1;
    e = cudaLaunchCooperativeKernel((const void*)kb_pcg<DEG>, grid, kBatchBlock, args, 0, st);
    if (tm) timer_stop(tm, rec, st);
    return e;
}

}  // namespace

size_t grid_bar_bytes() { return sizeof(GridBar); }

cudaError_t launch_b_pcg(const BatchTables& t, int deg, int iters, void* bar, double timeout_s, cudaStream_t st) {
    const unsigned long long ns = (unsigned long long)(timeout_s * 1e9);
    GridBar* b = static_cast<GridBar*>(bar);
    cudaError_t e = cudaMemsetAsync(b, 0, sizeof(GridBar), st);
    if (e != cudaSuccess) return e;
    switch (deg) {
        case 0: return pcg_deg<0>(t, iters, b, ns, st);
        case 1: return pcg_deg<1>(t, iters, b, ns, st);
        case 2: return pcg_deg<2>(t, iters, b, ns, st);
        default: return pcg_deg<3>(t, iters, b, ns, st);
    }
}

int grid_bar_error(const void* bar_host_copy) { return static_cast<const GridBar*>(bar_host_copy)->err; }

}  // namespace lmrs

using namespace lmrs;

extern "C" lmrs_status lmrs_grid_barrier_selftest(int32_t missing, double timeout_s, void* cuda_stream) {
    if (missing < 0 || !(timeout_s > 0.0) || timeout_s > 10.0) return LMRS_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int grid = 0;
    if (cooperative_grid(k_barrier_selftest, 32, &grid) != cudaSuccess) {
        cudaGetLastError();
        return LMRS_ERR_CUDA;
    }
    void* d = nullptr;
    if (pool_alloc(&d, sizeof(GridBar), st) != cudaSuccess) {
        cudaGetLastError();
        return LMRS_ERR_OOM;
    }
    GridBar* bar = static_cast<GridBar*>(d);
    GridBar h{};
    unsigned int m = (unsigned int)missing;
    unsigned long long ns = (unsigned long long)(timeout_s * 1e9);
    void* args[] = {&bar, &m, &ns};
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBar), st);
    if (e == cudaSuccess) {
        note_launch();
        e = cudaLaunchCooperativeKernel((const void*)k_barrier_selftest, grid, 32, args, 0, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, bar, sizeof(GridBar), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    pool_free(d, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LMRS_ERR_CUDA;
    }
    return h.err ? LMRS_ERR_TIMEOUT : LMRS_OK;
}
