// lair_internal.cuh -- shared device/host definitions of the lAIR CUDA library.
//
// Conventions
//  * Device CSR matrices use int32 row pointers and column indices (sizes are
//    checked against 2^31 - 1 on the host) and keep an FP64 value array plus,
//    in mixed precision, an FP32 copy used by the cycle.
//  * Every floating-point operation whose result feeds a structural decision on
//    a coarser level (strength, splitting, lumping) is written with explicit
//    __fma_rn / __dmul_rn / __dadd_rn / IEEE division, in the order documented at
//    each routine, so that the hierarchy is a deterministic function of A.
//  * Kernels report failures through a device status word (atomicCAS of a
//    lair_status code), read by the host at its synchronisation points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lair.h"

namespace lair {

constexpr int8_t CF_F = 0;
constexpr int8_t CF_C = 1;
constexpr int8_t CF_U = -1;

// the lumping kernels read a row of the Galerkin product ROW_CHUNK entries at a time (predicated loads, all
// independent), so a row costs a round of memory latency per chunk instead of one per entry
constexpr int ROW_CHUNK = 8;

struct DCsr {
    int nr = 0, nc = 0, nnz = 0;
    int *rp = nullptr;
    int *col = nullptr;
    double *val = nullptr;
    float *val32 = nullptr;
};

struct Graph {          // pattern-only CSR
    int n = 0, nnz = 0;     // nnz: capacity of col (at least rp[n])
    int *rp = nullptr;
    int *col = nullptr;
};

// -------------------------------------------------------------------------------------
// error reporting from device code
// -------------------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int *st, int code) {
    if (st) atomicCAS(st, 0, code);
}

// -------------------------------------------------------------------------------------
// grid-wide barrier for kernels whose blocks are all resident (cooperative launches), on one
// monotonic arrival counter *ctl (zero at launch): barrier b is passed once the counter reaches
// b * gridDim.x. Arrival is an acquire-release atomic and the wait an acquire load, so the
// barrier orders the blocks' memory operations without separate fences and nothing is reset
// between barriers. `passed` is thread 0's running target (zero at kernel start). A wait gives
// up after `limit` polls, or as soon as another block has reported LAIR_ERR_DEVICE_TIMEOUT; it
// then reports LAIR_ERR_DEVICE_TIMEOUT and the call returns false, after which the kernel
// returns (its other blocks do the same at their next barrier).
// -------------------------------------------------------------------------------------
__device__ __forceinline__ bool grid_barrier(unsigned *ctl, int *status, long long limit, unsigned &passed) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        passed += gridDim.x;
        unsigned old;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(ctl) : "memory");
        if (old + 1 != passed) {
            long long spins = 0;
            for (;;) {
                unsigned v;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctl) : "memory");
                if ((int)(v - passed) >= 0) break;
                ++spins;
                if (spins > limit ||
                    ((spins & 63) == 0 && status && *(volatile int *)status == LAIR_ERR_DEVICE_TIMEOUT)) {
                    set_status(status, LAIR_ERR_DEVICE_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return ok != 0;
}

// -------------------------------------------------------------------------------------
// programmatic dependent launch (the V-cycle's kernels): the kernel first lets the next kernel of the
// stream begin launching (its blocks may be scheduled once every block of this one has started), then
// waits until the previous kernel has completed and its writes are visible. Both are no-ops when the
// launch does not carry the programmatic-serialization attribute (launch_pdl below).
// -------------------------------------------------------------------------------------
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// -------------------------------------------------------------------------------------
// warp helpers
// -------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Ascending bitonic sort of 32 R (key, value) pairs held by a warp, element e = 32 r + lane
// in key[r], val[r]. Exchanges at distance < 32 go through shuffles, the others stay inside a
// lane's registers; every index is a compile-time constant. Keys are distinct apart from
// padding (INT_MAX), which ends up last.
template <int R>
__device__ __forceinline__ void warp_bitonic(int (&key)[R], double (&val)[R], int lane) {
#pragma unroll
    for (int k = 2; k <= 32 * R; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int r2 = r ^ (j >> 5);
                    if (r2 > r) {
                        const bool up = ((32 * r + lane) & k) == 0;
                        if (up ? key[r] > key[r2] : key[r] < key[r2]) {
                            const int tk = key[r]; key[r] = key[r2]; key[r2] = tk;
                            const double tv = val[r]; val[r] = val[r2]; val[r2] = tv;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int pk = __shfl_xor_sync(0xffffffffu, key[r], j);
                    const double pv = __shfl_xor_sync(0xffffffffu, val[r], j);
                    const bool up = ((32 * r + lane) & k) == 0, lower = (lane & j) == 0;
                    if (lower == up ? pk < key[r] : pk > key[r]) {
                        key[r] = pk;
                        val[r] = pv;
                    }
                }
            }
        }
    }
}

// -------------------------------------------------------------------------------------
// host-side launch helpers (defined in lair_api.cu)
// -------------------------------------------------------------------------------------
void count_launch(int k = 1);
// a kernel that starts with pdl_enter(), launched so that it may overlap the tail of the previous kernel in
// the stream (a programmatic edge when the stream is captured into a graph)
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}
// streaming multiprocessors of the current device (read once per device; 152 on a GB300)
int device_sms();
inline int grid_for(long long work, int block, int max_blocks = 0) {
    if (max_blocks <= 0) max_blocks = device_sms() * 32;
    long long g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}


}  // namespace lair
