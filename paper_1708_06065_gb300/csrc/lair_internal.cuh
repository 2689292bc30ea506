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
