// Warp reduction of eight values per lane in a fixed order, used by the
// low-rank partial sums of the apply kernels and the column-wise dot products
// of the Krylov kernels.
//
// A butterfly that halves the vector at each exchange: lanes l and l^16 swap
// half of their eight accumulators and add (4 adds), then l^8 (2), then l^4
// (1); each lane now holds one value summed over eight lanes, and two more
// exchanges (l^2, l^1) finish it.  9 dependent adds per warp for eight sums,
// instead of 5 for each of the eight with independent shuffle trees - which
// matters in FP64 on GB300, where every warp-wide FP64 add holds the
// scheduler's FP64 pipe for many cycles.  On return lane l holds the warp sum
// of value (l >> 2).  (Measured: 64^3 apply 513 -> 490 us in FP64.  In the
// Krylov kernels it pays once each warp reduces after many rows - lanes over
// rows, a warp per chunk of columns - rather than after a few rows per
// thread: 64^3 FGMRES(120) 541 -> 460 ms in FP64.)
#pragma once

namespace pslr {

template <class T>
__device__ __forceinline__ T warp_reduce8(const T (&a)[8]) {
    const int lane = threadIdx.x & 31;
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    T b[4], c[2];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const T keep = h16 ? a[t + 4] : a[t], send = h16 ? a[t] : a[t + 4];
        b[t] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const T keep = h8 ? b[t + 2] : b[t], send = h8 ? b[t] : b[t + 2];
        c[t] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    T d = (h4 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, h4 ? c[0] : c[1], 4);
    d += __shfl_xor_sync(0xffffffffu, d, 2);
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    return d;
}

}  // namespace pslr
