// Batched apply kernel, one precision form: FP32 arithmetic and BF16 V on FP64 vectors (the FP32 preconditioner inside the FP64 batched FGMRES); one
// instantiation per number of right-hand sides (1..kMaxBatchRhs), so the rhs
// loops and vector accesses are resolved at compile time.
#include "pslr_batch.cuh"

namespace pslr {

namespace {
using P_t = BatchParams<float, double>;

template <int NR>
cudaError_t launch_nr(const P_t &P, int smem, cudaStream_t st) {
    auto kern = pslr_batch_apply_kernel<float, __nv_bfloat16, double, NR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<P_t *>(&P)};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(P.grid), dim3(kThreads), args, smem, st);
}

template <int NR>
int coresident_nr(int smem) {
    auto kern = pslr_batch_apply_kernel<float, __nv_bfloat16, double, NR>;
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, smem) != cudaSuccess) return 0;
    return per * nsm;
}
}  // namespace

cudaError_t launch_batch_f32d(const void *params, int smem, cudaStream_t st) {
    const P_t &P = *static_cast<const P_t *>(params);
    switch (P.nrhs) {
    case 1: return launch_nr<1>(P, smem, st);
    case 2: return launch_nr<2>(P, smem, st);
    case 3: return launch_nr<3>(P, smem, st);
    case 4: return launch_nr<4>(P, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

int coresident_batch_f32d(int smem, int nrhs) {
    switch (nrhs) {
    case 1: return coresident_nr<1>(smem);
    case 2: return coresident_nr<2>(smem);
    case 3: return coresident_nr<3>(smem);
    case 4: return coresident_nr<4>(smem);
    default: return 0;
    }
}

}  // namespace pslr
