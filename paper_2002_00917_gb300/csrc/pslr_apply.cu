// Persistent PSLR kernels for sm_103a (bodies in pslr_kernels.cuh): the
// Algorithm 3 apply and its transpose, and the E_rr(m) matvec of the Arnoldi
// set-up, each one cooperative launch.
//
// This translation unit instantiates them for one-level sweep segments (every
// layout but the merged one) and holds the host launchers; pslr_apply_ml.cu
// instantiates them for merged, multi-level segments.

#include "pslr_kernels.cuh"

namespace pslr {

// Launchers of one sweep form (kMerged), instantiated where used.
template <bool kMerged>
struct Launch {
    static cudaError_t apply_fp64(const ApplyParams<double> &P, int smem, bool dual, cudaStream_t st) {
        if (dual) return launch_coop(pslr_apply_kernel_x2<double, double, double, kMerged>, P, P.grid, smem, st);
        return launch_coop(pslr_apply_kernel<double, double, double, kMerged>, P, P.grid, smem, st);
    }
    static cudaError_t apply_fp32(const ApplyParams<float> &P, int smem, bool dual, cudaStream_t st) {
        if (dual) return launch_coop(pslr_apply_kernel_x2<float, __nv_bfloat16, float, kMerged>, P, P.grid, smem, st);
        return launch_coop(pslr_apply_kernel<float, __nv_bfloat16, float, kMerged>, P, P.grid, smem, st);
    }
    static cudaError_t apply_f32d(const ApplyParams<float, double> &P, int smem, bool dual, cudaStream_t st) {
        if (dual) return launch_coop(pslr_apply_kernel_x2<float, __nv_bfloat16, double, kMerged>, P, P.grid, smem, st);
        return launch_coop(pslr_apply_kernel<float, __nv_bfloat16, double, kMerged>, P, P.grid, smem, st);
    }
    static cudaError_t err_fp64(const ErrParams<double> &P, int smem, bool dual, cudaStream_t st) {
        if (dual) return launch_coop(pslr_err_kernel_x2<double, kMerged>, P, P.grid, smem, st);
        return launch_coop(pslr_err_kernel<double, kMerged>, P, P.grid, smem, st);
    }
    // CTAs per SM of the kernels that launch with this smem size (the smaller
    // of the FP64 apply and E_rr, or of the two FP32 apply forms).
    static cudaError_t per_sm(int smem, bool fp32, bool dual, int *per) {
        int a = 0, b = 0;
        cudaError_t e;
        if (fp32 && dual) {
            e = blocks_per_sm(pslr_apply_kernel_x2<float, __nv_bfloat16, float, kMerged>, smem, &a);
            if (e == cudaSuccess) e = blocks_per_sm(pslr_apply_kernel_x2<float, __nv_bfloat16, double, kMerged>, smem, &b);
        } else if (fp32) {
            e = blocks_per_sm(pslr_apply_kernel<float, __nv_bfloat16, float, kMerged>, smem, &a);
            if (e == cudaSuccess) e = blocks_per_sm(pslr_apply_kernel<float, __nv_bfloat16, double, kMerged>, smem, &b);
        } else if (dual) {
            e = blocks_per_sm(pslr_apply_kernel_x2<double, double, double, kMerged>, smem, &a);
            if (e == cudaSuccess) e = blocks_per_sm(pslr_err_kernel_x2<double, kMerged>, smem, &b);
        } else {
            e = blocks_per_sm(pslr_apply_kernel<double, double, double, kMerged>, smem, &a);
            if (e == cudaSuccess) e = blocks_per_sm(pslr_err_kernel<double, kMerged>, smem, &b);
        }
        *per = a < b ? a : b;
        return e;
    }
};

// The merged-segment instances (pslr_apply_ml.cu).
cudaError_t launch_apply_fp64_ml(const ApplyParams<double> &P, int smem, bool dual, cudaStream_t st);
cudaError_t launch_apply_fp32_ml(const ApplyParams<float> &P, int smem, bool dual, cudaStream_t st);
cudaError_t launch_apply_f32d_ml(const ApplyParams<float, double> &P, int smem, bool dual, cudaStream_t st);
cudaError_t launch_err_fp64_ml(const ErrParams<double> &P, int smem, bool dual, cudaStream_t st);
cudaError_t per_sm_ml(int smem, bool fp32, bool dual, int *per);

cudaError_t launch_apply_fp64(const ApplyParams<double> &P, int smem, bool dual, bool merged, cudaStream_t st) {
    return merged ? launch_apply_fp64_ml(P, smem, dual, st) : Launch<false>::apply_fp64(P, smem, dual, st);
}
cudaError_t launch_apply_fp32(const ApplyParams<float> &P, int smem, bool dual, bool merged, cudaStream_t st) {
    return merged ? launch_apply_fp32_ml(P, smem, dual, st) : Launch<false>::apply_fp32(P, smem, dual, st);
}
cudaError_t launch_apply_f32d(const ApplyParams<float, double> &P, int smem, bool dual, bool merged,
                              cudaStream_t st) {
    return merged ? launch_apply_f32d_ml(P, smem, dual, st) : Launch<false>::apply_f32d(P, smem, dual, st);
}
cudaError_t launch_err_fp64(const ErrParams<double> &P, int smem, bool dual, bool merged, cudaStream_t st) {
    return merged ? launch_err_fp64_ml(P, smem, dual, st) : Launch<false>::err_fp64(P, smem, dual, st);
}

// Largest cooperative grid of the persistent kernels for a dynamic smem size
// (the smallest occupancy of the kernels that launch with it: FP64 apply and
// E_rr, or the two FP32 apply forms - their two-CTAs-per-SM instances when
// dual is set - in the sweep form of the layout).
int max_coresident_apply(int smem, bool fp32, bool dual, bool merged) {
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const cudaError_t e = merged ? per_sm_ml(smem, fp32, dual, &per) : Launch<false>::per_sm(smem, fp32, dual, &per);
    if (e != cudaSuccess) return 0;
    return per * nsm;
}

}  // namespace pslr
