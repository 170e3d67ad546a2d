// The persistent PSLR kernels instantiated for merged sweep segments: several
// consecutive levels of a factor in one ring slot (kSegMore blocks), used
// where the ring is too shallow for one bulk copy per level to keep ahead of
// the level sweeps.  Same bodies as pslr_apply.cu's one-level instances.

#include "pslr_kernels.cuh"

namespace pslr {

// Launchers of one sweep form (kMerged), instantiated by this translation unit.
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

cudaError_t launch_apply_fp64_ml(const ApplyParams<double> &P, int smem, bool dual, cudaStream_t st) {
    return Launch<true>::apply_fp64(P, smem, dual, st);
}
cudaError_t launch_apply_fp32_ml(const ApplyParams<float> &P, int smem, bool dual, cudaStream_t st) {
    return Launch<true>::apply_fp32(P, smem, dual, st);
}
cudaError_t launch_apply_f32d_ml(const ApplyParams<float, double> &P, int smem, bool dual, cudaStream_t st) {
    return Launch<true>::apply_f32d(P, smem, dual, st);
}
cudaError_t launch_err_fp64_ml(const ErrParams<double> &P, int smem, bool dual, cudaStream_t st) {
    return Launch<true>::err_fp64(P, smem, dual, st);
}
cudaError_t per_sm_ml(int smem, bool fp32, bool dual, int *per) { return Launch<true>::per_sm(smem, fp32, dual, per); }

}  // namespace pslr
