// Bodies of the persistent PSLR kernels and their launch helpers, shared by
// the two translation units that instantiate them: one-level sweep segments
// (pslr_apply.cu) and multi-level ones (pslr_apply_ml.cu).  The sweep form is
// a template parameter, so a kernel that never meets a merged segment carries
// no code for it.
//
// pslr_apply_kernel runs Algorithm 3 (Eq. 3.24) - and, with the transposed
// operator set, its exact transpose - in ONE cooperative launch.  One CTA owns
// one subdomain at a time (looping when there are more subdomains than
// resident CTAs); the subdomain's interior and interface vectors live in
// shared memory.  The CTA is warp-specialised:
//   * warp 8 (producer) walks the CTA's segment stream and copies every
//     segment (a level of a local factor, or a slice of E_i, F_i, C_g,i) into
//     a shared-memory ring with cp.async.bulk as soon as a slot is free
//     (full/empty mbarrier pair per slot).  It runs ahead of the consumers,
//     also across grid barriers.
//   * warps 0-7 (consumers) take the segments in order and do the arithmetic;
//     they synchronise with a named barrier that the producer never joins.
// The only cross-subdomain couplings in the method are C_g (once per series
// term, Eq. 3.1) and the reduction V^T t of the low-rank term (Eq. 3.18); they
// are the only grid barriers, split into arrive/wait so local work overlaps
// the wait.
//
// pslr_err_kernel computes E_rr(m) v = (E_s C0^{-1})^{m+1} v (Eq. 3.19) for the
// Arnoldi process with the same machinery (m+1 grid barriers).
//
// Every wait is bounded.  A grid-barrier wait that gives up latches
// PSLR_ERR_TIMEOUT; the consumers then stop the producer, wait (bounded) for
// the copies it issued, and the kernel returns.

#pragma once
#include "pslr_device.cuh"

namespace pslr {

// ------------------------------------------------------------------ the apply

// kUnit: the forward apply on the unit-diagonal operator set (no row
// pivots): L~ = D L D^{-1} and U^ = D U with D = diag(1/u_rr) of each local
// factor, so both sweeps have unit diagonals, E's rows are scaled by D_B when
// packed, and the two other right-hand sides of a solve are scaled here: f by
// D_B where it is gathered, and the C0 right-hand side by D_C0 before each C0
// solve.  Same solves as B~^{-1} and C0~^{-1} in exact arithmetic, one FP64
// instruction less per U row.
template <class T, class VT, class IO, bool kMerged, bool kUnit = false>
__device__ __forceinline__ void apply_body(const ApplyParams<T, IO> &P) {
    extern __shared__ __align__(128) char smem[];
    if (P.skip != nullptr && ld_volatile(P.skip) != 0) return;
    if (ld_volatile(P.err) != 0) return;
    const bool pivots = P.bpiv != nullptr;
    const SmemLayout L = smem_layout(P.slot_bytes, P.ring, P.max_p, P.max_q, sizeof(T), pivots, P.rs, true);
    Cta<T> c;
    if (!cta_start(c, smem, L, P.ring, P.slot_bytes, P.stream, P.stream_off, P.segbase)) return;

    const VT *V = reinterpret_cast<const VT *>(P.V);
    const int q = P.q, p = P.p, r = P.r, m = P.m;
    const bool lr_before = r > 0 && !P.lowrank_after;
    const bool lr_after = r > 0 && P.lowrank_after;
    const T om = P.omega;
    const bool scaled = om != T(1);  // the Sec. 1 Neumann polynomial instead of Eq. 3.3
    const int tid = threadIdx.x;
    bool ok = true;

    // ---- phase 0: u = B^{-1} f, t = g - F u (Algorithm 3, step 2); without a
    // low-rank term before the series also w_0 = C0^{-1} t.
    for (int i = blockIdx.x; i < P.s; i += gridDim.x) {
        const Counts k = counts_of(P.cnt, i);
        const int io = P.ioff[i], np_ = P.ioff[i + 1] - io;
        const int go = P.goff[i], nq = P.goff[i + 1] - go;
        for (int j = tid; j < np_; j += kConsumers) {
            T f = T(P.b[P.perm[io + j]]);
            if constexpr (kUnit) f *= __ldg(P.dB + io + j);
            c.xi[j] = f;
        }
        if (tid == 0) c.xi[np_] = T(0);
        for (int j = tid; j < nq; j += kConsumers) c.si[j] = T(P.b[P.perm[p + go + j]]);
        csync();
        solve_local<T, kMerged, kUnit>(c, c.xi, np_, pivots ? P.bpiv + io : nullptr, P.pivot_post, k.n[kB1],
                                       k.n[kB2], P.err);
        ell_op<T, false>(c, c.si, c.xi, true, k.n[kF], P.err);
        if (lr_before) {
            lowrank_partial(c, V, P.ldv, r, go, nq, c.si, P.part + (int64_t)i * r, 1, P.rs);
            for (int j = tid; j < nq; j += kConsumers) P.acc[go + j] = c.si[j];
        } else {
            if (tid == 0) c.si[nq] = T(0);
            if constexpr (kUnit)
                for (int j = tid; j < nq; j += kConsumers) c.si[j] *= __ldg(P.dC + go + j);
            csync();
            solve_local<T, kMerged, kUnit>(c, c.si, nq, pivots ? P.cpiv + go : nullptr, P.pivot_post, k.n[kC1],
                                           k.n[kC2], P.err);
            for (int j = tid; j < nq; j += kConsumers) {
                P.wbuf[go + j] = c.si[j];
                P.acc[go + j] = c.si[j];
            }
        }
        csync();
    }
    if (tid == 0 && blockIdx.x == 0) {
        P.wbuf[q] = T(0);
        P.wbuf[(q + 1) + q] = T(0);
    }

    // ---- phase 1: t <- t + V G V^T t, then w_0 = C0^{-1} t (steps 3-4)
    if (lr_before) {
        grid_arrive(c, P.bar, P.grid);
        ok = grid_wait(c, P.bar, P.err, P.wait_limit);
        if (!ok) goto abort;
        lowrank_coeffs(c, P.part, P.G, P.s, r, P.rs);
        for (int i = blockIdx.x; i < P.s; i += gridDim.x) {
            const Counts k = counts_of(P.cnt, i);
            const int go = P.goff[i], nq = P.goff[i + 1] - go;
            for (int j = tid; j < nq; j += kConsumers) c.si[j] = __ldcg(P.acc + go + j);
            if (tid == 0) c.si[nq] = T(0);
            csync();
            lowrank_update(c, V, P.ldv, r, go, nq, c.si, 1, P.rs);
            if constexpr (kUnit) {
                for (int j = tid; j < nq; j += kConsumers) c.si[j] *= __ldg(P.dC + go + j);
                csync();
            }
            solve_local<T, kMerged, kUnit>(c, c.si, nq, pivots ? P.cpiv + go : nullptr, P.pivot_post, k.n[kC1],
                                           k.n[kC2], P.err);
            for (int j = tid; j < nq; j += kConsumers) {
                P.wbuf[go + j] = c.si[j];
                P.acc[go + j] = c.si[j];
            }
            csync();
        }
    }

    // ---- series terms w_k = C0^{-1}(F B^{-1} E w_{k-1} - C_g w_{k-1}), acc += w_k (Eq. 3.3)
    for (int kk = 1; kk <= m; ++kk) {
        const T *wprev = P.wbuf + ((kk - 1) & 1) * (q + 1);
        T *wnext = P.wbuf + (kk & 1) * (q + 1);
        grid_arrive(c, P.bar, P.grid);
        bool waited = false;
        for (int i = blockIdx.x; i < P.s; i += gridDim.x) {
            const Counts k = counts_of(P.cnt, i);
            const int io = P.ioff[i], np_ = P.ioff[i + 1] - io;
            const int go = P.goff[i], nq = P.goff[i + 1] - go;
            for (int j = tid; j < nq; j += kConsumers) c.wi[j] = __ldcg(wprev + go + j);
            if (tid == 0) c.wi[nq] = T(0);
            fill(c.xi, np_ + 1, T(0));
            csync();
            ell_op<T, false>(c, c.xi, c.wi, false, k.n[kE], P.err);                      // E w
            solve_local<T, kMerged, kUnit>(c, c.xi, np_, pivots ? P.bpiv + io : nullptr, P.pivot_post, k.n[kB1],
                                           k.n[kB2], P.err);                            // B^{-1}
            fill(c.si, nq + 1, T(0));
            csync();
            ell_op<T, false>(c, c.si, c.xi, false, k.n[kF], P.err);                      // F
            if (!waited) {
                ok = grid_wait(c, P.bar, P.err, P.wait_limit);
                waited = true;
                if (!ok) goto abort;
            }
            ell_op<T, true>(c, c.si, wprev, true, k.n[kCg], P.err);                      // - C_g w
            if constexpr (kUnit) {
                for (int j = tid; j < nq; j += kConsumers) c.si[j] *= __ldg(P.dC + go + j);
                csync();
            }
            solve_local<T, kMerged, kUnit>(c, c.si, nq, pivots ? P.cpiv + go : nullptr, P.pivot_post, k.n[kC1],
                                           k.n[kC2], P.err);                            // C0^{-1}
            if (scaled)  // N w = (1 - omega) w + omega C0^{-1} E_s w, N = I - omega C0^{-1} S
                for (int j = tid; j < nq; j += kConsumers)
                    c.si[j] = fma_t(T(1) - om, __ldcg(wprev + go + j), om * c.si[j]);
            for (int j = tid; j < nq; j += kConsumers) {
                wnext[go + j] = c.si[j];
                P.acc[go + j] = __ldcg(P.acc + go + j) + c.si[j];
            }
            csync();
        }
        if (!waited) {  // a CTA without subdomains still takes part in the barrier
            ok = grid_wait(c, P.bar, P.err, P.wait_limit);
            if (!ok) goto abort;
        }
    }

    // ---- transposed order: w <- w + V G^T V^T w after the series
    if (lr_after) {
        for (int i = blockIdx.x; i < P.s; i += gridDim.x) {
            const int go = P.goff[i], nq = P.goff[i + 1] - go;
            for (int j = tid; j < nq; j += kConsumers) c.si[j] = __ldcg(P.acc + go + j);
            csync();
            lowrank_partial(c, V, P.ldv, r, go, nq, c.si, P.part + (int64_t)i * r, 1, P.rs);
        }
        grid_arrive(c, P.bar, P.grid);
        ok = grid_wait(c, P.bar, P.err, P.wait_limit);
        if (!ok) goto abort;
        lowrank_coeffs(c, P.part, P.G, P.s, r, P.rs);
    }

    // ---- y = acc; x = B^{-1}(f - E y); scatter (steps 5-6)
    for (int i = blockIdx.x; i < P.s; i += gridDim.x) {
        const Counts k = counts_of(P.cnt, i);
        const int io = P.ioff[i], np_ = P.ioff[i + 1] - io;
        const int go = P.goff[i], nq = P.goff[i + 1] - go;
        for (int j = tid; j < nq; j += kConsumers) c.wi[j] = scaled ? om * __ldcg(P.acc + go + j) : __ldcg(P.acc + go + j);
        if (tid == 0) c.wi[nq] = T(0);
        for (int j = tid; j < np_; j += kConsumers) {
            T f = T(P.b[P.perm[io + j]]);
            if constexpr (kUnit) f *= __ldg(P.dB + io + j);
            c.xi[j] = f;
        }
        if (tid == 0) c.xi[np_] = T(0);
        csync();
        if (lr_after) lowrank_update(c, V, P.ldv, r, go, nq, c.wi, 1, P.rs);
        ell_op<T, false>(c, c.xi, c.wi, true, k.n[kE], P.err);
        solve_local<T, kMerged, kUnit>(c, c.xi, np_, pivots ? P.bpiv + io : nullptr, P.pivot_post, k.n[kB1],
                                       k.n[kB2], P.err);
        for (int j = tid; j < np_; j += kConsumers) P.z[P.perm[io + j]] = IO(c.xi[j]);
        for (int j = tid; j < nq; j += kConsumers) P.z[P.perm[p + go + j]] = IO(c.wi[j]);
        csync();
    }
    return;
abort:
    consumers_abort_drain(c);
}

// Two instances of each persistent kernel: one CTA per SM with all the
// registers it wants, and (suffix _x2) an instance of which two CTAs fit an
// SM, for problems with more subdomains than SMs: two subdomains' level
// chains then share an SM and hide each other's latencies instead of one CTA
// sweeping them one after the other.  Two CTAs are 18 warps, so one SM
// sub-partition holds five of them in its 16K registers: at most 96 registers
// per thread, which is what the launch bound asks the compiler for.
template <class T, class VT, class IO, bool kMerged, bool kUnit = false>
__global__ void __launch_bounds__(kThreads, 1) pslr_apply_kernel(const ApplyParams<T, IO> P) {
    apply_body<T, VT, IO, kMerged, kUnit>(P);
}
template <class T, class VT, class IO, bool kMerged, bool kUnit = false>
__global__ void __launch_bounds__(kThreads, 2) pslr_apply_kernel_x2(const ApplyParams<T, IO> P) {
    apply_body<T, VT, IO, kMerged, kUnit>(P);
}

// ------------------------------------------------------------ E_rr(m) matvec

template <class T, bool kMerged>
__device__ __forceinline__ void err_body(const ErrParams<T> &P) {
    extern __shared__ __align__(128) char smem[];
    if (ld_volatile(P.err) != 0) return;
    const bool pivots = P.bpiv != nullptr;
    const SmemLayout L = smem_layout(P.slot_bytes, P.ring, P.max_p, P.max_q, sizeof(T), pivots, P.rs, true);
    Cta<T> c;
    if (!cta_start(c, smem, L, P.ring, P.slot_bytes, P.stream, P.stream_off, P.segbase)) return;
    const int q = P.q, tid = threadIdx.x;
    bool ok = true;
    if (tid == 0 && blockIdx.x == 0) {
        P.abuf[q] = T(0);
        P.abuf[(q + 1) + q] = T(0);
    }
    for (int rep = 0; rep <= P.m; ++rep) {
        T *a = P.abuf + (rep & 1) * (q + 1);
        const T *vsrc = rep == 0 ? P.vin : P.vout;
        // a_i = C0_i^{-1} v_i  (local)
        for (int i = blockIdx.x; i < P.s; i += gridDim.x) {
            const Counts k = counts_of(P.cnt, i);
            const int go = P.goff[i], nq = P.goff[i + 1] - go;
            for (int j = tid; j < nq; j += kConsumers) c.si[j] = __ldcg(vsrc + go + j);
            if (tid == 0) c.si[nq] = T(0);
            csync();
            solve_local<T, kMerged>(c, c.si, nq, pivots ? P.cpiv + go : nullptr, 0, k.n[kC1], k.n[kC2], P.err);
            for (int j = tid; j < nq; j += kConsumers) a[go + j] = c.si[j];
            csync();
        }
        grid_arrive(c, P.bar, P.grid);
        bool waited = false;
        // v_i = F_i B_i^{-1} E_i a_i - (C_g a)_i
        for (int i = blockIdx.x; i < P.s; i += gridDim.x) {
            const Counts k = counts_of(P.cnt, i);
            const int io = P.ioff[i], np_ = P.ioff[i + 1] - io;
            const int go = P.goff[i], nq = P.goff[i + 1] - go;
            for (int j = tid; j < nq; j += kConsumers) c.wi[j] = __ldcg(a + go + j);
            if (tid == 0) c.wi[nq] = T(0);
            fill(c.xi, np_ + 1, T(0));
            csync();
            ell_op<T, false>(c, c.xi, c.wi, false, k.n[kE], P.err);
            solve_local<T, kMerged>(c, c.xi, np_, pivots ? P.bpiv + io : nullptr, 0, k.n[kB1], k.n[kB2], P.err);
            fill(c.si, nq + 1, T(0));
            csync();
            ell_op<T, false>(c, c.si, c.xi, false, k.n[kF], P.err);
            if (!waited) {
                ok = grid_wait(c, P.bar, P.err, P.wait_limit);
                waited = true;
                if (!ok) goto abort;
            }
            ell_op<T, true>(c, c.si, a, true, k.n[kCg], P.err);
            for (int j = tid; j < nq; j += kConsumers) P.vout[go + j] = c.si[j];
            csync();
        }
        if (!waited) {
            ok = grid_wait(c, P.bar, P.err, P.wait_limit);
            if (!ok) goto abort;
        }
    }
    return;
abort:
    consumers_abort_drain(c);
}

template <class T, bool kMerged>
__global__ void __launch_bounds__(kThreads, 1) pslr_err_kernel(const ErrParams<T> P) {
    err_body<T, kMerged>(P);
}
template <class T, bool kMerged>
__global__ void __launch_bounds__(kThreads, 2) pslr_err_kernel_x2(const ErrParams<T> P) {
    err_body<T, kMerged>(P);
}

// ------------------------------------------------------------- launch helpers

template <class K, class Prm>
static inline cudaError_t launch_coop(K kern, const Prm &P, int grid, int smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<Prm *>(&P)};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(kThreads), args, smem, st);
}

template <class K>
static inline cudaError_t blocks_per_sm(K kern, int smem, int *per) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, kern, kThreads, smem);
    return e;
}

}  // namespace pslr
