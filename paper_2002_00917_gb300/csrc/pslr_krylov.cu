// FP64 Krylov kernels for sm_103a: the FGMRES of Section 4 and the Arnoldi
// process of Algorithm 1 (steps 6-7) share them.
//
// Classical Gram-Schmidt applied twice (CGS2) is split into three passes over
// the rows, each one launch whose blocks own contiguous row ranges, stream
// the basis V column-chunk by column-chunk (coalesced along rows) and leave
// one partial per block; the partials are added in a fixed two-level order
// (finish_reduction), so every reduction is deterministic:
//   pass 1  w = A z (optional, fused CSR SpMV), h1 = V^T w
//   pass 2  w -= V h1,                        h2 = V^T w
//   pass 3  w -= V h2,                        ||w||^2
// then, in FGMRES, one launch writes v_{j+1} = w / h_{j+1,j} while one warp
// of it forms h = h1 + h2, h_{j+1,j} = ||w|| and applies the Givens
// rotations (the Arnoldi of Algorithm 1 normalises with host-side norms).
// The second pass is not optional here: with a good preconditioner
// A M^{-1} v_j is close to v_j, so the first projection removes almost all of
// w and a selective test (norm drop below 1/sqrt(2)) asks for it every step.
// Every kernel returns at once when *skip is set (the cycle has converged).
#include <cuda_runtime.h>

#include <cstdint>

#include "pslr_reduce.cuh"

namespace pslr {

constexpr int kKThreads = 256;
constexpr int kChunk = 8;  // basis columns per register chunk
constexpr int kMaxK = 128; // basis columns of one CGS pass (Arnoldi rank <= 128, FGMRES restart + 1 <= 128)

__device__ __forceinline__ bool skipping(const int *skip) {
    return skip != nullptr && *(volatile const int *)skip != 0;
}

// Two-level deterministic reduction of the per-block partials (nres values
// each, part[b*nres + c]) into res: the last block of each group of kRedGroup
// consecutive blocks adds its group's partials in block order (into the
// group partials after the block partials), and the last group to finish adds
// the group partials in group order.  On GB300 a dependent FP64 add costs a
// full pass through the FP64 pipe, so the short chains (16 + groups instead of
// one add per block) matter.  ticket[0] counts finished groups, ticket[1 + g]
// the finished blocks of group g; the finishers reset them.  Returns true in
// the block that wrote res.
constexpr int kRedGroup = 16;
constexpr int kMaxTickets = 64;  // 1 + groups: up to 1008 blocks

__device__ bool finish_reduction(double *part, int nres, double *res, unsigned *ticket, bool accumulate) {
    __shared__ unsigned last;
    const int nb = gridDim.x, ng = (nb + kRedGroup - 1) / kRedGroup;
    const int g = blockIdx.x / kRedGroup, gb = g * kRedGroup, ge = min(nb, gb + kRedGroup);
    double *gpart = part + (int64_t)nb * nres;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket + 1 + g, 1u) == (unsigned)(ge - gb - 1);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int c = threadIdx.x; c < nres; c += blockDim.x) {
        double v = 0.0;
        for (int b = gb; b < ge; ++b) v += __ldcg(part + (int64_t)b * nres + c);
        gpart[(int64_t)g * nres + c] = v;
    }
    if (threadIdx.x == 0) ticket[1 + g] = 0u;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == (unsigned)(ng - 1);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int c = threadIdx.x; c < nres; c += blockDim.x) {
        double v = 0.0;
        for (int q = 0; q < ng; ++q) v += __ldcg(gpart + (int64_t)q * nres + c);
        res[c] = accumulate ? res[c] + v : v;
    }
    if (threadIdx.x == 0) ticket[0] = 0u;
    __syncthreads();
    return true;
}

// Block sum of one value per thread; thread 0 gets it.
__device__ __forceinline__ double block_reduce1(double v, double *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double a = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; ++w) a += sh[w];
    return a;
}

// Column sums a[u] += sum_i V[c0 + u, i] w[i], u < U, over the rows sb + lane,
// sb + lane + 32, ... < se.  U is the chunk's width as a compile-time
// constant: on GB300 an FP64 instruction holds the FP64 unit for its full
// time even when predicated off, so a chunk narrower than eight columns must
// not issue the other FMAs.
template <int U>
__device__ __forceinline__ void chunk_dots(double (&a)[kChunk], const double *__restrict__ V, int64_t ld, int c0,
                                           int sb, int se, int lane, const double *__restrict__ w) {
#pragma unroll 4
    for (int i = sb + lane; i < se; i += 32) {
        const double wi = w[i];
#pragma unroll
        for (int u = 0; u < U; ++u) a[u] = fma(V[(int64_t)(c0 + u) * ld + i], wi, a[u]);
    }
}

// One CGS pass.  If rp != nullptr: w = A z first (CSR, FP64).  If hsub !=
// nullptr: w -= V(:, 0:k) hsub.  Then either h = V(:, 0:k)^T w (norm == 0) or
// res[0] = ||w||^2 (norm != 0).
//
// Block b owns the contiguous rows [b R, (b+1) R).  The row-wise parts (SpMV,
// update, norm) take one thread per row.  The dot products run column-wise:
// a warp takes a chunk of eight columns and a subset of the block's rows,
// lanes stride over the rows (coalesced loads of V and w), and one butterfly
// reduction per chunk leaves eight column sums.  Reducing per thread instead
// (each thread a few rows, then eight shuffle trees per chunk) spent more
// FP64 instructions on the trees than on the products themselves, and FP64
// instructions are what this pass is bound by on GB300.
__global__ void __launch_bounds__(kKThreads) k_cgs_pass(
    int n, int k, const double *__restrict__ V, int64_t ld, double *__restrict__ w,
    const double *__restrict__ hsub, int norm, double *part, double *res, unsigned *ticket,
    const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ av,
    const double *__restrict__ z, const int *skip) {
    if (skipping(skip)) return;
    __shared__ double sh[(kKThreads / 32) * kMaxK];  // [row subset][column] partial sums
    __shared__ double hs[kMaxK];
    const int R = (n + gridDim.x - 1) / gridDim.x;
    const int rb = min(n, blockIdx.x * R), re = min(n, rb + R);
    if (hsub) {
        for (int c = threadIdx.x; c < k; c += blockDim.x) hs[c] = __ldcg(hsub + c);
        __syncthreads();
    }
    if (rp || hsub) {
        for (int i = rb + threadIdx.x; i < re; i += blockDim.x) {
            double wi;
            if (rp) {
                wi = 0.0;
                for (int e = rp[i]; e < rp[i + 1]; ++e) wi = fma(av[e], z[ci[e]], wi);
            } else {
                wi = w[i];
            }
            if (hsub)
                for (int c = 0; c < k; ++c) wi = fma(-V[(int64_t)c * ld + i], hs[c], wi);
            w[i] = wi;
        }
    }
    const int nres = norm ? 1 : k;
    if (norm) {
        double a = 0.0;
        for (int i = rb + threadIdx.x; i < re; i += blockDim.x) a = fma(w[i], w[i], a);
        a = block_reduce1(a, sh);
        if (threadIdx.x == 0) part[blockIdx.x] = a;
    } else {
        __syncthreads();  // the block's rows of w are written
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        const int nch = (k + kChunk - 1) / kChunk;
        const int nsub = nw / nch > 1 ? nw / nch : 1;
        const int rs = (re - rb + nsub - 1) / nsub;
        for (int t = warp; t < nch * nsub; t += nw) {
            const int c0 = (t % nch) * kChunk, sub = t / nch;
            const int sb = rb + sub * rs, se = min(re, sb + rs);
            double a[kChunk];
#pragma unroll
            for (int u = 0; u < kChunk; ++u) a[u] = 0.0;
            switch (min(kChunk, k - c0)) {  // the chunk's own width: no predicated-off FMAs
            case 8: chunk_dots<8>(a, V, ld, c0, sb, se, lane, w); break;
            case 7: chunk_dots<7>(a, V, ld, c0, sb, se, lane, w); break;
            case 6: chunk_dots<6>(a, V, ld, c0, sb, se, lane, w); break;
            case 5: chunk_dots<5>(a, V, ld, c0, sb, se, lane, w); break;
            case 4: chunk_dots<4>(a, V, ld, c0, sb, se, lane, w); break;
            case 3: chunk_dots<3>(a, V, ld, c0, sb, se, lane, w); break;
            case 2: chunk_dots<2>(a, V, ld, c0, sb, se, lane, w); break;
            default: chunk_dots<1>(a, V, ld, c0, sb, se, lane, w); break;
            }
            const double v = warp_reduce8(a);
            if ((lane & 3) == 0 && c0 + (lane >> 2) < k) sh[sub * kMaxK + c0 + (lane >> 2)] = v;
        }
        __syncthreads();
        for (int c = threadIdx.x; c < k; c += blockDim.x) {
            double v = 0.0;
            for (int u = 0; u < nsub; ++u) v += sh[u * kMaxK + c];
            part[(int64_t)blockIdx.x * nres + c] = v;
        }
    }
    finish_reduction(part, nres, res, ticket, false);
}

// Column j of the Hessenberg matrix from h1 + h2 and ||w||^2, and the FGMRES
// least-squares update with Givens rotations; the cycle stops once
// |gam(j+1)| <= *tol_abs (device memory, so a captured cycle serves every
// tolerance).
// H is (ldh x *) column-major; rot = [cs(0:ldh), sn(0:ldh)]; gam (ldh).
// state: [0] = iterations done in this cycle, [1] = converged/stop flag.
// One warp: the column and the rotations are staged in shared memory (c,
// scs, ssn), so the sequential rotation chain runs on shared-memory and
// register latency.
__device__ void hess_column(int j, const double *h1, const double *h2, const double *wn2, double *H, int ldh,
                            double *rot, double *gam, const double *tol_abs, int *state, int *skip, double *c,
                            double *scs, double *ssn) {
    const int lane = threadIdx.x & 31;
    double *col = H + (int64_t)j * ldh;
    double *cs = rot, *sn = rot + ldh;
    const double hn = sqrt(*wn2);
    for (int i = lane; i <= j; i += 32) c[i] = h1[i] + h2[i];
    for (int i = lane; i < j; i += 32) {
        scs[i] = cs[i];
        ssn[i] = sn[i];
    }
    __syncwarp();
    if (lane == 0) {
        c[j + 1] = hn;
        state[0] = j + 1;
        {
            double carry = c[0];  // entry i after the rotations before i
            for (int i = 0; i < j; ++i) {
                const double a = carry, b = c[i + 1], ci = scs[i], si = ssn[i];
                c[i] = ci * a + si * b;
                carry = -si * a + ci * b;
            }
            const double a = carry, b = c[j + 1];
            const double den = sqrt(a * a + b * b);
            const double cj = den > 0.0 ? a / den : 1.0, sj = den > 0.0 ? b / den : 0.0;
            cs[j] = cj;
            sn[j] = sj;
            c[j] = den;
            c[j + 1] = 0.0;
            const double g = gam[j];
            gam[j + 1] = -sj * g;
            gam[j] = cj * g;
            if (fabs(gam[j + 1]) <= *tol_abs || hn == 0.0 || !(den == den)) {
                state[1] = 1;
                if (skip) *skip = 1;
            }
        }
    }
    __syncwarp();
    for (int i = lane; i <= j + 1; i += 32) col[i] = c[i];
}

// The FGMRES step's last launch: v = w / ||w|| in blocks 0 .. gridDim.x-2
// (each block takes ||w|| from ||w||^2 itself, as hess_column does, so the
// results are those of the separate kernels), while one warp of the last
// block forms the Hessenberg column and applies the rotations.  If that stops
// the cycle, v is not used, so normalising blocks that start later may skip.
__global__ void k_hess_normalize(int j, const double *h1, const double *h2, const double *wn2, double *H,
                                 int ldh, double *rot, double *gam, const double *tol_abs, int *state,
                                 int *skip, int n, const double *w, double *v) {
    __shared__ double c[kMaxK + 2], scs[kMaxK + 1], ssn[kMaxK + 1];
    if (skipping(skip)) return;
    const int nb = gridDim.x - 1;
    if ((int)blockIdx.x == nb) {
        if (threadIdx.x < 32) hess_column(j, h1, h2, wn2, H, ldh, rot, gam, tol_abs, state, skip, c, scs, ssn);
        return;
    }
    const double h = sqrt(*wn2);
    const double s = h > 0.0 ? 1.0 / h : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nb * blockDim.x) v[i] = w[i] * s;
}

// v = w / *hn  (hn == 0 leaves v = 0).
__global__ void k_normalize(int n, const double *w, double *v, const double *hn, const int *skip) {
    if (skipping(skip)) return;
    const double h = *hn;
    const double s = h > 0.0 ? 1.0 / h : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        v[i] = w[i] * s;
}

// y += a x.
__global__ void k_axpy(int n, double a, const double *x, double *y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = fma(a, x[i], y[i]);
}

// x += Z(:, 0:k) y  (y on the device).
__global__ void k_gemv_add(int n, int k, const double *Z, int64_t ld, const double *y, double *x) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double a = x[i];
        for (int c = 0; c < k; ++c) a = fma(Z[(int64_t)c * ld + i], y[c], a);
        x[i] = a;
    }
}

// r = b - A x (CSR).  (A x with b == nullptr: r = A x.)
__global__ void k_residual(int n, const int32_t *rp, const int32_t *ci, const double *av,
                           const double *x, const double *b, double *r) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) a = fma(av[e], x[ci[e]], a);
        r[i] = b ? b[i] - a : a;
    }
}

// SplitMix64 (Steele, Lea, Flood 2014), output j of the generator seeded with
// seed, mapped to [-1, 1) from its top 53 bits: the Arnoldi start vector.
__global__ void k_splitmix(int n, uint64_t seed, uint64_t j0, double *v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint64_t x = seed + (j0 + (uint64_t)i + 1ull) * 0x9E3779B97F4A7C15ull;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        x = x ^ (x >> 31);
        v[i] = (double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    }
}

// Gradient of a loss with respect to the stored values of A for A u = b:
// dL/da_ij = -lambda_i u_j on A's pattern (lambda = A^{-T} dL/du).
__global__ void k_grad_values(int n, const int32_t *rp, const int32_t *ci, const double *lambda,
                              const double *u, double *g) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double li = lambda[i];
        for (int e = rp[i]; e < rp[i + 1]; ++e) g[e] = -li * u[ci[e]];
    }
}

// ---------------------------------------------------------------- launchers

// Blocks of the Krylov kernels: one row per thread, at most three blocks per
// SM (so large vectors spread evenly over every SM's FP64 pipe, with enough
// warps to cover the loads of V), and within the reduction's ticket array.
// (64^3 FGMRES(120) with the column-wise dot products: 3 blocks per SM
// 442 ms, 4 per SM 443 ms, 2 per SM 454 ms, 256 blocks 460 ms.)
int krylov_blocks(int n) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int want = (n + kKThreads - 1) / kKThreads;
    int cap = 3 * nsm;
    if (cap > (kMaxTickets - 1) * kRedGroup) cap = (kMaxTickets - 1) * kRedGroup;
    if (want > cap) want = cap;
    return want < 1 ? 1 : want;
}

// Sizes of the reduction buffers for up to `nres` results per block.
size_t krylov_part_doubles(int nblk, int nres) {
    return (size_t)(nblk + (nblk + kRedGroup - 1) / kRedGroup) * nres;
}
int krylov_tickets() { return kMaxTickets; }

void launch_cgs_pass(int n, int k, const double *V, int64_t ld, double *w, const double *hsub,
                     int norm, double *part, double *res, unsigned *ticket, const int32_t *rp,
                     const int32_t *ci, const double *av, const double *z, const int *skip,
                     cudaStream_t st) {
    k_cgs_pass<<<krylov_blocks(n), kKThreads, 0, st>>>(n, k, V, ld, w, hsub, norm, part, res, ticket,
                                                       rp, ci, av, z, skip);
}

void launch_hess_normalize(int j, const double *h1, const double *h2, const double *wn2, double *H, int ldh,
                           double *rot, double *gam, const double *tol_abs, int *state, int *skip, int n,
                           const double *w, double *v, cudaStream_t st) {
    k_hess_normalize<<<krylov_blocks(n) + 1, kKThreads, 0, st>>>(j, h1, h2, wn2, H, ldh, rot, gam, tol_abs,
                                                                 state, skip, n, w, v);
}

void launch_normalize(int n, const double *w, double *v, const double *hn, const int *skip,
                      cudaStream_t st) {
    k_normalize<<<krylov_blocks(n), kKThreads, 0, st>>>(n, w, v, hn, skip);
}

void launch_axpy(int n, double a, const double *x, double *y, cudaStream_t st) {
    k_axpy<<<krylov_blocks(n), kKThreads, 0, st>>>(n, a, x, y);
}

void launch_gemv_add(int n, int k, const double *Z, int64_t ld, const double *y, double *x,
                     cudaStream_t st) {
    k_gemv_add<<<krylov_blocks(n), kKThreads, 0, st>>>(n, k, Z, ld, y, x);
}

void launch_residual(int n, const int32_t *rp, const int32_t *ci, const double *av, const double *x,
                     const double *b, double *r, cudaStream_t st) {
    k_residual<<<krylov_blocks(n), kKThreads, 0, st>>>(n, rp, ci, av, x, b, r);
}

void launch_grad_values(int n, const int32_t *rp, const int32_t *ci, const double *lambda, const double *u,
                        double *g, cudaStream_t st) {
    k_grad_values<<<krylov_blocks(n), kKThreads, 0, st>>>(n, rp, ci, lambda, u, g);
}

void launch_splitmix(int n, uint64_t seed, uint64_t j0, double *v, cudaStream_t st) {
    k_splitmix<<<krylov_blocks(n), kKThreads, 0, st>>>(n, seed, j0, v);
}

}  // namespace pslr
