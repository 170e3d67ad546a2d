// Batched FP64 FGMRES kernels (Section 4) for many independent problems at
// once: every (system, right-hand side) pair of a batch runs its own FGMRES
// with its own basis, Hessenberg matrix, Givens rotations and stopping test,
// while each kernel launch serves all of them.
//
// The batched vector is the concatenation of the problems (system-major,
// right-hand side minor), cut into chunks of at most kBkChunk rows that never
// straddle two problems; one CTA per chunk.  CGS2 is three launches, as in the
// single-system FGMRES: (1) w = A z_j and per-chunk partials of V^T w;
// (2) h1 = sum of the partials (in chunk order, so deterministic), w -= V h1,
// partials of V^T w; (3) h2 likewise, w -= V h2, partials of ||w||^2.  One
// thread per problem then forms the Hessenberg column, applies the rotations
// and takes the stopping decision; a last launch writes v_{j+1} = w / h_{j+1,j}.
// The cycle end (least squares, x += Z y, true residual, restart) is also on
// the device, so one restart cycle needs no host round trip and can be
// replayed as one CUDA graph.  A problem that has stopped makes every later
// launch of the cycle return at once for its chunks, and a system whose
// problems have all stopped drops out of the batched apply (sys_active).
#include <cuda_runtime.h>

#include <cstdint>

#include "pslr_internal.h"
#include "pslr_reduce.cuh"

namespace pslr {

constexpr int kBkThreads = 256;
constexpr int kBkCols = 8;      // basis columns per register block
constexpr int kBkMaxK = 128;    // restart length + 1 at most

// a[u] += sum_i V[c0 + u, i] w[i] for u < U over rows sb + lane, sb + lane +
// 32, ... < se, U a compile-time width (an FP64 FMA that is predicated off
// still takes the FP64 unit's time on GB300).
template <int U>
__device__ __forceinline__ void bk_chunk_dots(double (&a)[kBkCols], const double *__restrict__ V, int64_t ldv, int c0,
                                              int64_t sb, int64_t se, int lane, const double *__restrict__ w) {
#pragma unroll 4
    for (int64_t i = sb + lane; i < se; i += 32) {
        const double wi = w[i];
#pragma unroll
        for (int u = 0; u < U; ++u) a[u] = fma(V[(int64_t)(c0 + u) * ldv + i], wi, a[u]);
    }
}

// part[blk * ldp + t] = V(:, t)^T w over the chunk [b, e), t = 0..k-1.  The
// rows of w were written by this block just before.  Column-wise: a warp
// takes a chunk of eight columns and a subset of the rows, lanes stride over
// the rows, one butterfly reduction per chunk (as in the single-system CGS
// pass: a per-thread reduction spends more FP64 instructions on the shuffle
// trees than on the products); subsets are added in a fixed order.
__device__ void bk_dots(int k, const double *__restrict__ V, int64_t ldv, const double *__restrict__ w,
                        int64_t b, int64_t e, double *part, int ldp) {
    __shared__ double sh[(kBkThreads / 32) * kBkMaxK];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kBkThreads / 32;
    const int nch = (k + kBkCols - 1) / kBkCols;
    const int nsub = nw / nch > 1 ? nw / nch : 1;
    const int64_t rs = (e - b + nsub - 1) / nsub;
    for (int t = warp; t < nch * nsub; t += nw) {
        const int c0 = (t % nch) * kBkCols, sub = t / nch;
        const int64_t sb = b + sub * rs, se = sb + rs < e ? sb + rs : e;
        double a[kBkCols];
#pragma unroll
        for (int u = 0; u < kBkCols; ++u) a[u] = 0.0;
        switch (min(kBkCols, k - c0)) {  // the chunk's own width: no predicated-off FMAs
        case 8: bk_chunk_dots<8>(a, V, ldv, c0, sb, se, lane, w); break;
        case 7: bk_chunk_dots<7>(a, V, ldv, c0, sb, se, lane, w); break;
        case 6: bk_chunk_dots<6>(a, V, ldv, c0, sb, se, lane, w); break;
        case 5: bk_chunk_dots<5>(a, V, ldv, c0, sb, se, lane, w); break;
        case 4: bk_chunk_dots<4>(a, V, ldv, c0, sb, se, lane, w); break;
        case 3: bk_chunk_dots<3>(a, V, ldv, c0, sb, se, lane, w); break;
        case 2: bk_chunk_dots<2>(a, V, ldv, c0, sb, se, lane, w); break;
        default: bk_chunk_dots<1>(a, V, ldv, c0, sb, se, lane, w); break;
        }
        const double v = warp_reduce8(a);
        if ((lane & 3) == 0 && c0 + (lane >> 2) < k) sh[sub * kBkMaxK + c0 + (lane >> 2)] = v;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += kBkThreads) {
        double v = 0.0;
        for (int u = 0; u < nsub; ++u) v += sh[u * kBkMaxK + c];
        part[(int64_t)blockIdx.x * ldp + c] = v;
    }
}

// part[blk * ld] = ||w||^2 over the chunk (rows this thread wrote).
__device__ void bk_norm2(const double *__restrict__ w, int64_t b, int64_t e, double *part, int ldp) {
    __shared__ double sh[kBkThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double a = 0.0;
    for (int64_t i = b + threadIdx.x; i < e; i += kBkThreads) a = fma(w[i], w[i], a);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) sh[warp] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int u = 0; u < kBkThreads / 32; ++u) v += sh[u];
        part[(int64_t)blockIdx.x * ldp] = v;
    }
}

// CGS2 pass 1: w = A z_j on the chunk's rows, then partials of V(:, 0:j+1)^T w.
__global__ void __launch_bounds__(kBkThreads) kb_spmv_dots(int j, const BkChunk *__restrict__ chunks,
                                                           const BkProb *__restrict__ probs,
                                                           const BkSys *__restrict__ sys,
                                                           const double *__restrict__ z, double *__restrict__ w,
                                                           const double *__restrict__ V, int64_t ld, BkState S) {
    const BkChunk ch = chunks[blockIdx.x];
    if (S.stop[ch.prob]) return;
    const BkProb pr = probs[ch.prob];
    const BkSys A = sys[pr.sys];
    const double *zp = z + pr.off;
    for (int64_t i = ch.b + threadIdx.x; i < ch.e; i += kBkThreads) {
        const int li = (int)(i - pr.off);
        double a = 0.0;
        for (int e = A.rp[li]; e < A.rp[li + 1]; ++e) a = fma(A.av[e], zp[A.ci[e]], a);
        w[i] = a;
    }
    bk_dots(j + 1, V, ld, w, ch.b, ch.e, S.pa, S.K + 1);
}

// CGS2 passes 2 and 3: h = sum over the problem's chunks of pin (chunk
// order); the problem's first chunk stores h in hout; w -= V(:, 0:j+1) h on
// the chunk; then partials of V^T w into pout (last == 0) or of ||w||^2 (last != 0).
__global__ void __launch_bounds__(kBkThreads) kb_update(int j, const BkChunk *__restrict__ chunks,
                                                        const BkProb *__restrict__ probs, double *__restrict__ w,
                                                        const double *__restrict__ V, int64_t ld,
                                                        const double *pin, double *pout, double *hout, int last,
                                                        BkState S) {
    __shared__ double hs[kBkMaxK];
    const BkChunk ch = chunks[blockIdx.x];
    if (S.stop[ch.prob]) return;
    const BkProb pr = probs[ch.prob];
    const int ldp = S.K + 1, k = j + 1;
    for (int t = threadIdx.x; t < k; t += kBkThreads) {
        double h = 0.0;
        for (int c = pr.c0; c < pr.c0 + pr.nc; ++c) h += pin[(int64_t)c * ldp + t];
        hs[t] = h;
        if ((int)blockIdx.x == pr.c0) hout[(int64_t)ch.prob * ldp + t] = h;
    }
    __syncthreads();
    for (int64_t i = ch.b + threadIdx.x; i < ch.e; i += kBkThreads) {
        double wi = w[i];
        for (int t = 0; t < k; ++t) wi = fma(-V[(int64_t)t * ld + i], hs[t], wi);
        w[i] = wi;
    }
    if (last) bk_norm2(w, ch.b, ch.e, pout, ldp);
    else bk_dots(k, V, ld, w, ch.b, ch.e, pout, ldp);
}

// sys_active[k] = some problem of system k still runs (after stop[] changed;
// one block, called after a __syncthreads).
__device__ void bk_sys_active(const BkState &S) {
    for (int k = threadIdx.x; k < S.nsys; k += blockDim.x) {
        int a = 0;
        for (int j = 0; j < S.nrhs; ++j) a |= S.stop[k * S.nrhs + j] == 0;
        S.sys_active[k] = a;
    }
}

// One thread per problem: Hessenberg column j = h1 + h2 with h_{j+1,j} = ||w||,
// the Givens rotations of the least-squares problem, and the stopping test
// (estimated residual |gamma_{j+1}| <= rtol ||b||, breakdown, iteration
// limit, end of the cycle).  *skip is set once no problem runs.
__global__ void kb_hessenberg(int j, int nprob, const BkProb *__restrict__ probs, BkState S) {
    __shared__ int active;
    if (threadIdx.x == 0) active = 0;
    __syncthreads();
    const int K = S.K, ldp = K + 1;
    int mine = 0;
    for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
        if (S.stop[p]) continue;
        const BkProb pr = probs[p];
        double wn2 = 0.0;
        for (int c = pr.c0; c < pr.c0 + pr.nc; ++c) wn2 += S.pa[(int64_t)c * ldp];
        double *col = S.H + ((int64_t)p * K + j) * ldp;
        const double *h1 = S.h1 + (int64_t)p * ldp, *h2 = S.h2 + (int64_t)p * ldp;
        for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
        const double hn = sqrt(wn2);
        col[j + 1] = hn;
        S.hn[p] = hn;
        S.jd[p] = j + 1;
        double *cs = S.rot + (int64_t)p * 2 * K, *sn = cs + K, *gam = S.gam + (int64_t)p * ldp;
        for (int i = 0; i < j; ++i) {
            const double a = col[i], b = col[i + 1];
            col[i] = cs[i] * a + sn[i] * b;
            col[i + 1] = -sn[i] * a + cs[i] * b;
        }
        const double a = col[j], b = col[j + 1];
        const double den = sqrt(a * a + b * b);
        cs[j] = den > 0.0 ? a / den : 1.0;
        sn[j] = den > 0.0 ? b / den : 0.0;
        col[j] = den;
        col[j + 1] = 0.0;
        gam[j + 1] = -sn[j] * gam[j];
        gam[j] = cs[j] * gam[j];
        const bool stop = fabs(gam[j + 1]) <= *S.rtol * S.bn[p] || hn == 0.0 || !(den == den) ||
                          S.its[p] + j + 1 >= *S.maxit || j + 1 == K;
        if (stop) S.stop[p] = 1;
        else ++mine;
    }
    if (mine) atomicAdd(&active, mine);
    __syncthreads();
    if (threadIdx.x == 0) *S.skip = active == 0;
    bk_sys_active(S);
}

// v_{j+1} = w / h_{j+1,j} for the problems still running.
__global__ void __launch_bounds__(kBkThreads) kb_normalize(const BkChunk *__restrict__ chunks,
                                                           const double *__restrict__ w, double *__restrict__ v,
                                                           BkState S) {
    const BkChunk ch = chunks[blockIdx.x];
    if (S.stop[ch.prob]) return;
    const double h = S.hn[ch.prob];
    const double s = h > 0.0 ? 1.0 / h : 0.0;
    for (int64_t i = ch.b + threadIdx.x; i < ch.e; i += kBkThreads) v[i] = w[i] * s;
}

// One thread per problem: the cycle's least-squares solution, the triangular
// system H(0:jd, 0:jd) y = gamma(0:jd) left by the rotations.
__global__ void kb_lsq(int nprob, BkState S) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob || S.conv[p] != 0) return;
    const int K = S.K, ldp = K + 1, jd = S.jd[p];
    const double *H = S.H + (int64_t)p * K * ldp, *gam = S.gam + (int64_t)p * ldp;
    double *y = S.y + (int64_t)p * K;
    for (int i = jd - 1; i >= 0; --i) {
        double a = gam[i];
        for (int l = i + 1; l < jd; ++l) a -= H[(int64_t)l * ldp + i] * y[l];
        y[i] = a / H[(int64_t)i * ldp + i];
    }
}

// x += Z(:, 0:jd) y on the chunk (problems still running).
__global__ void __launch_bounds__(kBkThreads) kb_gemv_add(const BkChunk *__restrict__ chunks,
                                                          const double *__restrict__ Z, int64_t ld,
                                                          double *__restrict__ x, BkState S) {
    const BkChunk ch = chunks[blockIdx.x];
    if (S.conv[ch.prob] != 0) return;
    const int jd = S.jd[ch.prob];
    const double *y = S.y + (int64_t)ch.prob * S.K;
    for (int64_t i = ch.b + threadIdx.x; i < ch.e; i += kBkThreads) {
        double a = x[i];
        for (int t = 0; t < jd; ++t) a = fma(Z[(int64_t)t * ld + i], y[t], a);
        x[i] = a;
    }
}

// r = b - A x (x == nullptr: r = b) on the chunk, and the partials of ||r||^2.
__global__ void __launch_bounds__(kBkThreads) kb_residual(const BkChunk *__restrict__ chunks,
                                                          const BkProb *__restrict__ probs,
                                                          const BkSys *__restrict__ sys,
                                                          const double *__restrict__ x,
                                                          const double *__restrict__ b, double *__restrict__ r,
                                                          BkState S) {
    const BkChunk ch = chunks[blockIdx.x];
    if (S.conv[ch.prob] != 0) return;
    const BkProb pr = probs[ch.prob];
    const BkSys A = sys[pr.sys];
    for (int64_t i = ch.b + threadIdx.x; i < ch.e; i += kBkThreads) {
        double a = 0.0;
        if (x) {
            const int li = (int)(i - pr.off);
            const double *xp = x + pr.off;
            for (int e = A.rp[li]; e < A.rp[li + 1]; ++e) a = fma(A.av[e], xp[A.ci[e]], a);
        }
        r[i] = b[i] - a;
    }
    bk_norm2(r, ch.b, ch.e, S.pa, S.K + 1);
}

// One thread per problem, at the start of the solve (first != 0) and at the
// end of every cycle: ||r|| from the partials, the iteration count, the
// convergence decision, and the next cycle's start (gamma = ||r|| e_1).
__global__ void kb_restart(int first, int nprob, const BkProb *__restrict__ probs, BkState S) {
    __shared__ int running;
    if (threadIdx.x == 0) running = 0;
    __syncthreads();
    const int ldp = S.K + 1;
    int mine = 0;
    for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
        if (S.conv[p] != 0) continue;
        const BkProb pr = probs[p];
        double r2 = 0.0;
        for (int c = pr.c0; c < pr.c0 + pr.nc; ++c) r2 += S.pa[(int64_t)c * ldp];
        const double rn = sqrt(r2);
        if (first) {
            S.bn[p] = rn;
            S.its[p] = 0;
        } else {
            S.its[p] += S.jd[p];
        }
        const double bn = S.bn[p];
        int cv = 0;
        bool finite = rn == rn && rn <= 1.79e308;
        if (!first) {
            const double *y = S.y + (int64_t)p * S.K;
            for (int t = 0; t < S.jd[p]; ++t) finite = finite && (y[t] == y[t]) && fabs(y[t]) <= 1.79e308;
        }
        if (bn == 0.0) cv = 1;
        else if (!finite) cv = 3;
        else if (rn <= *S.rtol * bn) cv = 1;
        else if (S.its[p] >= *S.maxit) cv = 2;
        S.conv[p] = cv;
        S.relres[p] = bn > 0.0 ? rn / bn : 0.0;
        S.rn[p] = rn;
        S.jd[p] = 0;
        S.stop[p] = cv != 0;
        if (cv == 0) {
            S.gam[(int64_t)p * ldp] = rn;
            ++mine;
        }
    }
    if (mine) atomicAdd(&running, mine);
    __syncthreads();
    if (threadIdx.x == 0) {
        *S.remaining = running;
        *S.skip = running == 0;
    }
    bk_sys_active(S);
}

// v_0 = r / ||r|| for the problems still running.
__global__ void __launch_bounds__(kBkThreads) kb_start(const BkChunk *__restrict__ chunks,
                                                       const double *__restrict__ r, double *__restrict__ v,
                                                       BkState S) {
    const BkChunk ch = chunks[blockIdx.x];
    if (S.conv[ch.prob] != 0) return;
    const double s = 1.0 / S.rn[ch.prob];
    for (int64_t i = ch.b + threadIdx.x; i < ch.e; i += kBkThreads) v[i] = r[i] * s;
}

// ---------------------------------------------------------------- launchers

void bk_spmv_dots(int nchunk, int j, const BkChunk *ch, const BkProb *pr, const BkSys *sys, const double *z,
                  double *w, const double *V, int64_t ld, const BkState &S, cudaStream_t st) {
    kb_spmv_dots<<<nchunk, kBkThreads, 0, st>>>(j, ch, pr, sys, z, w, V, ld, S);
}
void bk_update(int nchunk, int j, const BkChunk *ch, const BkProb *pr, double *w, const double *V, int64_t ld,
               const double *pin, double *pout, double *hout, int last, const BkState &S, cudaStream_t st) {
    kb_update<<<nchunk, kBkThreads, 0, st>>>(j, ch, pr, w, V, ld, pin, pout, hout, last, S);
}
void bk_hessenberg(int j, int nprob, const BkProb *pr, const BkState &S, cudaStream_t st) {
    kb_hessenberg<<<1, 256, 0, st>>>(j, nprob, pr, S);
}
void bk_normalize(int nchunk, const BkChunk *ch, const double *w, double *v, const BkState &S, cudaStream_t st) {
    kb_normalize<<<nchunk, kBkThreads, 0, st>>>(ch, w, v, S);
}
void bk_lsq(int nprob, const BkState &S, cudaStream_t st) {
    kb_lsq<<<(nprob + 127) / 128, 128, 0, st>>>(nprob, S);
}
void bk_gemv_add(int nchunk, const BkChunk *ch, const double *Z, int64_t ld, double *x, const BkState &S,
                 cudaStream_t st) {
    kb_gemv_add<<<nchunk, kBkThreads, 0, st>>>(ch, Z, ld, x, S);
}
void bk_residual(int nchunk, const BkChunk *ch, const BkProb *pr, const BkSys *sys, const double *x,
                 const double *b, double *r, const BkState &S, cudaStream_t st) {
    kb_residual<<<nchunk, kBkThreads, 0, st>>>(ch, pr, sys, x, b, r, S);
}
void bk_restart(int first, int nprob, const BkProb *pr, const BkState &S, cudaStream_t st) {
    kb_restart<<<1, 256, 0, st>>>(first, nprob, pr, S);
}
void bk_start(int nchunk, const BkChunk *ch, const double *r, double *v, const BkState &S, cudaStream_t st) {
    kb_start<<<nchunk, kBkThreads, 0, st>>>(ch, r, v, S);
}

}  // namespace pslr
