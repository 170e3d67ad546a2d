// Persistent PSLR kernels for sm_103a.
//
// pslr_apply_kernel runs Algorithm 3 (Eq. 3.24) - and, with the transposed
// operator set, its exact transpose - in ONE cooperative launch.  One CTA owns
// one subdomain at a time (looping when there are more subdomains than
// resident CTAs); the subdomain's interior and interface vectors live in
// shared memory, and every sparse operand (the level segments of the local
// factors, E_i, F_i, C_g,i) is streamed into a shared-memory ring by TMA bulk
// copies issued a few segments ahead of use.  The only cross-subdomain
// couplings in the method are C_g (once per series term, Eq. 3.1) and the
// reduction V^T t of the low-rank term (Eq. 3.18); they are the only grid
// barriers, split into arrive/wait so local work overlaps the wait.
//
// pslr_err_kernel computes E_rr(m) v = (E_s C0^{-1})^{m+1} v (Eq. 3.19) for the
// Arnoldi process with the same machinery (m+1 grid barriers).
//
// Every wait (grid barrier, TMA completion) is bounded: when it gives up it
// latches PSLR_ERR_TIMEOUT, drains the copies it issued and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pslr_internal.h"

namespace pslr {

constexpr int kErrTimeout = 8;          // PSLR_ERR_TIMEOUT
constexpr long long kTmaWaitLimit = 1ll << 24;

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                              uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile(const int *p) { return *(volatile const int *)p; }

template <class T>
__device__ __forceinline__ T fma_t(T a, T b, T c) {
    return fma(a, b, c);
}

__device__ __forceinline__ double load_v(const double *V, int64_t i) { return V[i]; }
__device__ __forceinline__ float load_v(const __nv_bfloat16 *V, int64_t i) {
    return __bfloat162float(V[i]);
}

// ----------------------------------------------------- per-CTA shared state

template <class T>
struct Cta {
    char *ring;           // kRing slots
    uint32_t ring_s;      // shared address of slot 0
    uint32_t mbar_s;      // shared address of mbarrier 0
    SegDesc *desc;        // descriptor table of the current subdomain
    T *xi, *wi, *si, *tmp;
    T *red;               // reduction scratch
    int slot_bytes;
    const char *segbase;
    int cur_sub;          // subdomain whose descriptors are cached
    // segment program (thread 0 drives the producer side)
    int prog_b[8], prog_n[8], nprog, total;
    unsigned seq_base;    // ring sequence number of program segment 0
    int issued;           // program segments issued so far
    unsigned seq_issued;  // ring sequence numbers issued in total
    unsigned seq_done;    // ring sequence numbers consumed in total
    int failed;           // a wait gave up
    unsigned bar_gen;     // thread 0: generation seen at the last grid arrive
};

// Map program position k to its descriptor index in the cached table.
template <class T>
__device__ __forceinline__ int prog_desc(const Cta<T> &c, int k) {
    for (int i = 0; i < c.nprog; ++i) {
        if (k < c.prog_n[i]) return c.prog_b[i] + k;
        k -= c.prog_n[i];
    }
    return -1;
}

// Thread 0: issue program segment k into its ring slot.
template <class T>
__device__ __forceinline__ void issue_segment(Cta<T> &c, int k) {
    unsigned seq = c.seq_base + k;
    int slot = seq % kRing;
    uint32_t bar = c.mbar_s + 8 * slot;
    const SegDesc &d = c.desc[prog_desc(c, k)];
    if (d.bytes > 0) {
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, d.bytes);
        bulk_copy_g2s(c.ring_s + slot * c.slot_bytes, c.segbase + d.off, d.bytes, bar);
    } else {
        mbar_arrive(bar);
    }
    c.seq_issued = seq + 1;
}

// Start a program of descriptor ranges (all threads call; thread 0 issues).
template <class T>
__device__ void prog_start(Cta<T> &c, int nr, const int *b, const int *n) {
    __syncthreads();
    if (threadIdx.x == 0) {
        c.nprog = nr;
        c.total = 0;
        for (int i = 0; i < nr; ++i) {
            c.prog_b[i] = b[i];
            c.prog_n[i] = n[i];
            c.total += n[i];
        }
        c.seq_base = c.seq_issued;
        c.issued = 0;
        while (c.issued < c.total && c.issued < kRing) issue_segment(c, c.issued++);
    }
    __syncthreads();
}

// Wait until program segment k has landed; returns its shared-memory copy.
template <class T>
__device__ char *seg_acquire(Cta<T> &c, int k, int *err) {
    unsigned seq = c.seq_base + k;
    int slot = seq % kRing;
    uint32_t bar = c.mbar_s + 8 * slot;
    uint32_t parity = (seq / kRing) & 1u;
    long long it = 0;
    while (!mbar_try_wait(bar, parity)) {
        if (++it > kTmaWaitLimit) {
            atomicCAS(err, 0, kErrTimeout);
            break;
        }
    }
    return c.ring + slot * c.slot_bytes;
}

// Segment k fully consumed by every thread (caller synchronised): recycle slot.
template <class T>
__device__ __forceinline__ void seg_release(Cta<T> &c, int k) {
    if (threadIdx.x == 0) {
        c.seq_done = c.seq_base + k + 1;
        if (c.issued < c.total) issue_segment(c, c.issued++);
    }
}

// Before leaving the kernel: wait (bounded) for every copy still in flight.
template <class T>
__device__ void drain_ring(Cta<T> &c) {
    __syncthreads();
    if (threadIdx.x == 0) {
        for (unsigned seq = c.seq_done; seq < c.seq_issued; ++seq) {
            uint32_t bar = c.mbar_s + 8 * (seq % kRing);
            long long it = 0;
            while (!mbar_try_wait(bar, (seq / kRing) & 1u) && ++it < kTmaWaitLimit) {
            }
        }
        c.seq_done = c.seq_issued;
    }
    __syncthreads();
}

// ----------------------------------------------------------------- grid barrier

// Sense-reversing barrier over all CTAs of the cooperative grid.  arrive()
// publishes this CTA's writes; wait() returns once every CTA has arrived.
template <class T>
__device__ void grid_arrive(Cta<T> &c, unsigned *bar, int grid) {
    __syncthreads();
    if (threadIdx.x == 0) {
        c.bar_gen = ld_acquire(bar + 1);
        __threadfence();
        unsigned old = atomicAdd(bar, 1u);
        if (old == (unsigned)grid - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        }
    }
}

template <class T>
__device__ bool grid_wait(Cta<T> &c, unsigned *bar, int *err, long long limit) {
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        long long it = 0;
        while (ld_acquire(bar + 1) == c.bar_gen) {
            if (limit <= 0 || ++it > limit || ld_volatile(err) != 0) {
                atomicCAS(err, 0, kErrTimeout);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// -------------------------------------------------------------- local operators

// Segment field pointers.
template <class T, class IDX>
struct SegView {
    const T *vals, *dinv;
    const IDX *cols;
    const uint16_t *rows;
    int n, w, np;
};

template <class T, class IDX>
__device__ __forceinline__ SegView<T, IDX> seg_view(const char *seg, const SegDesc &d) {
    SegView<T, IDX> v;
    v.n = d.n;
    v.w = d.w;
    v.np = seg_npad(d.n);
    v.vals = reinterpret_cast<const T *>(seg);
    const char *p = seg + (size_t)v.np * v.w * sizeof(T);
    v.dinv = reinterpret_cast<const T *>(p);
    if (d.flags & kSegDiag) p += (size_t)v.np * sizeof(T);
    v.cols = reinterpret_cast<const IDX *>(p);
    p += (size_t)v.np * v.w * sizeof(IDX);
    v.rows = reinterpret_cast<const uint16_t *>(p);
    return v;
}

// One triangular sweep over `nlev` level segments starting at program
// position k0: x[r] = (x[r] - sum_k T_rk x[c_k]) (* dinv[r]), in place.
template <class T>
__device__ void tri_sweep(Cta<T> &c, T *x, int k0, int nlev, int *err) {
    for (int L = 0; L < nlev; ++L) {
        const SegDesc &d = c.desc[prog_desc(c, k0 + L)];
        const char *seg = seg_acquire(c, k0 + L, err);
        SegView<T, uint16_t> v = seg_view<T, uint16_t>(seg, d);
        const bool diag = (d.flags & kSegDiag) != 0;
        for (int j = threadIdx.x; j < v.n; j += blockDim.x) {
            int r = v.rows[j];
            T a = x[r];
            for (int k = 0; k < v.w; ++k) a = fma_t(-v.vals[k * v.np + j], x[v.cols[k * v.np + j]], a);
            if (diag) a *= v.dinv[j];
            x[r] = a;
        }
        __syncthreads();
        seg_release(c, k0 + L);
    }
}

// ELL product over nseg program segments from k0: out[row] = sum (assign) or
// out[row] -= sum (subtract), src in shared (local columns) or global memory.
template <class T, bool GLOBAL>
__device__ void ell_op(Cta<T> &c, T *out, const T *src, bool subtract, int k0, int nseg, int *err) {
    for (int k = k0; k < k0 + nseg; ++k) {
        const SegDesc &d = c.desc[prog_desc(c, k)];
        const char *seg = seg_acquire(c, k, err);
        if (GLOBAL) {
            SegView<T, int32_t> v = seg_view<T, int32_t>(seg, d);
            for (int j = threadIdx.x; j < v.n; j += blockDim.x) {
                T a = T(0);
                for (int kk = 0; kk < v.w; ++kk)
                    a = fma_t(v.vals[kk * v.np + j], __ldcg(src + v.cols[kk * v.np + j]), a);
                int r = v.rows[j];
                out[r] = subtract ? out[r] - a : a;
            }
        } else {
            SegView<T, uint16_t> v = seg_view<T, uint16_t>(seg, d);
            for (int j = threadIdx.x; j < v.n; j += blockDim.x) {
                T a = T(0);
                for (int kk = 0; kk < v.w; ++kk) a = fma_t(v.vals[kk * v.np + j], src[v.cols[kk * v.np + j]], a);
                int r = v.rows[j];
                out[r] = subtract ? out[r] - a : a;
            }
        }
        __syncthreads();
        seg_release(c, k);
    }
}

// Exact-LU row permutation: x <- P x (gather, before the sweeps) or
// x <- P^T x (scatter, after the transposed sweeps), via tmp.
template <class T>
__device__ void permute(T *x, T *tmp, const uint16_t *piv, int n, bool scatter) {
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) tmp[j] = x[j];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        if (scatter) x[piv[j]] = tmp[j];
        else x[j] = tmp[piv[j]];
    }
    __syncthreads();
}

// Local solve x <- B_i~^{-1} x (or its transpose) with the sweeps at k0.
template <class T>
__device__ void solve_local(Cta<T> &c, T *x, int n, const uint16_t *piv, int pivot_post, int k0,
                            int n1, int n2, int *err) {
    if (piv && !pivot_post) permute(x, c.tmp, piv, n, false);
    tri_sweep(c, x, k0, n1, err);
    tri_sweep(c, x, k0 + n1, n2, err);
    if (piv && pivot_post) permute(x, c.tmp, piv, n, true);
}

// Segment counts of subdomain i and their positions in its descriptor table.
struct SubOps {
    int n[kNCnt], pos[kNCnt], total;
};

__device__ __forceinline__ SubOps sub_ops(const OpSetDev &ops, int i) {
    SubOps o;
    int acc = 0;
#pragma unroll
    for (int t = 0; t < kNCnt; ++t) {
        o.n[t] = ops.cnt[kNCnt * i + t];
        o.pos[t] = acc;
        acc += o.n[t];
    }
    o.total = acc;
    return o;
}

// A program under construction: ranges of the descriptor table, in order.
struct ProgBuild {
    int b[8], n[8], k = 0, total = 0;
    __device__ int add(int pos, int cnt) {
        b[k] = pos;
        n[k] = cnt;
        ++k;
        int at = total;
        total += cnt;
        return at;
    }
};

// Cache subdomain i's descriptor table in shared memory.
template <class T>
__device__ void load_desc(Cta<T> &c, const OpSetDev &ops, int i, int nd) {
    if (c.cur_sub == i) return;
    __syncthreads();
    const int4 *src = reinterpret_cast<const int4 *>(ops.desc + ops.sub_desc[i]);
    int4 *dst = reinterpret_cast<int4 *>(c.desc);
    for (int j = threadIdx.x; j < nd; j += blockDim.x) dst[j] = src[j];
    __syncthreads();
    if (threadIdx.x == 0) c.cur_sub = i;
    __syncthreads();
}

template <class T>
__device__ void fill(T *x, int n, T v) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) x[j] = v;
}

// Partial dots part[i*r + c] = sum_j V[go + j, c] * y[j] over this subdomain,
// eight columns at a time so each thread has many independent loads in flight.
template <class T, class VT>
__device__ void lowrank_partial(Cta<T> &c, const VT *V, int q, int r, int go, int nq, const T *y,
                                T *part_i) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c0 = 0; c0 < r; c0 += 8) {
        T a[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = T(0);
        for (int j = threadIdx.x; j < nq; j += blockDim.x) {
            const T yj = y[j];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (c0 + k < r) a[k] = fma_t(T(load_v(V, (int64_t)(c0 + k) * q + go + j)), yj, a[k]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            T v = a[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && c0 + k < r) c.red[warp * kMaxRank + c0 + k] = v;
        }
    }
    __syncthreads();
    for (int col = threadIdx.x; col < r; col += blockDim.x) {
        T a = T(0);
        for (int w = 0; w < nw; ++w) a += c.red[w * kMaxRank + col];
        part_i[col] = a;
    }
    __syncthreads();
}

// d = G u with u = sum over subdomains of the partials, into the tail of
// c.red.  Threads split as (column, group of subdomains); the group sums are
// combined in a fixed order, so every CTA computes the same d.
template <class T>
__device__ void lowrank_coeffs(Cta<T> &c, const T *part, const T *G, int s, int r) {
    T *u = c.red + (kThreads / 32) * kMaxRank;
    T *d = u + kMaxRank;
    const int tpc = blockDim.x / r;  // groups per column (r <= kMaxRank <= blockDim)
    const int col = threadIdx.x % r, grp = threadIdx.x / r;
    if (grp < tpc) {
        T a = T(0);
#pragma unroll 4
        for (int i = grp; i < s; i += tpc) a += __ldcg(part + (int64_t)i * r + col);
        c.red[grp * r + col] = a;
    }
    __syncthreads();
    if (threadIdx.x < r) {
        T a = T(0);
        for (int g = 0; g < tpc; ++g) a += c.red[g * r + threadIdx.x];
        u[threadIdx.x] = a;
    }
    __syncthreads();
    for (int row = threadIdx.x; row < r; row += blockDim.x) {
        T a = T(0);
        for (int k = 0; k < r; ++k) a = fma_t(G[k * r + row], u[k], a);
        d[row] = a;
    }
    __syncthreads();
}

// y[j] += sum_c V[go + j, c] d[c]
template <class T, class VT>
__device__ void lowrank_update(Cta<T> &c, const VT *V, int q, int r, int go, int nq, T *y) {
    const T *d = c.red + (kThreads / 32) * kMaxRank + kMaxRank;
    for (int j = threadIdx.x; j < nq; j += blockDim.x) {
        T a = y[j];
        for (int col = 0; col < r; ++col) a = fma_t(T(load_v(V, (int64_t)col * q + go + j)), d[col], a);
        y[j] = a;
    }
    __syncthreads();
}

template <class T>
__device__ void cta_init(Cta<T> &c, char *smem, const SmemLayout &L, int slot_bytes,
                         const char *segbase) {
    c.ring = smem + L.ring;
    c.ring_s = smem_addr(c.ring);
    c.mbar_s = smem_addr(smem + L.mbar);
    c.desc = reinterpret_cast<SegDesc *>(smem + L.desc);
    c.xi = reinterpret_cast<T *>(smem + L.xi);
    c.wi = reinterpret_cast<T *>(smem + L.wi);
    c.si = reinterpret_cast<T *>(smem + L.si);
    c.tmp = reinterpret_cast<T *>(smem + L.tmp);
    c.red = reinterpret_cast<T *>(smem + L.red);
    c.slot_bytes = slot_bytes;
    c.segbase = segbase;
    __syncthreads();
    if (threadIdx.x == 0) {
        c.cur_sub = -1;
        c.seq_issued = 0;
        c.seq_done = 0;
        c.failed = 0;
        for (int i = 0; i < kRing; ++i) mbar_init(c.mbar_s + 8 * i, 1);
        fence_mbar_init();
    }
    __syncthreads();
}

// ------------------------------------------------------------------ the apply

template <class T, class VT>
__global__ void __launch_bounds__(kThreads, 1) pslr_apply_kernel(const ApplyParams<T> P) {
    extern __shared__ __align__(128) char smem[];
    __shared__ Cta<T> c;
    if (P.skip != nullptr && ld_volatile(P.skip) != 0) return;
    const bool pivots = P.bpiv != nullptr;
    const SmemLayout L = smem_layout(P.slot_bytes, P.max_desc, P.max_p, P.max_q, sizeof(T), pivots);
    cta_init(c, smem, L, P.slot_bytes, P.ops.segbase);
    if (ld_volatile(P.err) != 0) return;

    const OpSetDev &ops = P.ops;
    const VT *V = reinterpret_cast<const VT *>(P.V);
    const int q = P.q, p = P.p, r = P.r, m = P.m;
    const bool lr_before = r > 0 && !ops.lowrank_after;
    const bool lr_after = r > 0 && ops.lowrank_after;
    const T *w_cur;
    bool ok = true;

    // ---- phase 0: u = B^{-1} f, t = g - F u (Algorithm 3, step 2); without a
    // low-rank term before the series also w_0 = C0^{-1} t.
    for (int i = blockIdx.x; i < P.s; i += gridDim.x) {
        const SubOps so = sub_ops(ops, i);
        load_desc(c, ops, i, so.total);
        const int io = P.ioff[i], np_ = P.ioff[i + 1] - io;
        const int go = P.goff[i], nq = P.goff[i + 1] - go;
        ProgBuild pb;
        const int kB = pb.add(so.pos[kB1], so.n[kB1] + so.n[kB2]);
        const int kF_ = pb.add(so.pos[kF], so.n[kF]);
        const int kC = lr_before ? 0 : pb.add(so.pos[kC1], so.n[kC1] + so.n[kC2]);
        prog_start(c, pb.k, pb.b, pb.n);
        for (int j = threadIdx.x; j < np_; j += blockDim.x) c.xi[j] = P.b[P.perm[io + j]];
        if (threadIdx.x == 0) c.xi[np_] = T(0);
        for (int j = threadIdx.x; j < nq; j += blockDim.x) c.si[j] = P.b[P.perm[p + go + j]];
        __syncthreads();
        solve_local(c, c.xi, np_, pivots ? P.bpiv + io : nullptr, ops.pivot_post, kB, so.n[kB1],
                    so.n[kB2], P.err);
        ell_op<T, false>(c, c.si, c.xi, true, kF_, so.n[kF], P.err);
        if (lr_before) {
            lowrank_partial(c, V, q, r, go, nq, c.si, P.part + (int64_t)i * r);
            for (int j = threadIdx.x; j < nq; j += blockDim.x) P.acc[go + j] = c.si[j];
        } else {
            if (threadIdx.x == 0) c.si[nq] = T(0);
            solve_local(c, c.si, nq, pivots ? P.cpiv + go : nullptr, ops.pivot_post, kC, so.n[kC1],
                        so.n[kC2], P.err);
            for (int j = threadIdx.x; j < nq; j += blockDim.x) {
                P.wbuf[go + j] = c.si[j];
                P.acc[go + j] = c.si[j];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        P.wbuf[q] = T(0);
        P.wbuf[(q + 1) + q] = T(0);
    }

    // ---- phase 1: t <- t + V G V^T t, then w_0 = C0^{-1} t (steps 3-4)
    if (lr_before) {
        grid_arrive(c, P.bar, P.grid);
        ok = grid_wait(c, P.bar, P.err, P.wait_limit);
        if (!ok) goto out;
        lowrank_coeffs(c, P.part, P.G, P.s, r);
        for (int i = blockIdx.x; i < P.s; i += gridDim.x) {
            const SubOps so = sub_ops(ops, i);
            load_desc(c, ops, i, so.total);
            const int go = P.goff[i], nq = P.goff[i + 1] - go;
            ProgBuild pb;
            const int kC = pb.add(so.pos[kC1], so.n[kC1] + so.n[kC2]);
            prog_start(c, pb.k, pb.b, pb.n);
            for (int j = threadIdx.x; j < nq; j += blockDim.x) c.si[j] = __ldcg(P.acc + go + j);
            if (threadIdx.x == 0) c.si[nq] = T(0);
            __syncthreads();
            lowrank_update(c, V, q, r, go, nq, c.si);
            solve_local(c, c.si, nq, pivots ? P.cpiv + go : nullptr, ops.pivot_post, kC, so.n[kC1],
                        so.n[kC2], P.err);
            for (int j = threadIdx.x; j < nq; j += blockDim.x) {
                P.wbuf[go + j] = c.si[j];
                P.acc[go + j] = c.si[j];
            }
            __syncthreads();
        }
    }

    // ---- series terms w_k = C0^{-1}(F B^{-1} E w_{k-1} - C_g w_{k-1}), acc += w_k (Eq. 3.3)
    for (int k = 1; k <= m; ++k) {
        const T *wprev = P.wbuf + ((k - 1) & 1) * (q + 1);
        T *wnext = P.wbuf + (k & 1) * (q + 1);
        grid_arrive(c, P.bar, P.grid);
        bool waited = false;
        for (int i = blockIdx.x; i < P.s; i += gridDim.x) {
            const SubOps so = sub_ops(ops, i);
            load_desc(c, ops, i, so.total);
            const int io = P.ioff[i], np_ = P.ioff[i + 1] - io;
            const int go = P.goff[i], nq = P.goff[i + 1] - go;
            ProgBuild pb;
            const int kE_ = pb.add(so.pos[kE], so.n[kE]);
            const int kB = pb.add(so.pos[kB1], so.n[kB1] + so.n[kB2]);
            const int kF_ = pb.add(so.pos[kF], so.n[kF]);
            const int kG = pb.add(so.pos[kCg], so.n[kCg]);
            const int kC = pb.add(so.pos[kC1], so.n[kC1] + so.n[kC2]);
            prog_start(c, pb.k, pb.b, pb.n);
            for (int j = threadIdx.x; j < nq; j += blockDim.x) c.wi[j] = __ldcg(wprev + go + j);
            if (threadIdx.x == 0) c.wi[nq] = T(0);
            fill(c.xi, np_ + 1, T(0));
            __syncthreads();
            ell_op<T, false>(c, c.xi, c.wi, false, kE_, so.n[kE], P.err);             // E w
            solve_local(c, c.xi, np_, pivots ? P.bpiv + io : nullptr, ops.pivot_post, kB, so.n[kB1],
                        so.n[kB2], P.err);                                            // B^{-1}
            fill(c.si, nq + 1, T(0));
            __syncthreads();
            ell_op<T, false>(c, c.si, c.xi, false, kF_, so.n[kF], P.err);             // F
            if (!waited) {
                ok = grid_wait(c, P.bar, P.err, P.wait_limit);
                waited = true;
                if (!ok) goto out;
            }
            ell_op<T, true>(c, c.si, wprev, true, kG, so.n[kCg], P.err);              // - C_g w
            solve_local(c, c.si, nq, pivots ? P.cpiv + go : nullptr, ops.pivot_post, kC, so.n[kC1],
                        so.n[kC2], P.err);                                            // C0^{-1}
            for (int j = threadIdx.x; j < nq; j += blockDim.x) {
                wnext[go + j] = c.si[j];
                P.acc[go + j] = __ldcg(P.acc + go + j) + c.si[j];
            }
            __syncthreads();
        }
        if (!waited) {  // a CTA without subdomains still takes part in the barrier
            ok = grid_wait(c, P.bar, P.err, P.wait_limit);
            if (!ok) goto out;
        }
    }

    // ---- transposed order: w <- w + V G^T V^T w after the series
    if (lr_after) {
        for (int i = blockIdx.x; i < P.s; i += gridDim.x) {
            const int go = P.goff[i], nq = P.goff[i + 1] - go;
            for (int j = threadIdx.x; j < nq; j += blockDim.x) c.si[j] = __ldcg(P.acc + go + j);
            __syncthreads();
            lowrank_partial(c, V, q, r, go, nq, c.si, P.part + (int64_t)i * r);
        }
        grid_arrive(c, P.bar, P.grid);
        ok = grid_wait(c, P.bar, P.err, P.wait_limit);
        if (!ok) goto out;
        lowrank_coeffs(c, P.part, P.G, P.s, r);
    }

    // ---- y = acc; x = B^{-1}(f - E y); scatter (steps 5-6)
    w_cur = P.acc;
    for (int i = blockIdx.x; i < P.s; i += gridDim.x) {
        const SubOps so = sub_ops(ops, i);
        load_desc(c, ops, i, so.total);
        const int io = P.ioff[i], np_ = P.ioff[i + 1] - io;
        const int go = P.goff[i], nq = P.goff[i + 1] - go;
        ProgBuild pb;
        const int kE_ = pb.add(so.pos[kE], so.n[kE]);
        const int kB = pb.add(so.pos[kB1], so.n[kB1] + so.n[kB2]);
        prog_start(c, pb.k, pb.b, pb.n);
        for (int j = threadIdx.x; j < nq; j += blockDim.x) c.wi[j] = __ldcg(w_cur + go + j);
        if (threadIdx.x == 0) c.wi[nq] = T(0);
        for (int j = threadIdx.x; j < np_; j += blockDim.x) c.xi[j] = P.b[P.perm[io + j]];
        if (threadIdx.x == 0) c.xi[np_] = T(0);
        __syncthreads();
        if (lr_after) lowrank_update(c, V, q, r, go, nq, c.wi);
        ell_op<T, false>(c, c.xi, c.wi, true, kE_, so.n[kE], P.err);
        solve_local(c, c.xi, np_, pivots ? P.bpiv + io : nullptr, ops.pivot_post, kB, so.n[kB1],
                    so.n[kB2], P.err);
        for (int j = threadIdx.x; j < np_; j += blockDim.x) P.z[P.perm[io + j]] = c.xi[j];
        for (int j = threadIdx.x; j < nq; j += blockDim.x) P.z[P.perm[p + go + j]] = c.wi[j];
        __syncthreads();
    }
out:
    drain_ring(c);
}

// ------------------------------------------------------------ E_rr(m) matvec

template <class T>
__global__ void __launch_bounds__(kThreads, 1) pslr_err_kernel(const ErrParams<T> P) {
    extern __shared__ __align__(128) char smem[];
    __shared__ Cta<T> c;
    const bool pivots = P.bpiv != nullptr;
    const SmemLayout L = smem_layout(P.slot_bytes, P.max_desc, P.max_p, P.max_q, sizeof(T), pivots);
    cta_init(c, smem, L, P.slot_bytes, P.ops.segbase);
    if (ld_volatile(P.err) != 0) return;
    const OpSetDev &ops = P.ops;
    const int q = P.q;
    bool ok = true;
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        P.abuf[q] = T(0);
        P.abuf[(q + 1) + q] = T(0);
    }
    for (int rep = 0; rep <= P.m; ++rep) {
        T *a = P.abuf + (rep & 1) * (q + 1);
        const T *vsrc = rep == 0 ? P.vin : P.vout;
        // a_i = C0_i^{-1} v_i  (local)
        for (int i = blockIdx.x; i < P.s; i += gridDim.x) {
            const SubOps so = sub_ops(ops, i);
            load_desc(c, ops, i, so.total);
            const int go = P.goff[i], nq = P.goff[i + 1] - go;
            ProgBuild pb;
            const int kC = pb.add(so.pos[kC1], so.n[kC1] + so.n[kC2]);
            prog_start(c, pb.k, pb.b, pb.n);
            for (int j = threadIdx.x; j < nq; j += blockDim.x) c.si[j] = __ldcg(vsrc + go + j);
            if (threadIdx.x == 0) c.si[nq] = T(0);
            __syncthreads();
            solve_local(c, c.si, nq, pivots ? P.cpiv + go : nullptr, ops.pivot_post, kC, so.n[kC1],
                        so.n[kC2], P.err);
            for (int j = threadIdx.x; j < nq; j += blockDim.x) a[go + j] = c.si[j];
            __syncthreads();
        }
        grid_arrive(c, P.bar, P.grid);
        bool waited = false;
        // v_i = F_i B_i^{-1} E_i a_i - (C_g a)_i
        for (int i = blockIdx.x; i < P.s; i += gridDim.x) {
            const SubOps so = sub_ops(ops, i);
            load_desc(c, ops, i, so.total);
            const int io = P.ioff[i], np_ = P.ioff[i + 1] - io;
            const int go = P.goff[i], nq = P.goff[i + 1] - go;
            ProgBuild pb;
            const int kE_ = pb.add(so.pos[kE], so.n[kE]);
            const int kB = pb.add(so.pos[kB1], so.n[kB1] + so.n[kB2]);
            const int kF_ = pb.add(so.pos[kF], so.n[kF]);
            const int kG = pb.add(so.pos[kCg], so.n[kCg]);
            prog_start(c, pb.k, pb.b, pb.n);
            for (int j = threadIdx.x; j < nq; j += blockDim.x) c.wi[j] = __ldcg(a + go + j);
            if (threadIdx.x == 0) c.wi[nq] = T(0);
            fill(c.xi, np_ + 1, T(0));
            __syncthreads();
            ell_op<T, false>(c, c.xi, c.wi, false, kE_, so.n[kE], P.err);
            solve_local(c, c.xi, np_, pivots ? P.bpiv + io : nullptr, ops.pivot_post, kB, so.n[kB1],
                        so.n[kB2], P.err);
            fill(c.si, nq + 1, T(0));
            __syncthreads();
            ell_op<T, false>(c, c.si, c.xi, false, kF_, so.n[kF], P.err);
            if (!waited) {
                ok = grid_wait(c, P.bar, P.err, P.wait_limit);
                waited = true;
                if (!ok) goto out;
            }
            ell_op<T, true>(c, c.si, a, true, kG, so.n[kCg], P.err);
            for (int j = threadIdx.x; j < nq; j += blockDim.x) P.vout[go + j] = c.si[j];
            __syncthreads();
        }
        if (!waited) {
            ok = grid_wait(c, P.bar, P.err, P.wait_limit);
            if (!ok) goto out;
        }
    }
out:
    drain_ring(c);
}

// ------------------------------------------------------------- host launchers

template <class T, class VT>
cudaError_t launch_apply_t(const ApplyParams<T> &P, int smem_bytes, cudaStream_t st) {
    auto kern = pslr_apply_kernel<T, VT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<ApplyParams<T> *>(&P)};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(P.grid), dim3(kThreads), args,
                                       smem_bytes, st);
}

cudaError_t launch_apply_fp64(const ApplyParams<double> &P, int smem, cudaStream_t st) {
    return launch_apply_t<double, double>(P, smem, st);
}
cudaError_t launch_apply_fp32(const ApplyParams<float> &P, int smem, cudaStream_t st) {
    return launch_apply_t<float, __nv_bfloat16>(P, smem, st);
}

cudaError_t launch_err_fp64(const ErrParams<double> &P, int smem, cudaStream_t st) {
    auto kern = pslr_err_kernel<double>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<ErrParams<double> *>(&P)};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(P.grid), dim3(kThreads), args, smem, st);
}

// Largest cooperative grid of the persistent kernels for a dynamic smem size.
int max_coresident_apply(int smem, bool fp32) {
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e;
    if (fp32) {
        e = cudaFuncSetAttribute(pslr_apply_kernel<float, __nv_bfloat16>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pslr_apply_kernel<float, __nv_bfloat16>,
                                                              kThreads, smem);
    } else {
        e = cudaFuncSetAttribute(pslr_apply_kernel<double, double>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pslr_apply_kernel<double, double>,
                                                              kThreads, smem);
    }
    if (e != cudaSuccess) return 0;
    return per * nsm;
}

}  // namespace pslr
