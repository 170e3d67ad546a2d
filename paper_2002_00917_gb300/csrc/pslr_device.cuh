// Device building blocks shared by the persistent kernels (pslr_apply.cu,
// pslr_batch.cuh): PTX wrappers (mbarrier, cp.async.bulk, named barriers,
// explicit shared-memory accesses), the producer warp that streams segments
// into the shared-memory ring, the consumers' ring cursor and waits, the
// sense-reversing grid barrier, the level-sweep and ELL kernels-within-a-
// kernel, and the low-rank reductions.  Included once per translation unit.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "pslr_internal.h"
#include "pslr_reduce.cuh"

namespace pslr {

constexpr int kErrTimeout = 8;  // PSLR_ERR_TIMEOUT
constexpr long long kTmaWaitLimit = 1ll << 26;
constexpr int kProducerWarp = kConsumers / 32;
// A ring slot is free again once every consumer warp has arrived on its empty
// barrier: a level sweep (which synchronises the CTA per level anyway) arrives
// once for all warps; the products E, F, C_g, whose segments write disjoint
// rows, let every warp arrive on its own and move on without a CTA barrier.
constexpr uint32_t kConsumerWarps = kConsumers / 32;

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

__device__ __forceinline__ void mbar_arrive_cnt(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(count) : "memory");
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

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Explicit shared-memory accesses on 32-bit shared addresses (the hot loops
// reach their vectors through struct members, where generic addressing
// would otherwise be used).  volatile keeps them in program order with the
// barriers and with each other.
__device__ __forceinline__ float lds(uint32_t a, float) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ double lds(uint32_t a, double) {
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts(uint32_t a, float v) {
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void sts(uint32_t a, double v) {
    asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ uint2 lds_u2(uint32_t a) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ uint4 lds_u4(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ float4 lds_f4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ double2 lds_d2(uint32_t a) {
    double2 v;
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
    return v;
}

// Barrier among the consumer warps only (named barrier 1).
__device__ __forceinline__ void csync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory");
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

// Eight consecutive entries of one row of the row-major V (16-byte aligned:
// the row stride is a multiple of 8 entries), with read-only vector loads.
__device__ __forceinline__ void load_v8(const double *p, double (&v)[8]) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double2 t = __ldg(q + k);
        v[2 * k] = t.x;
        v[2 * k + 1] = t.y;
    }
}
__device__ __forceinline__ void load_v8(const __nv_bfloat16 *p, float (&v)[8]) {
    const uint4 t = __ldg(reinterpret_cast<const uint4 *>(p));
    const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[2 * k] = __uint_as_float(w[k] << 16);           // bf16 -> f32: the bits move up
        v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
}

// ----------------------------------------------------------- shared state

// Control words in shared memory.
struct Ctl {
    int abort;          // consumers ask the producer to stop
    int prod_done;      // producer has stopped issuing
    unsigned issued;    // segments the producer issued
    int ok;             // broadcast of a grid-wait result
};

// Consumer-side ring cursor (every consumer thread keeps an identical copy).
struct Ring {
    char *base;
    uint32_t full_s, empty_s;
    int slots, slot_bytes;
    int slot;
    uint32_t phase;
    unsigned consumed;
};

template <class T>
struct Cta {
    T *xi, *wi, *si, *tmp, *red;
    Ctl *ctl;
    Ring ring;
    unsigned bar_gen;  // consumer thread 0: generation seen at the last grid arrive
};

// Producer warp: copy the CTA's stream into the ring.
// With active != nullptr an entry is skipped when active[entry.pad] == 0
// (the batched kernel tags each entry with its system; the consumers skip the
// same systems, from the same flags, which no launch changes while it runs).
static __device__ void producer(const StreamEnt *stream, int64_t b, int64_t e, const char *segbase,
                         char *ring, int slots, int slot_bytes, uint32_t full_s, uint32_t empty_s,
                         Ctl *ctl, const int *active) {
    const int lane = threadIdx.x & 31;
    const uint32_t ring_s = smem_addr(ring);
    int slot = 0;
    uint32_t phase = 0;
    unsigned issued = 0;
    bool stop = false;
    StreamEnt nxt;
    nxt.off = 0;
    nxt.bytes = 0;
    if (b + lane < e) nxt = stream[b + lane];
    for (int64_t base = b; base < e && !stop; base += 32) {
        const StreamEnt cur = nxt;
        if (base + 32 + lane < e) nxt = stream[base + 32 + lane];  // prefetch the next chunk
        const int cnt = (int)((e - base) < 32 ? (e - base) : 32);
        for (int t = 0; t < cnt; ++t) {
            const long long off = __shfl_sync(0xffffffffu, (long long)cur.off, t);
            const int bytes = __shfl_sync(0xffffffffu, cur.bytes, t);
            if (active != nullptr && __ldg(active + __shfl_sync(0xffffffffu, cur.pad, t)) == 0) continue;
            if (lane == 0) {
                // slot free?  (the first pass over the ring finds every slot free)
                const uint32_t ebar = empty_s + 8 * slot;
                long long it = 0;
                // the ring is normally full here: back off instead of polling,
                // so this warp does not take issue slots from the consumers
                while (!mbar_try_wait(ebar, phase ^ 1u)) {
                    if (ld_volatile(&ctl->abort) || ++it > kTmaWaitLimit) {
                        stop = true;
                        break;
                    }
                    __nanosleep(128);
                }
                if (!stop) {
                    const uint32_t fbar = full_s + 8 * slot;
                    mbar_arrive_expect_tx(fbar, (uint32_t)bytes);
                    bulk_copy_g2s(ring_s + slot * slot_bytes, segbase + off, (uint32_t)bytes, fbar);
                    ++issued;
                }
            }
            stop = __shfl_sync(0xffffffffu, stop, 0);
            if (stop) break;
            if (++slot == slots) {
                slot = 0;
                phase ^= 1u;
            }
        }
    }
    if (lane == 0) {
        *(volatile unsigned *)&ctl->issued = issued;
        __threadfence_block();
        *(volatile int *)&ctl->prod_done = 1;
    }
}

// Consumers, on the way out after an abort: stop the producer, wait
// (bounded) for it, then for the copies it issued that nobody consumed.
template <class T>
__device__ void consumers_abort_drain(Cta<T> &c) {
    csync();
    if (threadIdx.x == 0) {
        *(volatile int *)&c.ctl->abort = 1;
        long long it = 0;
        while (!ld_volatile(&c.ctl->prod_done) && ++it < kTmaWaitLimit) {
        }
        const unsigned issued = *(volatile unsigned *)&c.ctl->issued;
        Ring R = c.ring;
        for (unsigned s = R.consumed; s < issued; ++s) {
            const uint32_t bar = R.full_s + 8 * R.slot;
            long long w = 0;
            while (!mbar_try_wait(bar, R.phase) && ++w < kTmaWaitLimit) {
            }
            if (++R.slot == R.slots) {
                R.slot = 0;
                R.phase ^= 1u;
            }
        }
    }
    csync();
}

// ----------------------------------------------------------------- grid barrier

// Sense-reversing barrier over all CTAs of the cooperative grid (consumers
// only).  arrive() publishes this CTA's writes; wait() returns once every CTA
// has arrived, or gives up (bounded) and latches PSLR_ERR_TIMEOUT.
template <class T>
__device__ void grid_arrive(Cta<T> &c, unsigned *bar, int grid) {
    csync();
    if (threadIdx.x == 0) {
        c.bar_gen = ld_acquire(bar + 1);
        __threadfence();
        const unsigned old = atomicAdd(bar, 1u);
        if (old == (unsigned)grid - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        }
    }
}

template <class T>
__device__ bool grid_wait(Cta<T> &c, unsigned *bar, int *err, long long limit) {
    if (threadIdx.x == 0) {
        int ok = 1;
        long long it = 0;
        while (ld_acquire(bar + 1) == c.bar_gen) {
            if (limit <= 0 || ++it > limit || ld_volatile(err) != 0) {
                atomicCAS(err, 0, kErrTimeout);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        c.ctl->ok = ok;
    }
    csync();
    return c.ctl->ok != 0;
}

// -------------------------------------------------------------- local operators

template <class T, class IDX>
struct Tile {
    const T *vals, *dinv;
    const IDX *cols;
    const uint16_t *rows;
    int n, w, np;
    bool diag;
};

template <class T, class IDX>
__device__ __forceinline__ Tile<T, IDX> tile_of(const char *seg) {
    const SegHdr h = *reinterpret_cast<const SegHdr *>(seg);
    Tile<T, IDX> t;
    t.n = h.n;
    t.w = h.w;
    t.np = h.np;
    t.diag = (h.flags & kSegDiag) != 0;
    const char *p = seg + sizeof(SegHdr);
    t.vals = reinterpret_cast<const T *>(p);
    p += (size_t)t.np * t.w * sizeof(T);
    t.dinv = reinterpret_cast<const T *>(p);
    if (t.diag) p += (size_t)t.np * sizeof(T);
    t.cols = reinterpret_cast<const IDX *>(p);
    p += (size_t)t.np * t.w * sizeof(IDX);
    t.rows = reinterpret_cast<const uint16_t *>(p);
    return t;
}

// Everything one thread needs of its row of a segment, read ahead of use:
// the row index, the K column indices and values and the reciprocal diagonal
// (record encodings), or a pointer for the rare wide tile.  None of it
// depends on the vector being solved for, so it is loaded while the previous
// level is still computing.
template <class T, class IDX>
struct RowPre {
    const char *seg;
    int n, np, fmt;
    bool diag;
    int r;
    IDX c[3];
    T v[3];
    T dv;
};

// The 7-entry record of row j, read when it is used.
template <class T, class IDX>
struct Rec7 {
    int r;
    IDX c[7];
    T v[7];
    T dv;
};

// Vector loads of one record (K+1 indices, K+1 values), unpacked into the
// named register fields of q.
template <class IDX>
struct IdxLoad;

template <>
struct IdxLoad<uint16_t> {
    template <class Q>
    __device__ __forceinline__ static void rec3(Q &q, const char *p) {
        const uint2 u = *reinterpret_cast<const uint2 *>(p);
        q.r = (int)(u.x & 0xffffu);
        q.c[0] = (uint16_t)(u.x >> 16);
        q.c[1] = (uint16_t)(u.y & 0xffffu);
        q.c[2] = (uint16_t)(u.y >> 16);
    }
    template <class Q>
    __device__ __forceinline__ static void rec7(Q &q, const char *p) {
        const uint4 u = *reinterpret_cast<const uint4 *>(p);
        q.r = (int)(u.x & 0xffffu);
        q.c[0] = (uint16_t)(u.x >> 16);
        q.c[1] = (uint16_t)(u.y & 0xffffu);
        q.c[2] = (uint16_t)(u.y >> 16);
        q.c[3] = (uint16_t)(u.z & 0xffffu);
        q.c[4] = (uint16_t)(u.z >> 16);
        q.c[5] = (uint16_t)(u.w & 0xffffu);
        q.c[6] = (uint16_t)(u.w >> 16);
    }
};

template <>
struct IdxLoad<int32_t> {
    template <class Q>
    __device__ __forceinline__ static void rec3(Q &q, const char *p) {
        const int4 u = *reinterpret_cast<const int4 *>(p);
        q.r = u.x;
        q.c[0] = u.y;
        q.c[1] = u.z;
        q.c[2] = u.w;
    }
    template <class Q>
    __device__ __forceinline__ static void rec7(Q &q, const char *p) {
        const int4 u = reinterpret_cast<const int4 *>(p)[0];
        const int4 v = reinterpret_cast<const int4 *>(p)[1];
        q.r = u.x;
        q.c[0] = u.y;
        q.c[1] = u.z;
        q.c[2] = u.w;
        q.c[3] = v.x;
        q.c[4] = v.y;
        q.c[5] = v.z;
        q.c[6] = v.w;
    }
};

template <class T>
struct ValLoad;

template <>
struct ValLoad<float> {
    template <class Q>
    __device__ __forceinline__ static void rec3(Q &q, const char *p) {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        q.v[0] = a.x;
        q.v[1] = a.y;
        q.v[2] = a.z;
        q.dv = a.w;
    }
    template <class Q>
    __device__ __forceinline__ static void rec7(Q &q, const char *p) {
        const float4 a = reinterpret_cast<const float4 *>(p)[0];
        const float4 b = reinterpret_cast<const float4 *>(p)[1];
        q.v[0] = a.x;
        q.v[1] = a.y;
        q.v[2] = a.z;
        q.v[3] = a.w;
        q.v[4] = b.x;
        q.v[5] = b.y;
        q.v[6] = b.z;
        q.dv = b.w;
    }
};

template <>
struct ValLoad<double> {
    template <class Q>
    __device__ __forceinline__ static void rec3(Q &q, const char *p) {
        const double2 a = reinterpret_cast<const double2 *>(p)[0];
        const double2 b = reinterpret_cast<const double2 *>(p)[1];
        q.v[0] = a.x;
        q.v[1] = a.y;
        q.v[2] = b.x;
        q.dv = b.y;
    }
    template <class Q>
    __device__ __forceinline__ static void rec7(Q &q, const char *p) {
        const double2 *d = reinterpret_cast<const double2 *>(p);
        const double2 a = d[0], b = d[1], c = d[2], e = d[3];
        q.v[0] = a.x;
        q.v[1] = a.y;
        q.v[2] = b.x;
        q.v[3] = b.y;
        q.v[4] = c.x;
        q.v[5] = c.y;
        q.v[6] = e.x;
        q.dv = e.y;
    }
};

template <class T, class IDX>
__device__ __forceinline__ void load_rec3(RowPre<T, IDX> &q, const char *seg, int np, int j) {
    const char *ib = seg + sizeof(SegHdr);
    const char *vb = ib + (size_t)np * 4 * sizeof(IDX);
    IdxLoad<IDX>::rec3(q, ib + (size_t)j * 4 * sizeof(IDX));
    ValLoad<T>::rec3(q, vb + (size_t)j * 4 * sizeof(T));
}

template <class T, class IDX>
__device__ __forceinline__ Rec7<T, IDX> load_rec7(const char *seg, int np, int j) {
    Rec7<T, IDX> q;
    const char *ib = seg + sizeof(SegHdr);
    const char *vb = ib + (size_t)np * 8 * sizeof(IDX);
    IdxLoad<IDX>::rec7(q, ib + (size_t)j * 8 * sizeof(IDX));
    ValLoad<T>::rec7(q, vb + (size_t)j * 8 * sizeof(T));
    return q;
}

template <class T, class IDX>
__device__ __forceinline__ RowPre<T, IDX> row_pre(const char *seg, int j) {
    RowPre<T, IDX> q;
    const SegHdr h = *reinterpret_cast<const SegHdr *>(seg);
    q.seg = seg;
    q.n = h.n;
    q.np = h.np;
    q.fmt = h.fmt;
    q.diag = (h.flags & kSegDiag) != 0;
    q.r = 0;
    q.dv = T(1);
    if (j < h.n) {
        if (h.fmt == kRec3) {
            load_rec3(q, seg, h.np, j);
        } else if (h.fmt == kRec7) {
            const char *ib = seg + sizeof(SegHdr);
            q.r = (int)reinterpret_cast<const IDX *>(ib)[(size_t)j * 8];
        } else {
            const Tile<T, IDX> t = tile_of<T, IDX>(seg);
            q.r = t.rows[j];
            if (t.diag) q.dv = t.dinv[j];
        }
    }
    return q;
}

// a - sum_k v_k src(c_k) for the thread's row.  Record rows run exactly K
// fused multiply-adds (padding entries multiply the zero slot by 0); wide
// tiles read their entries straight from the segment.
template <class T, class IDX, class SRC>
__device__ __forceinline__ T row_sub(RowPre<T, IDX> &q, int j, T a, SRC src) {
    if (q.fmt == kRec3) {
        T x[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) x[k] = src(q.c[k]);
#pragma unroll
        for (int k = 0; k < 3; ++k) a = fma_t(-q.v[k], x[k], a);
    } else if (q.fmt == kRec7) {
        const Rec7<T, IDX> e = load_rec7<T, IDX>(q.seg, q.np, j);
        q.dv = e.dv;
        T x[7];
#pragma unroll
        for (int k = 0; k < 7; ++k) x[k] = src(e.c[k]);
#pragma unroll
        for (int k = 0; k < 7; ++k) a = fma_t(-e.v[k], x[k], a);
    } else {
        const Tile<T, IDX> t = tile_of<T, IDX>(q.seg);
        for (int k = 0; k < t.w; ++k) a = fma_t(-t.vals[k * t.np + j], src(t.cols[k * t.np + j]), a);
    }
    return a;
}

// The 3-entry record of row j of a kRec3 segment.
template <class T>
struct Rec3 {
    int r, c0, c1, c2;
    T v0, v1, v2, d;
};

// Rows of a level in the 7-entry record or tile encodings (exact local LU,
// irregular matrices): out of line, so the common path stays small.
template <class T>
__device__ __noinline__ void level_row_general(const char *seg, T *x, int j) {
    RowPre<T, uint16_t> g = row_pre<T, uint16_t>(seg, j);
    if (j < g.n) {
        T a = row_sub(g, j, x[g.r], [&](int col) { return x[col]; });
        if (g.diag) a *= g.dv;
        x[g.r] = a;
    }
}

// Slow path of a segment wait (the producer is normally far ahead).
static __device__ __noinline__ void wait_full_slow(uint32_t bar, uint32_t phase, int *err) {
    long long it = 0;
    while (!mbar_try_wait(bar, phase)) {
        if (++it > kTmaWaitLimit) {
            atomicCAS(err, 0, kErrTimeout);
            return;
        }
    }
}

// The 3-entry record of row j of the kRec3 segment at shared address seg.
template <class T>
__device__ __forceinline__ Rec3<T> rec3_shared(uint32_t seg, int np, int j) {
    Rec3<T> e;
    const uint2 id = lds_u2(seg + (uint32_t)sizeof(SegHdr) + 8u * j);
    e.r = (int)(id.x & 0xffffu);
    e.c0 = (int)(id.x >> 16);
    e.c1 = (int)(id.y & 0xffffu);
    e.c2 = (int)(id.y >> 16);
    const uint32_t vp = seg + (uint32_t)sizeof(SegHdr) + 8u * np + (uint32_t)(4 * sizeof(T)) * j;
    if constexpr (sizeof(T) == 4) {
        const float4 v = lds_f4(vp);
        e.v0 = v.x;
        e.v1 = v.y;
        e.v2 = v.z;
        e.d = v.w;
    } else {
        const double2 a = lds_d2(vp), b = lds_d2(vp + 16);
        e.v0 = a.x;
        e.v1 = a.y;
        e.v2 = b.x;
        e.d = b.y;
    }
    return e;
}

// One 3-entry row of a sweep level per thread j < n: x[r] = (x[r] - v0 x[c0]
// - v1 x[c1] - v2 x[c2]) (* 1/diag where DIAG and scale).  FP64 rows without
// a diagonal use DIAG = false, so that no multiply is issued: on GB300 an FP64
// instruction holds the FP64 unit for its full time even when predicated off.
template <class T, bool DIAG>
__device__ __forceinline__ void sweep_row3(uint32_t seg_s, int n, int np, uint32_t xs, int j, bool scale = true) {
    constexpr uint32_t ts = sizeof(T);
    if (j < n) {
        const Rec3<T> e = rec3_shared<T>(seg_s, np, j);
        const T x0 = lds(xs + ts * e.c0, T()), x1 = lds(xs + ts * e.c1, T());
        const T x2 = lds(xs + ts * e.c2, T()), xr = lds(xs + ts * e.r, T());
        T a = fma_t(-e.v0, x0, xr);
        a = fma_t(-e.v1, x1, a);
        a = fma_t(-e.v2, x2, a);
        if constexpr (DIAG)
            if (scale) a *= e.d;
        sts(xs + ts * e.r, a);
    }
}

// tri_sweep_levels: one triangular sweep over `nseg` one-level segments, in place:
// x[r] = (x[r] - sum_k T_rk x[c_k]) (* dinv[r]).  The loop is kept to a few
// instructions per level (the level chain is latency-bound with two warps per
// scheduler, so every instruction costs): ring cursor in registers advanced
// incrementally, one header load, the 3-entry record path inline and
// everything else out of line.  Only the first segment is awaited by every
// consumer; the arrival of each later one is awaited by the last consumer
// thread just before the level barrier, and the barrier passes it on to the
// others (the same ordering as waiting for one's own asynchronous copies and
// then synchronising), which takes the mbarrier poll of 256 threads out of
// every level step.  kUnit: the sweep's 3-entry rows have a unit diagonal
// (no scaling multiply in the code at all: on GB300 an FP64 instruction holds
// the FP64 unit for its full time even when predicated off).
template <class T, bool kUnit = false>
__device__ void tri_sweep_levels(Cta<T> &c, T *x, int nseg, int *err) {
    Ring &R = c.ring;
    int slot = R.slot;
    uint32_t phase = R.phase;
    uint32_t fbar = R.full_s + 8 * slot;
    const uint32_t edelta = R.empty_s - R.full_s;
    const uint32_t base_s = smem_addr(R.base);
    uint32_t ptr_s = base_s + (uint32_t)(slot * R.slot_bytes);
    const uint32_t xs = smem_addr(x);
    const int j = threadIdx.x;
    constexpr uint32_t ts = sizeof(T);
    if (nseg > 0 && !mbar_try_wait(fbar, phase)) wait_full_slow(fbar, phase, err);
    for (int L = 0; L < nseg; ++L) {
        const uint2 h = lds_u2(ptr_s);
        if (((h.y >> 16) & 0xffu) == kRec3) {
            const int n = (int)(h.x & 0xffffu), np = (int)(h.y & 0xffffu);
            if constexpr (kUnit) {
                sweep_row3<T, false>(ptr_s, n, np, xs, j);
            } else if constexpr (sizeof(T) == 8) {  // no FP64 multiply issued in rows without a diagonal
                if ((h.x >> 24) & kSegDiag) sweep_row3<T, true>(ptr_s, n, np, xs, j);
                else sweep_row3<T, false>(ptr_s, n, np, xs, j);
            } else {
                sweep_row3<T, true>(ptr_s, n, np, xs, j, (h.x >> 24) & kSegDiag);
            }
        } else {
            level_row_general(R.base + (ptr_s - base_s), x, j);
        }
        if (j == kConsumers - 1 && L + 1 < nseg) {
            const bool wrap = slot + 1 == R.slots;
            const uint32_t nbar = wrap ? R.full_s : fbar + 8, nph = wrap ? phase ^ 1u : phase;
            if (!mbar_try_wait(nbar, nph)) wait_full_slow(nbar, nph, err);
        }
        csync();
        if (j == 0) mbar_arrive_cnt(fbar + edelta, kConsumerWarps);
        ++slot;
        fbar += 8;
        ptr_s += R.slot_bytes;
        if (slot == R.slots) {
            slot = 0;
            phase ^= 1u;
            fbar = R.full_s;
            ptr_s = base_s;
        }
    }
    R.slot = slot;
    R.phase = phase;
    R.consumed += nseg;
}

// tri_sweep_blocks: the same sweep over `nseg` segments that each hold one or
// more consecutive levels (blocks chained by kSegMore, each header giving the
// block's size in bytes), one barrier step per block.  The arrival of the next
// segment is awaited before the barrier of the current segment's last block,
// and a segment's slot is released after its last block.  The rows of a block
// are computed exactly as those of a one-level segment, so the result is the
// same bit for bit.
template <class T, bool kUnit = false>
__device__ void tri_sweep_blocks(Cta<T> &c, T *x, int nseg, int *err) {
    Ring &R = c.ring;
    int slot = R.slot;
    uint32_t phase = R.phase;
    uint32_t fbar = R.full_s + 8 * slot;
    const uint32_t edelta = R.empty_s - R.full_s;
    const uint32_t base_s = smem_addr(R.base);
    uint32_t ptr_s = base_s + (uint32_t)(slot * R.slot_bytes);  // the segment's slot
    uint32_t blk_s = ptr_s;                                       // the level block
    const uint32_t xs = smem_addr(x);
    const int j = threadIdx.x;
    constexpr uint32_t ts = sizeof(T);
    if (nseg > 0 && !mbar_try_wait(fbar, phase)) wait_full_slow(fbar, phase, err);
    for (int L = 0; L < nseg;) {
        const uint4 h = lds_u4(blk_s);
        if (((h.y >> 16) & 0xffu) == kRec3) {
            const int n = (int)(h.x & 0xffffu), np = (int)(h.y & 0xffffu);
            if constexpr (kUnit) {
                sweep_row3<T, false>(blk_s, n, np, xs, j);
            } else if constexpr (sizeof(T) == 8) {  // no FP64 multiply issued in rows without a diagonal
                if ((h.x >> 24) & kSegDiag) sweep_row3<T, true>(blk_s, n, np, xs, j);
                else sweep_row3<T, false>(blk_s, n, np, xs, j);
            } else {
                sweep_row3<T, true>(blk_s, n, np, xs, j, (h.x >> 24) & kSegDiag);
            }
        } else {
            level_row_general(R.base + (blk_s - base_s), x, j);
        }
        const bool more = (h.x >> 24) & kSegMore;
        if (!more && j == kConsumers - 1 && L + 1 < nseg) {
            const bool wrap = slot + 1 == R.slots;
            const uint32_t nbar = wrap ? R.full_s : fbar + 8, nph = wrap ? phase ^ 1u : phase;
            if (!mbar_try_wait(nbar, nph)) wait_full_slow(nbar, nph, err);
        }
        csync();
        if (more) {
            blk_s += h.z;
            continue;
        }
        if (j == 0) mbar_arrive_cnt(fbar + edelta, kConsumerWarps);
        ++L;
        ++slot;
        fbar += 8;
        ptr_s += R.slot_bytes;
        if (slot == R.slots) {
            slot = 0;
            phase ^= 1u;
            fbar = R.full_s;
            ptr_s = base_s;
        }
        blk_s = ptr_s;
    }
    R.slot = slot;
    R.phase = phase;
    R.consumed += nseg;
}

// One triangular sweep: one-level segments (the common layout: a tight loop
// of one level per segment) or multi-level segments (merged where the ring is
// shallow).  The form is a template parameter of the kernel.
template <class T, bool kMerged, bool kUnit = false>
__device__ __forceinline__ void tri_sweep(Cta<T> &c, T *x, int nseg, int *err) {
    if constexpr (kMerged) tri_sweep_blocks<T, kUnit>(c, x, nseg, err);
    else tri_sweep_levels<T, kUnit>(c, x, nseg, err);
}

// Rows of an ELL segment in the general encodings (out of line).
template <class T, bool GLOBAL>
__device__ __noinline__ void ell_row_general(const char *seg, T *out, const T *src, bool subtract, int j) {
    using IDX = typename std::conditional<GLOBAL, int32_t, uint16_t>::type;
    RowPre<T, IDX> q = row_pre<T, IDX>(seg, j);
    if (j < q.n) {
        T a;
        if (GLOBAL) a = -row_sub(q, j, T(0), [&](int col) { return __ldcg(src + col); });
        else a = -row_sub(q, j, T(0), [&](int col) { return src[col]; });
        out[q.r] = subtract ? out[q.r] - a : a;
    }
}

// ELL product over nseg segments: out[row] = sum (assign) or out[row] -= sum
// (subtract); src in shared memory (local columns) or global memory.  The
// segments write disjoint rows, so the warps go through them without a CTA
// barrier (each releases a slot on its own); one barrier closes the product.
template <class T, bool GLOBAL>
__device__ void ell_op(Cta<T> &c, T *out, const T *src, bool subtract, int nseg, int *err) {
    Ring &R = c.ring;
    int slot = R.slot;
    uint32_t phase = R.phase;
    uint32_t fbar = R.full_s + 8 * slot;
    const uint32_t edelta = R.empty_s - R.full_s;
    const uint32_t base_s = smem_addr(R.base);
    uint32_t ptr_s = base_s + (uint32_t)(slot * R.slot_bytes);
    const uint32_t os = smem_addr(out);
    const int j = threadIdx.x;
    constexpr uint32_t ts = sizeof(T);
    for (int k = 0; k < nseg; ++k) {
        if (!mbar_try_wait(fbar, phase)) wait_full_slow(fbar, phase, err);
        const uint2 h = lds_u2(ptr_s);
        if (!GLOBAL && ((h.y >> 16) & 0xffu) == kRec3) {
            if (j < (int)(h.x & 0xffffu)) {
                const uint32_t ss = smem_addr(src);
                const Rec3<T> e = rec3_shared<T>(ptr_s, (int)(h.y & 0xffffu), j);
                const T s0 = lds(ss + ts * e.c0, T()), s1 = lds(ss + ts * e.c1, T()), s2 = lds(ss + ts * e.c2, T());
                T a = e.v0 * s0;
                a = fma_t(e.v1, s1, a);
                a = fma_t(e.v2, s2, a);
                if (subtract) a = lds(os + ts * e.r, T()) - a;
                sts(os + ts * e.r, a);
            }
        } else {
            ell_row_general<T, GLOBAL>(R.base + (ptr_s - base_s), out, src, subtract, j);
        }
        __syncwarp();
        if ((j & 31) == 0) mbar_arrive(fbar + edelta);  // this warp is done with the slot
        ++slot;
        fbar += 8;
        ptr_s += R.slot_bytes;
        if (slot == R.slots) {
            slot = 0;
            phase ^= 1u;
            fbar = R.full_s;
            ptr_s = base_s;
        }
    }
    R.slot = slot;
    R.phase = phase;
    R.consumed += nseg;
    csync();  // the product is complete before anyone reads it
}

// Exact-LU row permutation: x <- P x (gather, before the sweeps) or
// x <- P^T x (scatter, after the transposed sweeps), via tmp.
template <class T>
__device__ void permute(T *x, T *tmp, const uint16_t *piv, int n, bool scatter) {
    csync();
    for (int j = threadIdx.x; j < n; j += kConsumers) tmp[j] = x[j];
    csync();
    for (int j = threadIdx.x; j < n; j += kConsumers) {
        if (scatter) x[piv[j]] = tmp[j];
        else x[j] = tmp[piv[j]];
    }
    csync();
}

// Local solve x <- B_i~^{-1} x (or C0_i~^{-1}, or a transpose): two sweeps
// (kUnit: both with unit-diagonal 3-entry rows).
template <class T, bool kMerged, bool kUnit = false>
__device__ void solve_local(Cta<T> &c, T *x, int n, const uint16_t *piv, int pivot_post, int n1,
                            int n2, int *err) {
    if (piv && !pivot_post) permute(x, c.tmp, piv, n, false);
    tri_sweep<T, kMerged, kUnit>(c, x, n1, err);
    tri_sweep<T, kMerged, kUnit>(c, x, n2, err);
    if (piv && pivot_post) permute(x, c.tmp, piv, n, true);
}

template <class T>
__device__ __forceinline__ void fill(T *x, int n, T v) {
    for (int j = threadIdx.x; j < n; j += kConsumers) x[j] = v;
}

struct Counts {
    int n[kNCnt];
};

__device__ __forceinline__ Counts counts_of(const int32_t *cnt, int i) {
    Counts k;
#pragma unroll
    for (int t = 0; t < kNCnt; ++t) k.n[t] = __ldg(cnt + kNCnt * i + t);
    return k;
}

// Partial dots part[i*r + c] = sum_j V[go + j, c] * y[j * ys] over this
// subdomain (c.red holds the 8 warps' sums at column stride rs >= r).  V is row-major with row stride ldv (a multiple of 8, zero
// padded), so a thread reads eight columns of a row with vector loads; rows
// are taken four at a time so that many loads are in flight.
template <class T, class VT>
__device__ void lowrank_partial(Cta<T> &c, const VT *V, int ldv, int r, int go, int nq, const T *y,
                                T *part_i, int ys, int rs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const VT *Vs = V + (int64_t)go * ldv;
    for (int c0 = 0; c0 < r; c0 += 8) {
        T a[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = T(0);
#pragma unroll 4
        for (int j = threadIdx.x; j < nq; j += kConsumers) {
            T v[8];
            load_v8(Vs + (int64_t)j * ldv + c0, v);
            const T yj = y[j * ys];
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = fma_t(v[k], yj, a[k]);
        }
        const T v = warp_reduce8(a);
        if ((lane & 3) == 0 && c0 + (lane >> 2) < r) c.red[warp * rs + c0 + (lane >> 2)] = v;
    }
    csync();
    for (int col = threadIdx.x; col < r; col += kConsumers) {
        T a = T(0);
        for (int w = 0; w < kConsumers / 32; ++w) a += c.red[w * rs + col];
        part_i[col] = a;
    }
    csync();
}

// d = G u with u = sum over subdomains of the partials, into the tail of
// c.red.  Threads split as (column, group of subdomains); the group sums are
// combined in a fixed order, so every CTA computes the same d.
template <class T>
__device__ void lowrank_coeffs(Cta<T> &c, const T *part, const T *G, int s, int r, int rs) {
    T *u = c.red + red_u_off(rs);
    T *d = u + rs;
    const int tpc = kConsumers / r;  // groups per column (r <= kMaxRank <= kConsumers)
    const int col = threadIdx.x % r, grp = threadIdx.x / r;
    if (grp < tpc) {
        T a = T(0);
#pragma unroll 4
        for (int i = grp; i < s; i += tpc) a += __ldcg(part + (int64_t)i * r + col);
        c.red[grp * r + col] = a;
    }
    csync();
    if (threadIdx.x < r) {
        T a = T(0);
        for (int g = 0; g < tpc; ++g) a += c.red[g * r + threadIdx.x];
        u[threadIdx.x] = a;
    }
    csync();
    for (int row = threadIdx.x; row < r; row += kConsumers) {
        T a = T(0);
        for (int k = 0; k < r; ++k) a = fma_t(G[k * r + row], u[k], a);
        d[row] = a;
    }
    csync();
}

// y[j * ys] += sum_c V[go + j, c] d[c] (V row-major with row stride ldv, as
// in lowrank_partial; entries of d past r are not read).
template <class T, class VT>
__device__ void lowrank_update(Cta<T> &c, const VT *V, int ldv, int r, int go, int nq, T *y, int ys, int rs) {
    const T *d = c.red + red_u_off(rs) + rs;
    const VT *Vs = V + (int64_t)go * ldv;
#pragma unroll 2
    for (int j = threadIdx.x; j < nq; j += kConsumers) {
        T a = y[j * ys];
        for (int c0 = 0; c0 < r; c0 += 8) {
            T v[8];
            load_v8(Vs + (int64_t)j * ldv + c0, v);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (c0 + k < r) a = fma_t(v[k], d[c0 + k], a);
        }
        y[j * ys] = a;
    }
    csync();
}

// Set up the CTA; returns true in the consumer threads.  The producer warp
// runs its stream inside and returns false.
template <class T>
__device__ bool cta_start(Cta<T> &c, char *smem, const SmemLayout &L, int ring, int slot_bytes,
                          const StreamEnt *stream, const int64_t *stream_off, const char *segbase,
                          const int *active = nullptr) {
    c.xi = reinterpret_cast<T *>(smem + L.xi);
    c.wi = reinterpret_cast<T *>(smem + L.wi);
    c.si = reinterpret_cast<T *>(smem + L.si);
    c.tmp = reinterpret_cast<T *>(smem + L.tmp);
    c.red = reinterpret_cast<T *>(smem + L.red);
    c.ctl = reinterpret_cast<Ctl *>(smem + L.ctl);
    c.ring.base = smem + L.ring;
    c.ring.full_s = smem_addr(smem + L.full);
    c.ring.empty_s = smem_addr(smem + L.empty);
    c.ring.slots = ring;
    c.ring.slot_bytes = slot_bytes;
    c.ring.slot = 0;
    c.ring.phase = 0;
    c.ring.consumed = 0;
    if (threadIdx.x == 0) {
        c.ctl->abort = 0;
        c.ctl->prod_done = 0;
        c.ctl->issued = 0;
        c.ctl->ok = 1;
        for (int i = 0; i < ring; ++i) {
            mbar_init(c.ring.full_s + 8 * i, 1);
            mbar_init(c.ring.empty_s + 8 * i, kConsumerWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x / 32 == kProducerWarp) {
        producer(stream, stream_off[blockIdx.x], stream_off[blockIdx.x + 1], segbase, c.ring.base, ring,
                 slot_bytes, c.ring.full_s, c.ring.empty_s, c.ctl, active);
        return false;
    }
    return true;
}

}  // namespace pslr
