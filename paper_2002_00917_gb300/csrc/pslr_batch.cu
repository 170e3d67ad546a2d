// Batched PSLR apply for sm_103a: many independent systems of uneven sizes,
// each with up to kMaxBatchRhs right-hand sides, in ONE cooperative launch
// (Algorithm 3, Eq. 3.24, applied to every system and right-hand side).
//
// Work items are (system, subdomain) pairs.  The host assigns them to the
// CTAs of one co-resident grid (longest first, onto the least-loaded CTA) and
// lays out each CTA's segment stream; the segments stay where each system's
// set-up put them.  Within every phase a CTA takes its items one after the
// other.  For an item it holds all right-hand sides of the subdomain in
// shared memory (vector k at offset k * stride) and sweeps every level once
// for all of them: a thread reads its row's record once, issues the loads of
// all right-hand sides, then their stores, so the right-hand sides give the
// level step independent work instead of each paying the level latency.
//
// The phases and grid barriers are those of the single-system kernel
// (pslr_apply.cu); systems with fewer series terms (smaller m) sit out the
// later terms, and the low-rank coefficients d = G V^T t of each (system,
// right-hand side) pair are formed once, by the CTA that owns the pair,
// between two grid barriers.  Inside the batched FGMRES a system whose
// problems have all converged drops out: the producer skips its segments and
// the consumers its items (per-system flags, fixed for the launch).  Local
// exact-LU factors (row pivoting) are not supported here; the host rejects
// such systems.
#include "pslr_device.cuh"

namespace pslr {

// ---------------------------------------------------- multi-rhs local ops

// Work split of a level among the consumer threads.  FP32 (and one rhs): one
// thread per row, all right-hand sides (their loads issue back to back).
// FP64 with several rhs: one thread per (row, rhs) pair, so the rhs spread
// over more warps - on GB300 a warp-wide FP64 instruction occupies its
// scheduler's FP64 pipe for many cycles whatever the number of active lanes,
// and a level has few rows (measured on 64 systems x 4 rhs: 5.96 -> 4.63 ms).
// Pair u = row * nr + k; thread j takes u = j, j + kConsumers, ...
struct PairWalk {
    int row, k, drow, dk, nr;
    __device__ __forceinline__ PairWalk(int j, int nr_) : nr(nr_) {
        row = j / nr_;
        k = j - row * nr_;
        drow = kConsumers / nr_;
        dk = kConsumers - drow * nr_;
    }
    __device__ __forceinline__ void next() {
        row += drow;
        k += dk;
        if (k >= nr) {
            k -= nr;
            ++row;
        }
    }
};

// One level sweep per segment for nr vectors x + k*xs (k < nr <= kMaxBatchRhs):
// x_k[r] = (x_k[r] - sum_e T_re x_k[c_e]) (* dinv[r]).
template <class T>
__device__ __noinline__ void tri_sweep_multi(Cta<T> &c, T *x, int xs, int nr, int nseg, int *err) {
    Ring &R = c.ring;
    int slot = R.slot;
    uint32_t phase = R.phase;
    uint32_t fbar = R.full_s + 8 * slot;
    const uint32_t edelta = R.empty_s - R.full_s;
    const uint32_t base_s = smem_addr(R.base);
    uint32_t ptr_s = base_s + (uint32_t)(slot * R.slot_bytes);
    const uint32_t x0s = smem_addr(x);
    constexpr uint32_t ts = sizeof(T);
    const uint32_t kstep = ts * (uint32_t)xs;
    const int j = threadIdx.x;
    for (int L = 0; L < nseg; ++L) {
        if (!mbar_try_wait(fbar, phase)) wait_full_slow(fbar, phase, err);
        const uint2 h = lds_u2(ptr_s);
        if (sizeof(T) == 8 && nr > 1 && ((h.y >> 16) & 0xffu) == kRec3) {
            const int n = (int)(h.x & 0xffffu), np = (int)(h.y & 0xffffu);
            const bool diag = (h.x >> 24) & kSegDiag;
            for (PairWalk u(j, nr); u.row < n; u.next()) {
                const Rec3<T> e = rec3_shared<T>(ptr_s, np, u.row);
                const uint32_t b = x0s + kstep * u.k;
                const T x0 = lds(b + ts * e.c0, T()), x1 = lds(b + ts * e.c1, T());
                const T x2 = lds(b + ts * e.c2, T()), xr = lds(b + ts * e.r, T());
                T a = fma_t(-e.v0, x0, xr);
                a = fma_t(-e.v1, x1, a);
                a = fma_t(-e.v2, x2, a);
                if (diag) a *= e.d;
                sts(b + ts * e.r, a);
            }
        } else if (((h.y >> 16) & 0xffu) == kRec3) {
            if (j < (int)(h.x & 0xffffu)) {
                const Rec3<T> e = rec3_shared<T>(ptr_s, (int)(h.y & 0xffffu), j);
                const bool diag = (h.x >> 24) & kSegDiag;
                T a0[kMaxBatchRhs], a1[kMaxBatchRhs], a2[kMaxBatchRhs], ar[kMaxBatchRhs];
#pragma unroll
                for (int k = 0; k < kMaxBatchRhs; ++k)
                    if (k < nr) {
                        const uint32_t b = x0s + kstep * k;
                        a0[k] = lds(b + ts * e.c0, T());
                        a1[k] = lds(b + ts * e.c1, T());
                        a2[k] = lds(b + ts * e.c2, T());
                        ar[k] = lds(b + ts * e.r, T());
                    }
#pragma unroll
                for (int k = 0; k < kMaxBatchRhs; ++k)
                    if (k < nr) {
                        T a = fma_t(-e.v0, a0[k], ar[k]);
                        a = fma_t(-e.v1, a1[k], a);
                        a = fma_t(-e.v2, a2[k], a);
                        if (diag) a *= e.d;
                        sts(x0s + kstep * k + ts * e.r, a);
                    }
            }
        } else {
            const char *seg = R.base + (ptr_s - base_s);
            for (int k = 0; k < nr; ++k) level_row_general(seg, x + (size_t)k * xs, j);
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

// ELL product of nseg segments for nr vectors: out_k[row] = sum (assign) or
// out_k[row] -= sum (subtract), sum = sum_e v_e src_k[c_e]; src in shared
// memory (local columns) or global memory (GLOBAL, the C_g rows).  Disjoint
// rows per segment: no CTA barrier between segments, one at the end.
template <class T, bool GLOBAL>
__device__ __noinline__ void ell_op_multi(Cta<T> &c, T *out, int os, const T *src, int ss, int nr, bool subtract,
                             int nseg, int *err) {
    Ring &R = c.ring;
    int slot = R.slot;
    uint32_t phase = R.phase;
    uint32_t fbar = R.full_s + 8 * slot;
    const uint32_t edelta = R.empty_s - R.full_s;
    const uint32_t base_s = smem_addr(R.base);
    uint32_t ptr_s = base_s + (uint32_t)(slot * R.slot_bytes);
    constexpr uint32_t ts = sizeof(T);
    const int j = threadIdx.x;
    for (int kseg = 0; kseg < nseg; ++kseg) {
        if (!mbar_try_wait(fbar, phase)) wait_full_slow(fbar, phase, err);
        const uint2 h = lds_u2(ptr_s);
        if (!GLOBAL && sizeof(T) == 8 && nr > 1 && ((h.y >> 16) & 0xffu) == kRec3) {
            const int n = (int)(h.x & 0xffffu), np = (int)(h.y & 0xffffu);
            const uint32_t o0 = smem_addr(out), s0 = smem_addr(src);
            for (PairWalk u(j, nr); u.row < n; u.next()) {
                const Rec3<T> e = rec3_shared<T>(ptr_s, np, u.row);
                const uint32_t sb = s0 + ts * (uint32_t)(u.k * ss), ob = o0 + ts * (uint32_t)(u.k * os);
                T a = e.v0 * lds(sb + ts * e.c0, T());
                a = fma_t(e.v1, lds(sb + ts * e.c1, T()), a);
                a = fma_t(e.v2, lds(sb + ts * e.c2, T()), a);
                if (subtract) a = lds(ob + ts * e.r, T()) - a;
                sts(ob + ts * e.r, a);
            }
        } else if (!GLOBAL && ((h.y >> 16) & 0xffu) == kRec3) {
            if (j < (int)(h.x & 0xffffu)) {
                const uint32_t o0 = smem_addr(out), s0 = smem_addr(src);
                const Rec3<T> e = rec3_shared<T>(ptr_s, (int)(h.y & 0xffffu), j);
                T b0[kMaxBatchRhs], b1[kMaxBatchRhs], b2[kMaxBatchRhs], br[kMaxBatchRhs];
#pragma unroll
                for (int k = 0; k < kMaxBatchRhs; ++k)
                    if (k < nr) {
                        const uint32_t sb = s0 + ts * (uint32_t)(k * ss);
                        b0[k] = lds(sb + ts * e.c0, T());
                        b1[k] = lds(sb + ts * e.c1, T());
                        b2[k] = lds(sb + ts * e.c2, T());
                        br[k] = subtract ? lds(o0 + ts * (uint32_t)(k * os + e.r), T()) : T(0);
                    }
#pragma unroll
                for (int k = 0; k < kMaxBatchRhs; ++k)
                    if (k < nr) {
                        T a = e.v0 * b0[k];
                        a = fma_t(e.v1, b1[k], a);
                        a = fma_t(e.v2, b2[k], a);
                        if (subtract) a = br[k] - a;
                        sts(o0 + ts * (uint32_t)(k * os + e.r), a);
                    }
            }
        } else {
            const char *seg = R.base + (ptr_s - base_s);
            for (int k = 0; k < nr; ++k)
                ell_row_general<T, GLOBAL>(seg, out + (size_t)k * os, src + (size_t)k * ss, subtract, j);
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

// ------------------------------------------------------------------ kernel

// Does system k take part in this launch?  (The producer skips the same
// systems' segments: both read the flags, which no launch changes while it runs.)
template <class T, class IO>
__device__ __forceinline__ bool on(const BatchParams<T, IO> &P, int k) {
    return P.active == nullptr || __ldg(P.active + k) != 0;
}

// One item of a group: its subdomain's ranges in the system and in the
// group's shared-memory vectors.
struct ItemRange {
    int i, io, np, go, nq, xo, lo;  // subdomain; interior start/length; interface start/length; group offsets
};

template <class T>
__device__ __forceinline__ ItemRange item_range(const BatchSys<T> &S, const BatchGroup &g, int t) {
    ItemRange it;
    it.i = g.sub[t];
    it.io = S.ioff[it.i];
    it.np = S.ioff[it.i + 1] - it.io;
    it.go = S.goff[it.i];
    it.nq = S.goff[it.i + 1] - it.go;
    it.xo = g.xo[t];
    it.lo = g.go[t];
    return it;
}

template <class T, class VT, class IO>
__global__ void __launch_bounds__(kThreads, 1) pslr_batch_apply_kernel(const BatchParams<T, IO> P) {
    extern __shared__ __align__(128) char smem[];
    if (P.skip != nullptr && ld_volatile(P.skip) != 0) return;
    if (ld_volatile(P.err) != 0) return;
    const int nr = P.nrhs;
    const int xs = P.xs, gs = P.gs;  // per-rhs strides of the group vectors
    const SmemLayout L = smem_layout(P.slot_bytes, P.ring, nr * xs - 1, nr * gs - 1, sizeof(T), false);
    Cta<T> c;
    if (!cta_start(c, smem, L, P.ring, P.slot_bytes, P.stream, P.stream_off, P.segbase, P.active)) return;
    const int tid = threadIdx.x;
    const int gb = P.group_off[blockIdx.x], ge = P.group_off[blockIdx.x + 1];
    T *const dsh = c.red + (kConsumers / 32) * kMaxRank + kMaxRank;  // where lowrank_coeffs leaves d
    bool ok = true;

    // ---- phase 0: u = B^{-1} f, t = g - F u (Algorithm 3, step 2); a system
    // without a low-rank term also takes w_0 = C0^{-1} t here.
    for (int gi = gb; gi < ge; ++gi) {
        const BatchGroup &g = P.groups[gi];
        if (!on(P, g.sys)) continue;
        const BatchSys<T> &S = P.sys[g.sys];
        const IO *bs = P.b + S.voff;
        for (int t = 0; t < g.n; ++t) {
            const ItemRange it = item_range(S, g, t);
            for (int kr = 0; kr < nr; ++kr) {
                const IO *bk = bs + (int64_t)kr * S.n;
                T *x = c.xi + kr * xs + it.xo, *y = c.si + kr * gs + it.lo;
                for (int j = tid; j < it.np; j += kConsumers) x[j] = T(bk[S.perm[it.io + j]]);
                for (int j = tid; j < it.nq; j += kConsumers) y[j] = T(bk[S.perm[S.p + it.go + j]]);
                if (tid == 0) {
                    x[it.np] = T(0);
                    y[it.nq] = T(0);
                }
            }
        }
        csync();
        tri_sweep_multi(c, c.xi, xs, nr, g.cnt[kB1], P.err);
        tri_sweep_multi(c, c.xi, xs, nr, g.cnt[kB2], P.err);
        ell_op_multi<T, false>(c, c.si, gs, c.xi, xs, nr, true, g.cnt[kF], P.err);
        if (S.r == 0) {
            tri_sweep_multi(c, c.si, gs, nr, g.cnt[kC1], P.err);
            tri_sweep_multi(c, c.si, gs, nr, g.cnt[kC2], P.err);
        }
        const VT *V = reinterpret_cast<const VT *>(S.V);
        for (int t = 0; t < g.n; ++t) {
            const ItemRange it = item_range(S, g, t);
            for (int kr = 0; kr < nr; ++kr) {
                const T *y = c.si + kr * gs + it.lo;
                if (S.r > 0)
                    lowrank_partial(c, V, S.q, S.r, it.go, it.nq, y, S.part + ((int64_t)kr * S.s + it.i) * S.r);
                T *acc = S.acc + (int64_t)kr * (S.q + 1) + it.go;
                T *w0 = S.wbuf + (int64_t)kr * 2 * (S.q + 1) + it.go;
                for (int j = tid; j < it.nq; j += kConsumers) {
                    acc[j] = y[j];
                    if (S.r == 0) w0[j] = y[j];
                }
            }
            if (it.i == 0 && tid == 0)  // zero slots of the system's series iterates
                for (int kr = 0; kr < nr; ++kr) {
                    S.wbuf[(int64_t)kr * 2 * (S.q + 1) + S.q] = T(0);
                    S.wbuf[(int64_t)kr * 2 * (S.q + 1) + (S.q + 1) + S.q] = T(0);
                }
        }
        csync();
    }

    // ---- phase 1: d = G V^T t per (system, rhs); t <- t + V d; w_0 = C0^{-1} t (steps 3-4)
    if (P.any_lr) {
        grid_arrive(c, P.bar, P.grid);
        ok = grid_wait(c, P.bar, P.err, P.wait_limit);
        if (!ok) goto abort;
        for (int pi = P.pair_off[blockIdx.x]; pi < P.pair_off[blockIdx.x + 1]; ++pi) {
            if (!on(P, P.pairs[2 * pi])) continue;
            const BatchSys<T> &S = P.sys[P.pairs[2 * pi]];
            const int kr = P.pairs[2 * pi + 1];
            lowrank_coeffs(c, S.part + (int64_t)kr * S.s * S.r, S.G, S.s, S.r);
            for (int j = tid; j < S.r; j += kConsumers) S.dco[(int64_t)kr * S.r + j] = dsh[j];
            csync();
        }
        grid_arrive(c, P.bar, P.grid);
        ok = grid_wait(c, P.bar, P.err, P.wait_limit);
        if (!ok) goto abort;
        for (int gi = gb; gi < ge; ++gi) {
            const BatchGroup &g = P.groups[gi];
            if (!on(P, g.sys)) continue;
            const BatchSys<T> &S = P.sys[g.sys];
            if (S.r == 0) continue;
            const VT *V = reinterpret_cast<const VT *>(S.V);
            for (int kr = 0; kr < nr; ++kr) {
                for (int j = tid; j < S.r; j += kConsumers) dsh[j] = __ldcg(S.dco + (int64_t)kr * S.r + j);
                for (int t = 0; t < g.n; ++t) {
                    const ItemRange it = item_range(S, g, t);
                    T *y = c.si + kr * gs + it.lo;
                    const T *acc = S.acc + (int64_t)kr * (S.q + 1) + it.go;
                    for (int j = tid; j < it.nq; j += kConsumers) y[j] = __ldcg(acc + j);
                    if (tid == 0) y[it.nq] = T(0);
                    csync();
                    lowrank_update(c, V, S.q, S.r, it.go, it.nq, y);
                }
            }
            tri_sweep_multi(c, c.si, gs, nr, g.cnt[kC1], P.err);
            tri_sweep_multi(c, c.si, gs, nr, g.cnt[kC2], P.err);
            for (int t = 0; t < g.n; ++t) {
                const ItemRange it = item_range(S, g, t);
                for (int kr = 0; kr < nr; ++kr) {
                    const T *y = c.si + kr * gs + it.lo;
                    T *acc = S.acc + (int64_t)kr * (S.q + 1) + it.go;
                    T *w0 = S.wbuf + (int64_t)kr * 2 * (S.q + 1) + it.go;
                    for (int j = tid; j < it.nq; j += kConsumers) {
                        w0[j] = y[j];
                        acc[j] = y[j];
                    }
                }
            }
            csync();
        }
    }

    // ---- series terms w_k = C0^{-1}(F B^{-1} E w_{k-1} - C_g w_{k-1}), acc += w_k (Eq. 3.3),
    // for the systems with m >= k
    for (int kk = 1; kk <= P.max_m; ++kk) {
        grid_arrive(c, P.bar, P.grid);
        bool waited = false;
        for (int gi = gb; gi < ge; ++gi) {
            const BatchGroup &g = P.groups[gi];
            if (!on(P, g.sys)) continue;
            const BatchSys<T> &S = P.sys[g.sys];
            if (S.m < kk) continue;
            const int64_t wst = 2 * (int64_t)(S.q + 1);
            const T *wprev = S.wbuf + ((kk - 1) & 1) * (S.q + 1);
            T *wnext = S.wbuf + (kk & 1) * (S.q + 1);
            const int nx = g.xo[g.n], ng = g.go[g.n];
            for (int kr = 0; kr < nr; ++kr) {
                fill(c.xi + kr * xs, nx, T(0));
                fill(c.si + kr * gs, ng, T(0));
                for (int t = 0; t < g.n; ++t) {
                    const ItemRange it = item_range(S, g, t);
                    T *w = c.wi + kr * gs + it.lo;
                    const T *src = wprev + kr * wst + it.go;
                    for (int j = tid; j < it.nq; j += kConsumers) w[j] = __ldcg(src + j);
                    if (tid == 0) w[it.nq] = T(0);
                }
            }
            csync();
            ell_op_multi<T, false>(c, c.xi, xs, c.wi, gs, nr, false, g.cnt[kE], P.err);   // E w
            tri_sweep_multi(c, c.xi, xs, nr, g.cnt[kB1], P.err);                         // B^{-1}
            tri_sweep_multi(c, c.xi, xs, nr, g.cnt[kB2], P.err);
            ell_op_multi<T, false>(c, c.si, gs, c.xi, xs, nr, false, g.cnt[kF], P.err);   // F
            if (!waited) {
                ok = grid_wait(c, P.bar, P.err, P.wait_limit);
                waited = true;
                if (!ok) goto abort;
            }
            ell_op_multi<T, true>(c, c.si, gs, wprev, (int)wst, nr, true, g.cnt[kCg], P.err);  // - C_g w
            tri_sweep_multi(c, c.si, gs, nr, g.cnt[kC1], P.err);                               // C0^{-1}
            tri_sweep_multi(c, c.si, gs, nr, g.cnt[kC2], P.err);
            for (int t = 0; t < g.n; ++t) {
                const ItemRange it = item_range(S, g, t);
                for (int kr = 0; kr < nr; ++kr) {
                    const T *y = c.si + kr * gs + it.lo;
                    T *acc = S.acc + (int64_t)kr * (S.q + 1) + it.go;
                    T *wn = wnext + kr * wst + it.go;
                    for (int j = tid; j < it.nq; j += kConsumers) {
                        wn[j] = y[j];
                        acc[j] = __ldcg(acc + j) + y[j];
                    }
                }
            }
            csync();
        }
        if (!waited) {  // a CTA with no work in this term still takes part in the barrier
            ok = grid_wait(c, P.bar, P.err, P.wait_limit);
            if (!ok) goto abort;
        }
    }

    // ---- y = acc; x = B^{-1}(f - E y); scatter (steps 5-6)
    for (int gi = gb; gi < ge; ++gi) {
        const BatchGroup &g = P.groups[gi];
        if (!on(P, g.sys)) continue;
        const BatchSys<T> &S = P.sys[g.sys];
        const IO *bs = P.b + S.voff;
        for (int t = 0; t < g.n; ++t) {
            const ItemRange it = item_range(S, g, t);
            for (int kr = 0; kr < nr; ++kr) {
                const IO *bk = bs + (int64_t)kr * S.n;
                T *x = c.xi + kr * xs + it.xo, *w = c.wi + kr * gs + it.lo;
                const T *acc = S.acc + (int64_t)kr * (S.q + 1) + it.go;
                for (int j = tid; j < it.nq; j += kConsumers) w[j] = __ldcg(acc + j);
                for (int j = tid; j < it.np; j += kConsumers) x[j] = T(bk[S.perm[it.io + j]]);
                if (tid == 0) {
                    w[it.nq] = T(0);
                    x[it.np] = T(0);
                }
            }
        }
        csync();
        ell_op_multi<T, false>(c, c.xi, xs, c.wi, gs, nr, true, g.cnt[kE], P.err);
        tri_sweep_multi(c, c.xi, xs, nr, g.cnt[kB1], P.err);
        tri_sweep_multi(c, c.xi, xs, nr, g.cnt[kB2], P.err);
        IO *zs = P.z + S.voff;
        for (int t = 0; t < g.n; ++t) {
            const ItemRange it = item_range(S, g, t);
            for (int kr = 0; kr < nr; ++kr) {
                IO *zk = zs + (int64_t)kr * S.n;
                const T *x = c.xi + kr * xs + it.xo, *w = c.wi + kr * gs + it.lo;
                for (int j = tid; j < it.np; j += kConsumers) zk[S.perm[it.io + j]] = IO(x[j]);
                for (int j = tid; j < it.nq; j += kConsumers) zk[S.perm[S.p + it.go + j]] = IO(w[j]);
            }
        }
        csync();
    }
    return;
abort:
    consumers_abort_drain(c);
}

// ------------------------------------------------------------------ launchers

template <class T, class VT, class IO>
static cudaError_t launch_batch_t(const void *prm, int smem, cudaStream_t st) {
    const BatchParams<T, IO> &P = *static_cast<const BatchParams<T, IO> *>(prm);
    auto kern = pslr_batch_apply_kernel<T, VT, IO>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<BatchParams<T, IO> *>(&P)};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(P.grid), dim3(kThreads), args, smem, st);
}

// form 0: FP64 in and out; 1: FP32 in and out (BF16 V); 2: FP32 arithmetic on FP64 in and out.
cudaError_t launch_batch(int form, const void *params, int smem, cudaStream_t st) {
    switch (form) {
    case 0: return launch_batch_t<double, double, double>(params, smem, st);
    case 1: return launch_batch_t<float, __nv_bfloat16, float>(params, smem, st);
    case 2: return launch_batch_t<float, __nv_bfloat16, double>(params, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

template <class K>
static int coresident(K kern, int smem) {
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, smem) != cudaSuccess) return 0;
    return per * nsm;
}

// Largest cooperative grid of the batched kernel at this shared-memory size
// (the smaller over the forms that share the layout).
int max_coresident_batch(int smem, bool fp32) {
    if (!fp32) return coresident(pslr_batch_apply_kernel<double, double, double>, smem);
    const int a = coresident(pslr_batch_apply_kernel<float, __nv_bfloat16, float>, smem);
    const int b = coresident(pslr_batch_apply_kernel<float, __nv_bfloat16, double>, smem);
    return a < b ? a : b;
}

}  // namespace pslr
