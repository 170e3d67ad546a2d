// Batched PSLR apply for sm_103a (device code; pslr_batch_f64.cu,
// pslr_batch_f32.cu and pslr_batch_f32d.cu instantiate it, one precision form
// each, for 1..kMaxBatchRhs right-hand sides): many independent systems of uneven sizes,
// each with up to kMaxBatchRhs right-hand sides, in ONE cooperative launch
// (Algorithm 3, Eq. 3.24, applied to every system and right-hand side).
//
// Work items are (system, subdomain) pairs.  The host assigns them to the
// CTAs of one co-resident grid (longest first, onto the least-loaded CTA) and
// lays out each CTA's segment stream; the segments stay where each system's
// set-up put them.  Within every phase a CTA takes its items one after the
// other.  For an item it holds all right-hand sides of the subdomain in
// shared memory (interleaved: entry i of rhs k at i * nrhs + k) and sweeps every level once
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
#pragma once
#include "pslr_device.cuh"

namespace pslr {

// ---------------------------------------------------- multi-rhs local ops

// The local vectors hold the nr right-hand sides interleaved: entry i of
// right-hand side k is x[i * nr + k], so the values of one entry for all rhs
// are adjacent (one vector access for nr = 4 or 2).

template <int NR>
__device__ __forceinline__ void lds_rhs(uint32_t a, float (&v)[kMaxBatchRhs]) {
    if constexpr (NR == 4) {
        const float4 t = lds_f4(a);
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    } else if constexpr (NR == 2) {
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v[0]), "=f"(v[1]) : "r"(a));
    } else {
#pragma unroll
        for (int k = 0; k < NR; ++k) v[k] = lds(a + 4u * k, 0.f);
    }
}
template <int NR>
__device__ __forceinline__ void sts_rhs(uint32_t a, const float (&v)[kMaxBatchRhs]) {
    if constexpr (NR == 4) {
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3])
                     : "memory");
    } else if constexpr (NR == 2) {
        asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v[0]), "f"(v[1]) : "memory");
    } else {
#pragma unroll
        for (int k = 0; k < NR; ++k) sts(a + 4u * k, v[k]);
    }
}
template <int NR>
__device__ __forceinline__ void lds_rhs(uint32_t a, double (&v)[kMaxBatchRhs]) {
    if constexpr (NR == 4 || NR == 2) {
        const double2 t = lds_d2(a);
        v[0] = t.x;
        v[1] = t.y;
        if constexpr (NR == 4) {
            const double2 u = lds_d2(a + 16u);
            v[2] = u.x;
            v[3] = u.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < NR; ++k) v[k] = lds(a + 8u * k, 0.0);
    }
}
template <int NR>
__device__ __forceinline__ void sts_rhs(uint32_t a, const double (&v)[kMaxBatchRhs]) {
    if constexpr (NR == 4 || NR == 2) {
        asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v[0]), "d"(v[1]) : "memory");
        if constexpr (NR == 4)
            asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(a + 16u), "d"(v[2]), "d"(v[3]) : "memory");
    } else {
#pragma unroll
        for (int k = 0; k < NR; ++k) sts(a + 8u * k, v[k]);
    }
}

// Work split of a level among the consumer threads.  FP32 (and one rhs): one
// thread per row, all right-hand sides (one vector load per column).  FP64
// with several rhs: one thread per (row, rhs) pair, so the rhs spread over
// more warps - on GB300 a warp-wide FP64 instruction occupies its scheduler's
// FP64 pipe for many cycles whatever the number of active lanes, and a level
// has few rows (measured on 64 systems x 4 rhs: 5.96 -> 4.63 ms).
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

// Rows of a level in the 7-entry record or tile encodings, one rhs (out of line).
template <class T>
__device__ __noinline__ void level_row_general_rhs(const char *seg, T *x, int nr, int k, int j) {
    RowPre<T, uint16_t> g = row_pre<T, uint16_t>(seg, j);
    if (j < g.n) {
        T a = row_sub(g, j, x[g.r * nr + k], [&](int col) { return x[col * nr + k]; });
        if (g.diag) a *= g.dv;
        x[g.r * nr + k] = a;
    }
}

// Rows of a product segment in the general encodings, one rhs (out of line);
// GLOBAL: src is the system's interface iterate in global memory (rhs k at
// src + k * ss), else an interleaved shared-memory vector.
template <class T, bool GLOBAL>
__device__ __noinline__ void ell_row_general_rhs(const char *seg, T *out, int nr, const T *src, int64_t ss, int k,
                                                 bool subtract, int j) {
    using IDX = typename std::conditional<GLOBAL, int32_t, uint16_t>::type;
    RowPre<T, IDX> q = row_pre<T, IDX>(seg, j);
    if (j < q.n) {
        T a;
        if (GLOBAL) a = -row_sub(q, j, T(0), [&](int col) { return __ldcg(src + k * ss + col); });
        else a = -row_sub(q, j, T(0), [&](int col) { return src[col * nr + k]; });
        T &o = out[q.r * nr + k];
        o = subtract ? o - a : a;
    }
}

// One level sweep per segment for the nr interleaved right-hand sides of x:
// x_k[r] = (x_k[r] - sum_e T_re x_k[c_e]) (* dinv[r]).  As in tri_sweep, the
// arrival of each segment after the first is awaited by the last consumer
// thread before the level barrier.
// The 3-entry rows of one sweep level for the nr interleaved right-hand
// sides, one thread per (row, rhs) pair (FP64) or per row with all its rhs;
// DIAG: rows scaled by 1/diag.  Separate loops for the two, because an FP64
// multiply that is predicated off still holds the FP64 unit on GB300.
template <class T, int NR, bool DIAG>
__device__ __forceinline__ void sweep_pairs(uint32_t ptr_s, int n, int np, uint32_t x0s, int j) {
    constexpr uint32_t ts = sizeof(T);
    const uint32_t es = ts * (uint32_t)NR;
    for (PairWalk u(j, NR); u.row < n; u.next()) {
        const Rec3<T> e = rec3_shared<T>(ptr_s, np, u.row);
        const uint32_t b = x0s + ts * u.k;
        const T x0 = lds(b + es * e.c0, T()), x1 = lds(b + es * e.c1, T());
        const T x2 = lds(b + es * e.c2, T()), xr = lds(b + es * e.r, T());
        T a = fma_t(-e.v0, x0, xr);
        a = fma_t(-e.v1, x1, a);
        a = fma_t(-e.v2, x2, a);
        if constexpr (DIAG) a *= e.d;
        sts(b + es * e.r, a);
    }
}
template <class T, int NR, bool DIAG>
__device__ __forceinline__ void sweep_rows_rhs(uint32_t ptr_s, int n, int np, uint32_t x0s, int j, bool scale = true) {
    constexpr uint32_t es = sizeof(T) * (uint32_t)NR;
    if (j < n) {
        const Rec3<T> e = rec3_shared<T>(ptr_s, np, j);
        T a0[kMaxBatchRhs], a1[kMaxBatchRhs], a2[kMaxBatchRhs], ar[kMaxBatchRhs];
        lds_rhs<NR>(x0s + es * e.c0, a0);
        lds_rhs<NR>(x0s + es * e.c1, a1);
        lds_rhs<NR>(x0s + es * e.c2, a2);
        lds_rhs<NR>(x0s + es * e.r, ar);
#pragma unroll
        for (int k = 0; k < kMaxBatchRhs; ++k)
            if (k < NR) {
                T a = fma_t(-e.v0, a0[k], ar[k]);
                a = fma_t(-e.v1, a1[k], a);
                a = fma_t(-e.v2, a2[k], a);
                if constexpr (DIAG) ar[k] = scale ? a * e.d : a;
                else ar[k] = a;
            }
        sts_rhs<NR>(x0s + es * e.r, ar);
    }
}

template <class T, int NR>
__device__ __noinline__ void tri_sweep_multi(Cta<T> &c, T *x, int nseg, int *err, bool pair) {
    constexpr int nr = NR;
    Ring &R = c.ring;
    int slot = R.slot;
    uint32_t phase = R.phase;
    uint32_t fbar = R.full_s + 8 * slot;
    const uint32_t edelta = R.empty_s - R.full_s;
    const uint32_t base_s = smem_addr(R.base);
    uint32_t ptr_s = base_s + (uint32_t)(slot * R.slot_bytes);
    const uint32_t x0s = smem_addr(x);
    constexpr uint32_t ts = sizeof(T);
    const uint32_t es = ts * (uint32_t)nr;  // bytes per entry (all rhs)
    const int j = threadIdx.x;
    if (nseg > 0 && !mbar_try_wait(fbar, phase)) wait_full_slow(fbar, phase, err);
    for (int L = 0; L < nseg; ++L) {
        const uint2 h = lds_u2(ptr_s);
        if (sizeof(T) == 8 && nr > 1 && pair && ((h.y >> 16) & 0xffu) == kRec3) {
            const int n = (int)(h.x & 0xffffu), np = (int)(h.y & 0xffffu);
            if ((h.x >> 24) & kSegDiag) sweep_pairs<T, NR, true>(ptr_s, n, np, x0s, j);
            else sweep_pairs<T, NR, false>(ptr_s, n, np, x0s, j);
        } else if (((h.y >> 16) & 0xffu) == kRec3) {
            const int n = (int)(h.x & 0xffffu), np = (int)(h.y & 0xffffu);
            if constexpr (sizeof(T) == 8) {  // FP64: rows without a diagonal issue no multiply
                if ((h.x >> 24) & kSegDiag) sweep_rows_rhs<T, NR, true>(ptr_s, n, np, x0s, j);
                else sweep_rows_rhs<T, NR, false>(ptr_s, n, np, x0s, j);
            } else {
                sweep_rows_rhs<T, NR, true>(ptr_s, n, np, x0s, j, (h.x >> 24) & kSegDiag);
            }
        } else {
            const char *seg = R.base + (ptr_s - base_s);
            for (int k = 0; k < nr; ++k) level_row_general_rhs(seg, x, nr, k, j);
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

// ELL product of nseg segments for the nr interleaved right-hand sides:
// out_k[row] = sum (assign) or out_k[row] -= sum (subtract), sum = sum_e v_e
// src_k[c_e]; src interleaved in shared memory (local columns), or global
// (GLOBAL, the C_g rows: rhs k at src + k * ss).  Disjoint rows per segment:
// no CTA barrier between segments, one at the end.
template <class T, bool GLOBAL, int NR>
__device__ __noinline__ void ell_op_multi(Cta<T> &c, T *out, const T *src, int64_t ss, bool subtract, int nseg,
                                          int *err, bool pair) {
    constexpr int nr = NR;
    Ring &R = c.ring;
    int slot = R.slot;
    uint32_t phase = R.phase;
    uint32_t fbar = R.full_s + 8 * slot;
    const uint32_t edelta = R.empty_s - R.full_s;
    const uint32_t base_s = smem_addr(R.base);
    uint32_t ptr_s = base_s + (uint32_t)(slot * R.slot_bytes);
    constexpr uint32_t ts = sizeof(T);
    const uint32_t es = ts * (uint32_t)nr;
    const int j = threadIdx.x;
    for (int kseg = 0; kseg < nseg; ++kseg) {
        if (!mbar_try_wait(fbar, phase)) wait_full_slow(fbar, phase, err);
        const uint2 h = lds_u2(ptr_s);
        if (!GLOBAL && sizeof(T) == 8 && nr > 1 && pair && ((h.y >> 16) & 0xffu) == kRec3) {
            const int n = (int)(h.x & 0xffffu), np = (int)(h.y & 0xffffu);
            const uint32_t o0 = smem_addr(out), s0 = smem_addr(src);
            for (PairWalk u(j, nr); u.row < n; u.next()) {
                const Rec3<T> e = rec3_shared<T>(ptr_s, np, u.row);
                const uint32_t sb = s0 + ts * u.k, ob = o0 + ts * u.k;
                T a = e.v0 * lds(sb + es * e.c0, T());
                a = fma_t(e.v1, lds(sb + es * e.c1, T()), a);
                a = fma_t(e.v2, lds(sb + es * e.c2, T()), a);
                if (subtract) a = lds(ob + es * e.r, T()) - a;
                sts(ob + es * e.r, a);
            }
        } else if (!GLOBAL && ((h.y >> 16) & 0xffu) == kRec3) {
            if (j < (int)(h.x & 0xffffu)) {
                const uint32_t o0 = smem_addr(out), s0 = smem_addr(src);
                const Rec3<T> e = rec3_shared<T>(ptr_s, (int)(h.y & 0xffffu), j);
                T b0[kMaxBatchRhs], b1[kMaxBatchRhs], b2[kMaxBatchRhs], br[kMaxBatchRhs];
                lds_rhs<NR>(s0 + es * e.c0, b0);
                lds_rhs<NR>(s0 + es * e.c1, b1);
                lds_rhs<NR>(s0 + es * e.c2, b2);
                if (subtract) lds_rhs<NR>(o0 + es * e.r, br);
#pragma unroll
                for (int k = 0; k < kMaxBatchRhs; ++k)
                    if (k < nr) {
                        T a = e.v0 * b0[k];
                        a = fma_t(e.v1, b1[k], a);
                        a = fma_t(e.v2, b2[k], a);
                        br[k] = subtract ? br[k] - a : a;
                    }
                sts_rhs<NR>(o0 + es * e.r, br);
            }
        } else {
            const char *seg = R.base + (ptr_s - base_s);
            for (int k = 0; k < nr; ++k) ell_row_general_rhs<T, GLOBAL>(seg, out, nr, src, ss, k, subtract, j);
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

template <class T, class VT, class IO, int NR>
__global__ void __launch_bounds__(kThreads, 1) pslr_batch_apply_kernel(const BatchParams<T, IO> P) {
    extern __shared__ __align__(128) char smem[];
    if (P.skip != nullptr && ld_volatile(P.skip) != 0) return;
    if (ld_volatile(P.err) != 0) return;
    constexpr int nr = NR;  // == P.nrhs
    // group vectors: P.xs interior / P.gs interface entries, nr values each (interleaved)
    const SmemLayout L = smem_layout(P.slot_bytes, P.ring, nr * P.xs - 1, nr * P.gs - 1, sizeof(T), false);
    Cta<T> c;
    if (!cta_start(c, smem, L, P.ring, P.slot_bytes, P.stream, P.stream_off, P.segbase, P.active)) return;
    const int tid = threadIdx.x;
    const int gb = P.group_off[blockIdx.x], ge = P.group_off[blockIdx.x + 1];
    T *const dsh = c.red + red_u_off(kMaxRank) + kMaxRank;  // where lowrank_coeffs leaves d
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
            T *x = c.xi + it.xo * nr, *y = c.si + it.lo * nr;
            for (int j = tid; j < it.np; j += kConsumers) {
                const int o = S.perm[it.io + j];
                for (int kr = 0; kr < nr; ++kr) x[j * nr + kr] = T(bs[(int64_t)kr * S.n + o]);
            }
            for (int j = tid; j < it.nq; j += kConsumers) {
                const int o = S.perm[S.p + it.go + j];
                for (int kr = 0; kr < nr; ++kr) y[j * nr + kr] = T(bs[(int64_t)kr * S.n + o]);
            }
            for (int kr = tid; kr < nr; kr += kConsumers) {
                x[it.np * nr + kr] = T(0);
                y[it.nq * nr + kr] = T(0);
            }
        }
        csync();
        tri_sweep_multi<T, NR>(c, c.xi, g.cnt[kB1], P.err, P.pair64 != 0);
        tri_sweep_multi<T, NR>(c, c.xi, g.cnt[kB2], P.err, P.pair64 != 0);
        ell_op_multi<T, false, NR>(c, c.si, c.xi, 0, true, g.cnt[kF], P.err, P.pair64 != 0);
        if (S.r == 0) {
            tri_sweep_multi<T, NR>(c, c.si, g.cnt[kC1], P.err, P.pair64 != 0);
            tri_sweep_multi<T, NR>(c, c.si, g.cnt[kC2], P.err, P.pair64 != 0);
        }
        const VT *V = reinterpret_cast<const VT *>(S.V);
        for (int t = 0; t < g.n; ++t) {
            const ItemRange it = item_range(S, g, t);
            const T *y = c.si + it.lo * nr;
            if (S.r > 0)
                for (int kr = 0; kr < nr; ++kr)
                    lowrank_partial(c, V, S.ldv, S.r, it.go, it.nq, y + kr, S.part + ((int64_t)kr * S.s + it.i) * S.r,
                                    nr, kMaxRank);
            for (int j = tid; j < it.nq; j += kConsumers)
                for (int kr = 0; kr < nr; ++kr) {
                    const T v = y[j * nr + kr];
                    S.acc[(int64_t)kr * (S.q + 1) + it.go + j] = v;
                    if (S.r == 0) S.wbuf[(int64_t)kr * 2 * (S.q + 1) + it.go + j] = v;
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
            lowrank_coeffs(c, S.part + (int64_t)kr * S.s * S.r, S.G, S.s, S.r, kMaxRank);
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
            for (int t = 0; t < g.n; ++t) {
                const ItemRange it = item_range(S, g, t);
                T *y = c.si + it.lo * nr;
                for (int j = tid; j < it.nq; j += kConsumers)
                    for (int kr = 0; kr < nr; ++kr) y[j * nr + kr] = __ldcg(S.acc + (int64_t)kr * (S.q + 1) + it.go + j);
                for (int kr = tid; kr < nr; kr += kConsumers) y[it.nq * nr + kr] = T(0);
            }
            for (int kr = 0; kr < nr; ++kr) {
                for (int j = tid; j < S.r; j += kConsumers) dsh[j] = __ldcg(S.dco + (int64_t)kr * S.r + j);
                csync();
                for (int t = 0; t < g.n; ++t) {
                    const ItemRange it = item_range(S, g, t);
                    lowrank_update(c, V, S.ldv, S.r, it.go, it.nq, c.si + it.lo * nr + kr, nr, kMaxRank);
                }
            }
            tri_sweep_multi<T, NR>(c, c.si, g.cnt[kC1], P.err, P.pair64 != 0);
            tri_sweep_multi<T, NR>(c, c.si, g.cnt[kC2], P.err, P.pair64 != 0);
            for (int t = 0; t < g.n; ++t) {
                const ItemRange it = item_range(S, g, t);
                const T *y = c.si + it.lo * nr;
                for (int j = tid; j < it.nq; j += kConsumers)
                    for (int kr = 0; kr < nr; ++kr) {
                        const T v = y[j * nr + kr];
                        S.wbuf[(int64_t)kr * 2 * (S.q + 1) + it.go + j] = v;
                        S.acc[(int64_t)kr * (S.q + 1) + it.go + j] = v;
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
            fill(c.xi, g.xo[g.n] * nr, T(0));
            fill(c.si, g.go[g.n] * nr, T(0));
            for (int t = 0; t < g.n; ++t) {
                const ItemRange it = item_range(S, g, t);
                T *w = c.wi + it.lo * nr;
                for (int j = tid; j < it.nq; j += kConsumers)
                    for (int kr = 0; kr < nr; ++kr) w[j * nr + kr] = __ldcg(wprev + kr * wst + it.go + j);
                for (int kr = tid; kr < nr; kr += kConsumers) w[it.nq * nr + kr] = T(0);
            }
            csync();
            ell_op_multi<T, false, NR>(c, c.xi, c.wi, 0, false, g.cnt[kE], P.err, P.pair64 != 0);   // E w
            tri_sweep_multi<T, NR>(c, c.xi, g.cnt[kB1], P.err, P.pair64 != 0);                       // B^{-1}
            tri_sweep_multi<T, NR>(c, c.xi, g.cnt[kB2], P.err, P.pair64 != 0);
            ell_op_multi<T, false, NR>(c, c.si, c.xi, 0, false, g.cnt[kF], P.err, P.pair64 != 0);   // F
            if (!waited) {
                ok = grid_wait(c, P.bar, P.err, P.wait_limit);
                waited = true;
                if (!ok) goto abort;
            }
            ell_op_multi<T, true, NR>(c, c.si, wprev, wst, true, g.cnt[kCg], P.err, P.pair64 != 0);  // - C_g w
            tri_sweep_multi<T, NR>(c, c.si, g.cnt[kC1], P.err, P.pair64 != 0);                       // C0^{-1}
            tri_sweep_multi<T, NR>(c, c.si, g.cnt[kC2], P.err, P.pair64 != 0);
            for (int t = 0; t < g.n; ++t) {
                const ItemRange it = item_range(S, g, t);
                const T *y = c.si + it.lo * nr;
                for (int j = tid; j < it.nq; j += kConsumers)
                    for (int kr = 0; kr < nr; ++kr) {
                        const T v = y[j * nr + kr];
                        T *acc = S.acc + (int64_t)kr * (S.q + 1) + it.go + j;
                        wnext[kr * wst + it.go + j] = v;
                        *acc = __ldcg(acc) + v;
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
            T *x = c.xi + it.xo * nr, *w = c.wi + it.lo * nr;
            for (int j = tid; j < it.nq; j += kConsumers)
                for (int kr = 0; kr < nr; ++kr) w[j * nr + kr] = __ldcg(S.acc + (int64_t)kr * (S.q + 1) + it.go + j);
            for (int j = tid; j < it.np; j += kConsumers) {
                const int o = S.perm[it.io + j];
                for (int kr = 0; kr < nr; ++kr) x[j * nr + kr] = T(bs[(int64_t)kr * S.n + o]);
            }
            for (int kr = tid; kr < nr; kr += kConsumers) {
                w[it.nq * nr + kr] = T(0);
                x[it.np * nr + kr] = T(0);
            }
        }
        csync();
        ell_op_multi<T, false, NR>(c, c.xi, c.wi, 0, true, g.cnt[kE], P.err, P.pair64 != 0);
        tri_sweep_multi<T, NR>(c, c.xi, g.cnt[kB1], P.err, P.pair64 != 0);
        tri_sweep_multi<T, NR>(c, c.xi, g.cnt[kB2], P.err, P.pair64 != 0);
        IO *zs = P.z + S.voff;
        for (int t = 0; t < g.n; ++t) {
            const ItemRange it = item_range(S, g, t);
            const T *x = c.xi + it.xo * nr, *w = c.wi + it.lo * nr;
            for (int j = tid; j < it.np; j += kConsumers) {
                const int o = S.perm[it.io + j];
                for (int kr = 0; kr < nr; ++kr) zs[(int64_t)kr * S.n + o] = IO(x[j * nr + kr]);
            }
            for (int j = tid; j < it.nq; j += kConsumers) {
                const int o = S.perm[S.p + it.go + j];
                for (int kr = 0; kr < nr; ++kr) zs[(int64_t)kr * S.n + o] = IO(w[j * nr + kr]);
            }
        }
        csync();
    }
    return;
abort:
    consumers_abort_drain(c);
}

}  // namespace pslr
