// Host-side view of one set-up context, for the batched entry points
// (pslr_batch_host.cpp): sizes, device maps and matrices, the low-rank term
// and the forward segment tables, without exposing the context's layout.
#pragma once
#include <cstdint>
#include <vector>

#include "pslr.h"
#include "pslr_internal.h"

namespace pslr {

struct SysExport {
    int n, s, p, q, m, r, factor, max_p, max_q;
    const int32_t *ioff, *goff, *perm;      // device
    const int32_t *rp, *ci;                 // device CSR of A (original ordering)
    const double *av;
    const double *V;                        // device q x r FP64, row-major (row stride ldv)
    const uint16_t *Vb;                     // device q x r BF16, row-major (row stride ldv)
    int ldv;                                // r rounded up to a multiple of 8 (zero padded)
    const double *G;                        // device r x r
    const float *Gf;
    const char *seg[2];                     // device forward segments [FP64, FP32]
    const int32_t *cnt[2];                  // device kNCnt*s segment counts [FP64, FP32]
    int slot_bytes[2];
    uint64_t lr_gen;                        // changes whenever the low-rank term is replaced
    double omega;                           // 1 unless the context applies the Neumann polynomial
    int64_t seg_bytes[2];                   // bytes of the forward segments
    std::vector<int32_t> ioff_h, goff_h;    // host copies of the s+1 interior / interface offsets
};

// Fill e from a set-up context; false when the context has no device state.
bool sys_export(const pslr_ctx *c, SysExport *e);

// Append to out the forward segments of category cat (kE .. kC2) of subdomain
// i in precision prec, as stream entries whose offsets are relative to the
// context's segment base plus shift.
void sys_segments(const pslr_ctx *c, int prec, int i, int cat, int64_t shift, std::vector<StreamEnt> &out);

// Low-rank generation of a context (see SysExport::lr_gen).
uint64_t sys_lr_gen(const pslr_ctx *c);

}  // namespace pslr
