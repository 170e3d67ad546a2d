"""The boundary from plain C: a C99 program that includes only
include/pslr.h and links libpslr.so builds a 2D shifted Laplacian in CSR,
runs pslr_plan (the host-side set-up: Section 2 reordering, local factors,
device layout; no GPU touched) and pslr_status_string, and prints what it
got.  The header must compile as C (no C++ or torch types) and the figures
must equal those of the Python binding on the same matrix."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from pslr_inputs import generators as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SRC = r"""
#include <stdio.h>
#include <stdlib.h>
#include "pslr.h"

int main(void) {
    const int nx = 20, ny = 18, n = nx * ny;
    int32_t *rp = malloc(sizeof(int32_t) * (n + 1)), *ci = malloc(sizeof(int32_t) * 5 * n);
    double *v = malloc(sizeof(double) * 5 * n);
    int32_t *part = malloc(sizeof(int32_t) * n), *iface = malloc(sizeof(int32_t) * n),
            *perm = malloc(sizeof(int32_t) * n);
    int k = 0;
    rp[0] = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {  /* columns ascending: -nx, -1, 0, +1, +nx */
            int r = i + nx * j;
            if (j > 0) { ci[k] = r - nx; v[k++] = -1.0; }
            if (i > 0) { ci[k] = r - 1; v[k++] = -1.0; }
            ci[k] = r; v[k++] = 4.0 - 0.1;
            if (i < nx - 1) { ci[k] = r + 1; v[k++] = -1.0; }
            if (j < ny - 1) { ci[k] = r + nx; v[k++] = -1.0; }
            rp[r + 1] = k;
        }
    pslr_opts o = {0};
    o.dims[0] = nx; o.dims[1] = ny; o.dims[2] = 1;
    o.splits[0] = 3; o.splits[1] = 2; o.splits[2] = 1;
    o.factor = 0;
    pslr_info info;
    pslr_status st = pslr_plan(n, rp, ci, v, &o, 3, 5, &info, part, iface, perm);
    printf("%d %s\n", (int)st, pslr_status_string(st));
    if (st != PSLR_OK) return 1;
    printf("%d %d %d %d %d %d\n", info.n, info.s, info.p, info.q, info.levels_B, info.levels_C0);
    printf("%lld %lld %llu\n", (long long)info.nnz_ilu, (long long)info.apply_bytes_fp64,
           (unsigned long long)info.layout_hash);
    long long sum = 0;
    for (int t = 0; t < n; ++t) sum += (long long)perm[t] * (t + 1) + part[t] * 7 + iface[t];
    printf("%lld\n", sum);
    o.factor = 5;  /* an invalid option is an error status, not a crash */
    st = pslr_plan(n, rp, ci, v, &o, 3, 5, &info, NULL, NULL, NULL);
    printf("%d %s\n", (int)st, pslr_status_string(st));
    free(rp); free(ci); free(v); free(part); free(iface); free(perm);
    return 0;
}
"""


def test_plan_from_plain_c(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2002_00917_gb300 import build, pslr

    build.build()
    libdir = os.path.join(ROOT, "paper_2002_00917_gb300")
    src = tmp_path / "plan.c"
    src.write_text(C_SRC)
    exe = tmp_path / "plan"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-lpslr", f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    assert out[0] == "0 ok"
    A = G.shifted_laplacian((20, 18), 0.1)
    info, part, iface, perm = pslr.plan(A, (20, 18, 1), (3, 2, 1), factor=0, m=3, rank=5)
    assert list(map(int, out[1].split())) == [info[k] for k in ("n", "s", "p", "q", "levels_B", "levels_C0")]
    nnz, nbytes, h = map(int, out[2].split())
    assert (nnz, nbytes, h) == (info["nnz_ilu"], info["apply_bytes_fp64"], info["layout_hash"])
    t = np.arange(1, A.n + 1, dtype=np.int64)
    assert int(out[3]) == int((perm.astype(np.int64) * t).sum() + 7 * part.sum() + iface.sum())
    assert out[4].startswith(f"{pslr.PSLR_ERR_ARG} ")
