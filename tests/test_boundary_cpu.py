"""The C-ABI library on a machine without a GPU: it loads, exports every entry
point include/pslr.h declares, and its host-side set-up (pslr_plan: Section 2
reordering, local factors, layout) agrees bit for bit with the oracle."""
import os
import re

import numpy as np
import pytest

import oracle as O
from pslr_inputs import configs as C
from pslr_inputs import generators as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pslr():
    from paper_2002_00917_gb300 import build, pslr

    build.build()
    pslr.load()
    return pslr


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(pslr_\w+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(pslr):
    lib = pslr.load()
    names = declared_functions()
    assert {"pslr_setup", "pslr_apply", "pslr_apply_T", "pslr_build_lowrank", "pslr_solve"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


CASES = [
    ("lap", (32, 32), (2, 2), 1),
    ("lap", (13, 11, 9), (3, 2, 2), 0),
    ("cd", (12, 10, 8), (3, 2, 2), 0),
    ("kappa", (10, 9, 11), (2, 3, 2), 0),
    ("lap", (7, 6, 5), (7, 6, 5), 0),
    ("cd", (9, 9, 9), (1, 1, 1), 0),
]


@pytest.mark.parametrize("kind,dims,splits,factor", CASES)
def test_plan_maps_bit_exact_with_oracle(pslr, kind, dims, splits, factor):
    w = C.small_problem(kind, dims, splits, factor=factor, K=3)
    info, part, iface, perm = pslr.plan(w["A"], w["dims"], w["splits"], factor=factor, m=3, rank=4)
    o = O.from_workload(w)
    op, oi, operm = o.maps()
    np.testing.assert_array_equal(part, op)
    np.testing.assert_array_equal(iface, oi)
    np.testing.assert_array_equal(perm, operm)
    assert (info["n"], info["s"], info["p"], info["q"]) == (o.n, o.s, o.p, o.q)
    io, go = o.offsets()
    assert info["max_interior"] == int(np.diff(io).max())
    assert info["max_interface"] == int(np.diff(go).max())
    if factor == 0:
        nnz = o.block("LU_B")[1].size + o.block("LU_C0")[1].size
        assert info["nnz_ilu"] == nnz  # ILU(0) keeps the pattern of B and C0
    assert info["apply_bytes_fp64"] > info["apply_bytes_fp32"] > 0


def test_plan_user_partition_and_full_size_maps(pslr):
    w = C.lap3d_64_4x4x2_ilu0()
    info, part, iface, perm = pslr.plan(w["A"], w["dims"], w["splits"], m=3, rank=16)
    assert (info["n"], info["s"], info["p"], info["q"]) == (262144, 32, 208568, 53576)
    o = O.from_workload(w)
    for a, b in zip((part, iface, perm), o.maps()):
        np.testing.assert_array_equal(a, b)
    # a user partition equal to the geometric one gives the same maps
    info2, part2, iface2, perm2 = pslr.plan(w["A"], part=part, m=3, rank=16)
    np.testing.assert_array_equal(perm2, perm)
    assert info2["apply_bytes_fp64"] == info["apply_bytes_fp64"]


def test_plan_rejects_bad_input(pslr):
    A = G.shifted_laplacian((6, 5), 0.1)
    with pytest.raises(pslr.PslrError) as e:
        pslr.plan(A, (6, 4, 1), (2, 2, 1))
    assert e.value.status == pslr.PSLR_ERR_ARG
    bad = G.CSR(A.n, A.rowptr, A.col.copy(), A.val)
    bad.col[1], bad.col[2] = bad.col[2], bad.col[1]  # columns out of order
    with pytest.raises(pslr.PslrError) as e:
        pslr.plan(bad, (6, 5, 1), (2, 2, 1))
    assert e.value.status == pslr.PSLR_ERR_ARG
    zp = G.CSR(A.n, A.rowptr, A.col, A.val.copy())
    zp.val[zp.rowptr[0]] = 0.0
    with pytest.raises(pslr.PslrError) as e:
        pslr.plan(zp, (6, 5, 1), (2, 1, 1))
    assert e.value.status == pslr.PSLR_ERR_ZERO_PIVOT
    big = G.shifted_laplacian((200, 200), 0.1)  # one 40000-row subdomain exceeds shared memory
    with pytest.raises(pslr.PslrError) as e:
        pslr.plan(big, (200, 200, 1), (1, 1, 1))
    assert e.value.status == pslr.PSLR_ERR_TOO_LARGE


@pytest.mark.parametrize("kind,dims,splits,factor", [("lap", (16, 14, 12), (4, 3, 3), 0),
                                                     ("cd", (12, 11, 10), (3, 2, 2), 2),
                                                     ("lap", (32, 32), (2, 2), 1),
                                                     ("kappa", (10, 9, 11), (2, 3, 2), 0)])
@pytest.mark.parametrize("merge_levels", [0, 2])
def test_setup_threads_do_not_change_the_layout(pslr, kind, dims, splits, factor, merge_levels):
    """The set-up runs per subdomain on host threads; the packed device layout
    of both directions and precisions (its hash over every byte, descriptor
    and count), the fill and the levels are the same for 1, 2, 5 and all
    threads, with one level per sweep segment and with several."""
    w = C.small_problem(kind, dims, splits, factor=factor, drop_tol=1e-2)
    infos = []
    for t in (1, 2, 5, 0):
        info, part, iface, perm = pslr.plan(w["A"], w["dims"], w["splits"], factor=factor, m=3, rank=4,
                                            drop_tol=1e-2, setup_threads=t, merge_levels=merge_levels)
        assert info["setup_threads"] == (t if t else info["setup_threads"]) and info["setup_threads"] >= 1
        infos.append(({k: v for k, v in info.items() if k != "setup_threads"}, perm.tobytes()))
    assert infos[0][0]["layout_hash"] != 0
    assert all(x == infos[0] for x in infos[1:])


def test_setup_threads_argument_and_errors(pslr):
    """A negative thread count is an argument error; a zero pivot is reported
    with any thread count."""
    A = G.shifted_laplacian((12, 10), 0.1)
    with pytest.raises(pslr.PslrError) as e:
        pslr.plan(A, (12, 10, 1), (2, 2, 1), setup_threads=-1)
    assert e.value.status == pslr.PSLR_ERR_ARG
    _, part, iface, perm = pslr.plan(A, (12, 10, 1), (2, 2, 1))
    zp = G.CSR(A.n, A.rowptr, A.col, A.val.copy())
    # the first interior row of subdomains 1 and 3 loses its diagonal: nothing
    # is eliminated before it, so its pivot is exactly zero
    for sub in (1, 3):
        v = next(int(u) for u in perm if part[u] == sub and not iface[u])
        row = slice(zp.rowptr[v], zp.rowptr[v + 1])
        zp.val[row][zp.col[row] == v] = 0.0
    for t in (1, 4):
        with pytest.raises(pslr.PslrError) as e:
            pslr.plan(zp, (12, 10, 1), (2, 2, 1), setup_threads=t)
        assert e.value.status == pslr.PSLR_ERR_ZERO_PIVOT


@pytest.mark.parametrize("graph,k", [("rgg2000", 7), ("rgg20000", 16), ("rgg20000", 5), ("grid2d", 4),
                                     ("grid3d", 6), ("cd3d", 9)])
def test_graph_partition_bit_exact_with_oracle(pslr, graph, k):
    """The library's graph partition (nparts, no dims) and the oracle's
    independent implementation give the same part of every vertex, with any
    number of set-up threads, and the reordering built on it the same maps."""
    if graph.startswith("rgg"):
        A = G.random_geometric_laplacian(int(graph[3:]), 12.0, 0.0064, 0)
    elif graph == "grid2d":
        A = G.shifted_laplacian((13, 11), 0.1)
    elif graph == "grid3d":
        A = G.shifted_laplacian((9, 8, 7), 0.1)
    else:
        A = G.convection_diffusion((8, 7, 6), 50.0, 0.1)
    info, part, iface, perm = pslr.plan(A, nparts=k)
    po = O.graph_partition(A, k)
    assert np.array_equal(part, po)
    for t in (1, 3):  # the cuts below the first run on host threads
        assert np.array_equal(pslr.plan(A, nparts=k, setup_threads=t)[1], po)
    o = O.Oracle(A, part=po)
    for a, b in zip((part, iface, perm), o.maps()):
        assert np.array_equal(a, b)
    assert info["s"] == k


@pytest.mark.parametrize("kind,dims,splits,factor", [("lap", (32, 32), (2, 2), 1), ("lap", (13, 11, 9), (3, 2, 2), 0),
                                                     ("cd", (12, 10, 8), (3, 2, 2), 2), ("kappa", (10, 9, 11), (2, 3, 2), 0),
                                                     ("lap", (40, 33), (3, 4), 0), ("cd", (9, 9, 9), (1, 1, 1), 0),
                                                     ("lap", (7, 6, 5), (7, 6, 5), 0), ("lap", (13, 11, 9), (3, 2, 2), 2)])
@pytest.mark.parametrize("merge_levels", [0, 2])
def test_layout_check_finds_no_violation(pslr, kind, dims, splits, factor, merge_levels):
    """The host-side decode of every packed segment (both directions, both
    precisions) finds every index in range, no product writing a row twice,
    and every sweep row reading only rows written at an earlier barrier
    step: the level schedules the kernels run are race-free.  The same holds
    for sweep segments that carry several levels (merge_levels = 2), whose
    blocks must also fill their segment exactly."""
    w = C.small_problem(kind, dims, splits, factor=factor, drop_tol=1e-2)
    info = pslr.plan(w["A"], w["dims"], w["splits"], factor=factor, m=3, rank=4, drop_tol=1e-2,
                     merge_levels=merge_levels)[0]
    assert info["layout_errors"] == 0
    assert info["merged"] == [int(merge_levels == 2)] * 2
    assert info["unit_sweeps"] == int(factor != 1)  # no row pivots: the unit-diagonal forward FP64 set


def test_merge_levels_option(pslr):
    """Automatic merging only where the ring is shallow: the 128^3
    convection-diffusion problem (256 subdomains, two CTAs per SM) merges its
    FP64 sweeps and not its FP32 ones; the 64^3 Laplacian (32 subdomains)
    merges neither.  Forcing either layout keeps the decode clean and changes
    the packed bytes; the maps are the same."""
    w = C.WORKLOADS["cd3d_128_8x8x4_ilu0"]()
    kw = dict(factor=w["factor"], m=w["m"], rank=w["rank"])
    got = {ml: pslr.plan(w["A"], w["dims"], w["splits"], merge_levels=ml, **kw) for ml in (0, 1, 2)}
    assert [got[ml][0]["merged"] for ml in (0, 1, 2)] == [[1, 0], [0, 0], [1, 1]]
    assert all(got[ml][0]["layout_errors"] == 0 for ml in (0, 1, 2))
    assert len({got[ml][0]["layout_hash"] for ml in (0, 1, 2)}) == 3
    for ml in (1, 2):
        assert all(np.array_equal(a, b) for a, b in zip(got[0][1:], got[ml][1:]))
    w = C.lap3d_64_4x4x2_ilu0()
    info = pslr.plan(w["A"], w["dims"], w["splits"], factor=w["factor"], m=w["m"], rank=w["rank"])[0]
    assert info["merged"] == [0, 0]
    A = G.shifted_laplacian((12, 10), 0.1)
    for ml in (-1, 3):
        with pytest.raises(pslr.PslrError) as e:
            pslr.plan(A, (12, 10, 1), (2, 2, 1), merge_levels=ml)
        assert e.value.status == pslr.PSLR_ERR_ARG


@pytest.mark.parametrize("name", ["lap3d_64_4x4x2_ilu0", "kappa3d_48_3x3x3", "lap3d_50_shift014", "rgg2d_20k"])
def test_layout_check_full_size(pslr, name):
    w = C.WORKLOADS[name]()
    info = pslr.plan(w["A"], w.get("dims", (0, 0, 0)), w.get("splits", (1, 1, 1)), factor=w["factor"], m=w["m"],
                     rank=w["rank"], drop_tol=w.get("drop_tol", 0.0), nparts=w.get("nparts", 0))[0]
    assert info["layout_errors"] == 0


def test_graph_partition_edge_cases(pslr):
    """One part (no interface), one vertex per part (no interior), and a graph
    with isolated vertices (components listed by their smallest vertex): the
    library agrees with the oracle."""
    A = G.shifted_laplacian((10, 9), 0.1)
    for k, q in ((1, 0), (A.n, A.n)):
        info, part, iface, perm = pslr.plan(A, nparts=k, m=2, rank=3)
        assert np.array_equal(part, O.graph_partition(A, k)) and info["q"] == q
    n = 30
    rows = list(range(n)) + [0, 1, 5, 6]
    cols = list(range(n)) + [1, 0, 6, 5]
    B = G._assemble(n, np.array(rows), np.array(cols), np.array([2.0] * n + [-1.0] * 4), None)
    for k in (3, 7):
        part = pslr.plan(B, nparts=k, m=1, rank=2)[1]
        assert np.array_equal(part, O.graph_partition(B, k))


def test_graph_partition_arguments(pslr):
    A = G.shifted_laplacian((4, 4), 0.0)
    for k in (17, -1):
        with pytest.raises(pslr.PslrError) as e:
            pslr.plan(A, nparts=k)
        assert e.value.status == pslr.PSLR_ERR_ARG


@pytest.mark.parametrize("kind,dims,splits,tau", [("lap", (9, 8, 7), (2, 2, 2), 1e-2),
                                                  ("cd", (8, 7, 6), (2, 2, 1), 1e-2),
                                                  ("kappa", (7, 8, 6), (2, 1, 2), 3e-3)])
def test_ilut_factors_have_the_oracles_pattern(kind, dims, splits, tau):
    """The library's ILUT (set-up on the host, dry run) keeps exactly as many
    entries as the oracle's independent ILUT: the same drop decisions."""
    from paper_2002_00917_gb300 import pslr

    w = C.small_problem(kind, dims, splits, factor=2, drop_tol=tau)
    info, *_ = pslr.plan(w["A"], w["dims"], w["splits"], factor=2, m=2, rank=0, drop_tol=tau)
    o = O.from_workload(w)
    nnz = sum(np.count_nonzero(o.dense_block(f)) for f in ("LU_B", "LU_C0"))
    assert info["nnz_ilu"] == nnz
    o0 = O.from_workload(dict(w, factor=0))
    assert nnz > sum(np.count_nonzero(o0.dense_block(f)) for f in ("LU_B", "LU_C0"))


def test_device_factor_option(pslr):
    """pslr_opts.device_factor: ILU(0) only, 0 or 1; the host-only dry run
    factors on the host and reports device_factor 0 with the same layout."""
    A = G.shifted_laplacian((12, 10), 0.1)
    base = pslr.plan(A, (12, 10, 1), (2, 2, 1))
    info, *maps = pslr.plan(A, (12, 10, 1), (2, 2, 1), device_factor=1)
    assert info["device_factor"] == 0 and info["layout_hash"] == base[0]["layout_hash"]
    for bad in (dict(device_factor=2), dict(device_factor=-1), dict(device_factor=1, factor=2, drop_tol=0.01),
                dict(device_factor=1, factor=1)):
        with pytest.raises(pslr.PslrError) as e:
            pslr.plan(A, (12, 10, 1), (2, 2, 1), **bad)
        assert e.value.status == pslr.PSLR_ERR_ARG


def test_ilu0_device_rejects_bad_patterns_before_any_device_work(pslr):
    """pslr_ilu0_device checks the block-diagonal pattern on the host and
    returns PSLR_ERR_ARG without touching the device (so this runs without a
    GPU): bad block pointers, a column outside its row's block, columns out
    of order, a missing diagonal, negative sizes."""
    lib = pslr.load()
    val = np.ones(16)  # never read: every case fails on the host

    def call(n, bptr, rp, ci):
        bp = np.ascontiguousarray(bptr, np.int32)
        r = np.ascontiguousarray(rp, np.int32)
        c = np.ascontiguousarray(ci if len(ci) else [0], np.int32)
        return lib.pslr_ilu0_device(n, len(bp) - 1, bp.ctypes.data, r.ctypes.data, c.ctypes.data,
                                    val.ctypes.data, None)

    # two 2x2 blocks, full within each block: a valid pattern for reference
    rp, ci = [0, 2, 4, 6, 8], [0, 1, 0, 1, 2, 3, 2, 3]
    cases = [
        (4, [0, 2], rp, ci),              # block_ptr does not end at n
        (4, [0, 3, 2, 4], rp, ci),        # block_ptr not monotone
        (4, [1, 2, 4], rp, ci),           # block_ptr does not start at 0
        (4, [0, 1, 4], rp, ci),           # row 0 reaches column 1 in the next block
        (4, [0, 2, 4], rp, [1, 0, 0, 1, 2, 3, 2, 3]),   # row 0's columns descending
        (4, [0, 2, 4], [0, 1, 3, 5, 7], [1, 0, 1, 2, 3, 2, 3]),  # row 0 without its diagonal
        (4, [0, 2, 4], [0, 2, 4, 3, 8], ci),  # rowptr not monotone
    ]
    for n, bptr, r, c in cases:
        assert call(n, bptr, r, c) == pslr.PSLR_ERR_ARG, (bptr, r, c)
    assert lib.pslr_ilu0_device(-1, 1, val.ctypes.data, val.ctypes.data, val.ctypes.data, val.ctypes.data,
                                None) == pslr.PSLR_ERR_ARG
    assert lib.pslr_ilu0_device(4, 2, None, val.ctypes.data, val.ctypes.data, val.ctypes.data,
                                None) == pslr.PSLR_ERR_ARG
    # an empty matrix is a valid (empty) factorization
    z = np.zeros(1, np.int32)
    assert lib.pslr_ilu0_device(0, 0, z.ctypes.data, z.ctypes.data, None, None, None) == pslr.PSLR_OK
