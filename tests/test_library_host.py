"""Host-only checks of the C-ABI library (no GPU needed).

* the shared library loads and exports every function declared in include/pfmm.h
* plan parameters: canonical cell, m0, M from Eq. mpk0s, west/east nodes
* argument validation happens on the host before any launch
"""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2111_01083_gb300.build import build_library
    from paper_2111_01083_gb300 import _lib
    build_library()
    return _lib.lib()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(pfmm_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    from paper_2111_01083_gb300 import _lib
    assert set(_lib.EXPORTS) == set(names)


def test_version(L):
    assert b"sm_103a" in L.pfmm_version()


def _op(**kw):
    from paper_2111_01083_gb300 import PeriodicOp
    base = dict(kernel="laplace", e1=(1.0, 0.0), e2=(0.0, 1.0), tol=1e-6, ns_max=100, nt_max=100)
    base.update(kw)
    return PeriodicOp(**base)


def _mpk0s(d, eta, eps):
    r = 2 * math.pi * eta / d
    return math.ceil(d / (2 * math.pi * eta) * math.log(1 / ((1 - math.exp(-r)) * eps)))


@pytest.mark.parametrize("e1,e2", [
    ((1.0, 0.0), (0.0, 1.0)), ((0.0, 2.0), (1.0, 0.0)), ((1.0, 0.0), (0.3, 0.8)),
    ((1.0, 0.0), (0.45, 0.8)), ((1.0, 0.0), (5.3, 0.8)), ((16.0, 0.0), (0.0, 1.0)),
    ((1.0, 0.0), (0.5, 0.866)), ((2.0, 0.5), (-0.4, 1.7)),
])
def test_canonical_cell_and_m0(L, e1, e2):
    """Library canonicalisation vs the oracle's independent implementation."""
    from oracle import lattice
    c = lattice.canonicalize(e1, e2)
    d, xi, eta = c["d"], c["xi"], c["eta"]
    rot, m0 = lattice.choose_we(d, xi, "auto")
    desc = _op(e1=e1, e2=e2).describe()
    assert abs(desc["d"] - d) < 1e-12 and abs(abs(desc["xi"]) - abs(xi)) < 1e-12 and abs(desc["eta"] - eta) < 1e-12
    assert desc["m0"] == m0 and desc["we_rotated"] == int(rot)
    r = desc["rot"]
    # rot is a rotation and maps a lattice vector of length d onto the x axis
    assert abs(r[0] * r[3] - r[1] * r[2] - 1) < 1e-12 and abs(r[0] * r[1] + r[2] * r[3]) < 1e-12
    ok = False
    for a, b in ((1, 0), (0, 1), (1, 1), (1, -1), (1, -5), (-5, 1)):
        v = (a * e1[0] + b * e2[0], a * e1[1] + b * e2[1])
        x = r[0] * v[0] + r[1] * v[1]
        y = r[2] * v[0] + r[3] * v[1]
        ok |= abs(abs(x) - d) < 1e-9 and abs(y) < 1e-9
    assert ok


def test_west_east_direction_flags(L):
    """App. A: WE_ROTATED gives the 3 x 3 near block on any cell, with the
    frame (cos, sin) = (eta, xi)/|e2|; WE_AXIS keeps m0 = 2 on the hexagonal
    cell; the default rotates exactly there."""
    hexe2 = (0.5, math.sqrt(3) / 2)
    r = _op(e2=hexe2, we="rotated").describe()
    a = _op(e2=hexe2, we="axis").describe()
    dflt = _op(e2=hexe2).describe()
    assert (r["m0"], r["we_rotated"]) == (1, 1) and (a["m0"], a["we_rotated"]) == (2, 0)
    assert (dflt["m0"], dflt["we_rotated"]) == (1, 1)
    h = math.hypot(r["xi"], r["eta"])
    assert abs(r["we_dir"][0] - r["eta"] / h) < 1e-14 and abs(r["we_dir"][1] - r["xi"] / h) < 1e-14
    assert a["we_dir"] == [1.0, 0.0]
    sq = _op(we="rotated").describe()  # rectangle: the rotated frame is the axis frame
    assert sq["m0"] == 1 and sq["we_dir"] == [1.0, 0.0] and sq["Nq"] == _op().describe()["Nq"]
    skew = _op(e2=(0.3, 0.8)).describe()
    assert (skew["m0"], skew["we_rotated"]) == (1, 0)


@pytest.mark.parametrize("kw", [dict(flags=96), dict(flags=1024), dict(flags=48)])
def test_west_east_flag_errors(L, kw):
    from paper_2111_01083_gb300 import _lib
    o = _lib.Opts()
    o.e1[0], o.e1[1], o.e2[0], o.e2[1] = 1.0, 0.0, 0.0, 1.0
    o.kernel, o.tol, o.precision, o.path, o.nrhs = 0, 1e-6, 1, 1, 1
    o.flags = kw["flags"]  # both directions / unknown bit / rotated singly periodic
    h = ctypes.c_void_p()
    assert L.pfmm_plan_create(ctypes.byref(o), 10, 10, ctypes.byref(h)) == 1  # PFMM_ERR_INVALID_ARG


def test_mstokes_plan(L):
    """Modified Stokes: two plane-wave families (beta: m = 0..M, Laplace:
    m = 1..M, each with its west/east nodes); AUTO takes the NUFFT like the
    other kernels; the singly periodic operator and beta <= 0 are refused."""
    from paper_2111_01083_gb300 import _lib
    d = _op(kernel="mstokes", beta=2.0, e1=(40.0, 0.0)).describe()
    lap = _op(kernel="laplace", e1=(40.0, 0.0)).describe()
    assert d["path"] == 2 and lap["path"] == 2
    assert _op(kernel="mstokes", beta=2.0).describe()["path"] == 1
    assert d["M"] == lap["M"] and d["mode0"] == 1
    mh = _op(kernel="modhelm", beta=2.0, e1=(40.0, 0.0), path="direct").describe()
    assert d["Nq"] > mh["Nq"]  # both families' nodes
    for kw in (dict(singly=True), dict(beta=0.0)):
        args = dict(kernel="mstokes", beta=2.0)
        args.update(kw)
        with pytest.raises(_lib.PfmmError):
            _op(**args)


@pytest.mark.parametrize("d,tol", [(1.0, 1e-10), (16.0, 1e-6), (64.0, 1e-6)])
def test_modes_follow_mpk0s(L, d, tol):
    desc = _op(e1=(d, 0.0), e2=(0.0, 1.0), tol=tol).describe()
    assert desc["M"] == _mpk0s(d, 1.0, tol / 10)
    assert desc["Nq"] > 0 and desc["mode0"] == 1


def test_modhelm_pruning(L):
    big = _op(kernel="modhelm", beta=100.0, e1=(3.0, 0.0)).describe()
    assert big["M"] == 0 and big["mode0"] == 0 and big["Nq"] == 0
    small = _op(kernel="modhelm", beta=1.0, e1=(16.0, 0.0)).describe()
    assert 0 < small["M"] <= _mpk0s(16.0, 1.0, 1e-7)


def test_nufft_parameters(L):
    desc = _op(e1=(16.0, 0.0), path="nufft", nufft_w=8, n_gl=8).describe()
    assert desc["path"] == 2 and desc["nufft_w"] == 8 and desc["n_gl"] == 8
    nf = desc["nf"]
    assert nf & (nf - 1) == 0 and nf >= 2 * (2 * desc["M"] + 1)


@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 0.5), ("stokes", 0.0)])
def test_auto_path_picks_nufft_for_many_modes(L, kernel, beta):
    """AUTO takes the NUFFT path once M >= 64, for every kernel, and the direct
    path for a square cell."""
    long = _op(kernel=kernel, beta=beta, e1=(40.0, 0.0)).describe()
    assert long["M"] >= 64 and long["path"] == 2
    assert _op(kernel=kernel, beta=max(beta, 0.5) if kernel == "modhelm" else 0.0).describe()["path"] == 1


@pytest.mark.parametrize("kw,code", [
    (dict(e1=(1.0, 0.0), e2=(2.0, 0.0)), 2),
    (dict(tol=0.5), 4),
    (dict(tol=1e-16), 4),
    (dict(kernel="modhelm", beta=0.0), 1),
    (dict(nrhs=0), 1),
    (dict(e1=(2000.0, 0.0), path="nufft"), 1),  # fine grid above 8192 points
])
def test_host_validation(L, kw, code):
    from paper_2111_01083_gb300._lib import PfmmError
    with pytest.raises(PfmmError) as ei:
        _op(**kw)
    assert ei.value.code == code


def test_execute_rejects_bad_workspace_before_launch(L):
    op = _op()
    # NULL workspace: rejected on the host, nothing launched
    code = L.pfmm_execute(op._h, None, 0, 10, None, None, 10, None, None, None, None)
    assert code in (1, 5)
    code = L.pfmm_execute(op._h, ctypes.c_void_p(256), 1 << 40, 1000, None, None, 10, None, None, None, None)
    assert code == 1  # ns beyond the plan maximum


def test_workspace_size_grows_with_n(L):
    a = _op(ns_max=1000, nt_max=1000).ws_bytes
    b = _op(ns_max=100000, nt_max=100000).ws_bytes
    assert b > 50 * a / 2


def test_singly_periodic_plan(L):
    """P1: 3 near images, no south/north modes; west/east nodes grow for a
    tall strip, and AUTO then takes the west/east sums through the transforms
    (nodes above (w/2 + 2) pi / eta; the rest stay direct); a wide strip has no
    node above that cut and stays on the direct path even when NUFFT is asked for."""
    from paper_2111_01083_gb300 import PeriodicOp
    wide = PeriodicOp("laplace", (1.0, 0.0), (0.3, 0.5), singly=True, ns_max=8, nt_max=8).describe()
    assert wide["M"] == 0 and wide["path"] == 1 and wide["m0"] == 1 and wide["Nq"] > 0
    assert abs(wide["d"] - 1.0) < 1e-15 and abs(wide["eta"] - 0.5) < 1e-15 and wide["xi"] == 0.0
    assert wide["p1_nufft_nodes"] == 0
    forced = PeriodicOp("laplace", (1.0, 0.0), (0.3, 0.5), singly=True, path="nufft", ns_max=8, nt_max=8).describe()
    assert forced["path"] == 1 and forced["p1_nufft_nodes"] == 0
    tall = PeriodicOp("laplace", (1.0, 0.0), (0.0, 20.0), singly=True, ns_max=8, nt_max=8).describe()
    assert tall["Nq"] > wide["Nq"]
    assert tall["path"] == 2 and 128 <= tall["p1_nufft_nodes"] < tall["Nq"] and tall["M"] == 0
    w = tall["nufft_w"]
    # uniform frequencies u pi / eta up to the top node plus the kernel's half-width
    assert tall["nf"] <= 8192 and tall["nf"] >= 2 * (2 * int(16.1 * 20 / math.pi) + 1)
    direct = PeriodicOp("laplace", (1.0, 0.0), (0.0, 20.0), singly=True, path="direct", ns_max=8, nt_max=8).describe()
    assert direct["path"] == 1 and direct["p1_nufft_nodes"] == 0 and direct["Nq"] == tall["Nq"]
    mid = PeriodicOp("stokes", (1.0, 0.0), (0.0, 2.0), singly=True, path="nufft", ns_max=8, nt_max=8).describe()
    assert mid["path"] == 2 and 0 < mid["p1_nufft_nodes"] < mid["Nq"] and w == mid["nufft_w"]


@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 1.0), ("stokes", 0.0), ("mstokes", 1.0)])
def test_plans_for_the_paper_cells(L, kernel, beta):
    """Every cell of the paper's Tables 1-3 (rectangles and theta = pi/3, pi/6
    parallelograms, A = d/eta up to 1000, eta = 1) plans without error at the
    tables' precisions: near block 3 x 3 (m0 = 1) after reduction and the
    west/east direction rule, M from Eq. mpk0s on the reduced cell, a NUFFT
    fine grid that fits the single-block FFT whenever AUTO picks the NUFFT
    (longer cells at high precision take the direct path), and a workspace
    linear in the point count."""
    from oracle import lattice
    for shape in ("rectangle", math.pi / 3, math.pi / 6):
        for A in (1, 2, 10, 100, 1000):
            e1 = (float(A), 0.0)
            e2 = (0.0, 1.0) if shape == "rectangle" else (1.0 / math.tan(shape), 1.0)
            for tol in (1e-12, 1e-9, 1e-6):
                d = _op(kernel=kernel, beta=beta, e1=e1, e2=e2, tol=tol, ns_max=1000, nt_max=1000).describe()
                c = lattice.canonicalize(e1, e2)
                assert d["m0"] == 1
                if kernel in ("laplace", "stokes", "mstokes"):
                    assert d["M"] == _mpk0s(c["d"], c["eta"], tol / 10)
                # modified Helmholtz: no west/east nodes once the far columns are
                # beyond the K0 decay (beta d large)
                assert d["Nq"] < 4000 and (d["Nq"] > 0 or kernel == "modhelm")
                if d["path"] == 2:
                    assert d["nf"] <= 8192 and d["nf"] >= 2 * (2 * d["M"] + 1)
    small = _op(kernel=kernel, beta=beta, e1=(100.0, 0.0), tol=1e-9, ns_max=1000, nt_max=1000)
    big = _op(kernel=kernel, beta=beta, e1=(100.0, 0.0), tol=1e-9, ns_max=100000, nt_max=100000)
    assert big.ws_bytes < 150 * small.ws_bytes


def test_binding_validates_tensors():
    """The binding refuses tensors the library would misread (wrong dtype,
    shape, device or layout) before any call; checked on CPU tensors."""
    import torch
    from paper_2111_01083_gb300.periodic import check_inputs
    src = torch.zeros(2, 10, dtype=torch.float64)
    q = torch.zeros(3, 10, dtype=torch.float64)
    assert check_inputs("laplace", 3, src, q, None) == (10, 10)
    assert check_inputs("laplace", 3, src, q, torch.zeros(2, 4, dtype=torch.float64)) == (10, 4)
    f = torch.zeros(3, 2, 10, dtype=torch.float64)
    assert check_inputs("mstokes", 3, src, f, None) == (10, 10)
    bad = [
        ("laplace", q.float(), None, None),                                # dtype
        ("laplace", torch.zeros(3, 9, dtype=torch.float64), None, None),  # ns mismatch
        ("laplace", torch.zeros(2, 10, dtype=torch.float64), None, None), # nrhs mismatch
        ("stokes", q, None, None),                                        # forces need [nrhs, 2, ns]
        ("laplace", torch.zeros(10, 3, dtype=torch.float64).t(), None, None),  # not contiguous
        ("laplace", q, torch.zeros(3, 4, dtype=torch.float64), None),     # trg not [2, nt]
        ("laplace", q, None, (torch.zeros(3, 9, dtype=torch.float64), None)),  # out pot shape
        ("stokes", f, None, (torch.zeros(3, 2, 10, dtype=torch.float64),
                             torch.zeros(3, 2, 10, dtype=torch.float64))),    # grad out for Stokes
    ]
    for kernel, qq, trg, out in bad:
        with pytest.raises(ValueError):
            check_inputs(kernel, 3, src, qq, trg, out)


def test_near_field_mode_selection(L):
    """The tree code runs the near field of large mixed Laplace/Stokes plans by
    default; the flags force either sum; other kernels and FP64 stay direct."""
    big = dict(ns_max=100000, nt_max=100000)
    assert _op(**big).describe()["near_fmm"] == 1
    assert _op(kernel="stokes", **big).describe()["near_fmm"] == 1
    assert _op(**big, near="direct").describe()["near_fmm"] == 0
    assert _op(**big, precision="fp64").describe()["near_fmm"] == 0
    assert _op(kernel="modhelm", beta=1.0, **big).describe()["near_fmm"] == 0
    # small problems: direct unless forced
    assert _op().describe()["near_fmm"] == 0
    d = _op(near="fmm").describe()
    assert d["near_fmm"] == 1 and d["near_theta"] == 0.5 and d["near_leaf"] == 128
    # expansion terms from the tolerance (theta^p <= tol / 10), rounded up to a compiled order
    assert _op(near="fmm", tol=1e-6).describe()["near_order"] == 24
    assert _op(near="fmm", tol=1e-2).describe()["near_order"] == 12
    assert _op(near="fmm", near_order=14).describe()["near_order"] == 16
    assert _op(near="fmm", near_leaf=16).describe()["near_leaf"] == 16
    # the tree code's workspace only when it runs
    assert _op(near="fmm").ws_bytes > _op(near="direct").ws_bytes


@pytest.mark.parametrize("kw", [dict(near_order=7), dict(near_order=33), dict(near_leaf=4), dict(near_leaf=2000)])
def test_near_field_option_errors(L, kw):
    from paper_2111_01083_gb300 import _lib
    with pytest.raises(_lib.PfmmError) as ei:
        _op(near="fmm", **kw)
    assert ei.value.code == 1


def test_near_field_flags_exclusive(L):
    from paper_2111_01083_gb300 import _lib
    o = _lib.Opts()
    o.e1[0], o.e2[1] = 1.0, 1.0
    o.tol, o.precision, o.nrhs = 1e-6, 1, 1
    o.flags = _lib.PFMM_NEAR_DIRECT | _lib.PFMM_NEAR_FMM
    h = ctypes.c_void_p()
    assert L.pfmm_plan_create(ctypes.byref(o), 10, 10, ctypes.byref(h)) == 1
    o.flags = 1024
    assert L.pfmm_plan_create(ctypes.byref(o), 10, 10, ctypes.byref(h)) == 1


def test_near_stats_requires_tree_code(L):
    op = _op(near="direct")
    out = (ctypes.c_int64 * 5)()
    assert L.pfmm_near_stats(op._h, ctypes.c_void_p(256), None, out) == 1


def test_deterministic_plans(L):
    """PFMM_DETERMINISTIC: the direct far path and the direct near sum; the
    NUFFT path or the tree code with it are argument errors; batches refuse it."""
    from paper_2111_01083_gb300 import BatchOp, _lib
    big = dict(e1=(16.0, 0.0), ns_max=100000, nt_max=100000)
    d = _op(**big, deterministic=True).describe()
    assert d["path"] == 1 and d["near_fmm"] == 0
    assert _op(**big).describe()["path"] == 1 or _op(**big).describe()["M"] < 64
    assert _op(e1=(64.0, 0.0), ns_max=1000, nt_max=1000).describe()["path"] == 2
    assert _op(e1=(64.0, 0.0), ns_max=1000, nt_max=1000, deterministic=True).describe()["path"] == 1
    for kw in (dict(path="nufft"), dict(near="fmm")):
        with pytest.raises(_lib.PfmmError) as ei:
            _op(deterministic=True, **kw)
        assert ei.value.code == 1
    o = _lib.Opts()
    o.e1[0], o.e2[1] = 1.0, 1.0
    o.tol, o.precision, o.nrhs, o.kernel = 1e-6, 1, 1, 0
    o.flags = _lib.PFMM_DETERMINISTIC
    arr = (_lib.Opts * 1)(o)
    so = (ctypes.c_int64 * 2)(0, 10)
    h = ctypes.c_void_p()
    assert L.pfmm_batch_create(arr, 1, so, None, 0, ctypes.byref(h)) == 1


def test_batch_create_is_host_only(L):
    """pfmm_batch_create sizes the workspace, including the argument tables of
    the multi-cell launches (a recording of every cell's launches with
    placeholder addresses), without touching a GPU: mixed batches of all four
    kernels, NUFFT and direct cells, self and separate targets."""
    import numpy as np
    import workloads
    from paper_2111_01083_gb300 import BatchOp
    cells = workloads.batch_cells(ncell=12, seed=3, nrhs=8, scale=0.05)
    counts = [c["src"].shape[1] for c in cells]
    sizes = {}
    for kernel, beta, nrhs in (("modhelm", 1.0, 8), ("laplace", 0.0, 1), ("stokes", 0.0, 2), ("mstokes", 2.0, 1)):
        op = BatchOp(kernel, [dict(e1=c["e1"], e2=c["e2"], beta=beta) for c in cells], counts, precision="mixed",
                     nrhs=nrhs)
        assert op.ws_bytes > 0 and op.ws_bytes % 256 == 0
        sizes[kernel] = op.ws_bytes
    # separate targets and a forced NUFFT cell
    trg = [max(1, n // 2) for n in counts]
    cl = [dict(e1=c["e1"], e2=c["e2"], beta=1.0) for c in cells]
    cl[0]["path"] = "nufft"
    op = BatchOp("modhelm", cl, counts, trg_counts=trg, precision="mixed", nrhs=8)
    assert op.ws_bytes > 0
    # more cells need more table space
    op2 = BatchOp("modhelm", [dict(e1=c["e1"], e2=c["e2"], beta=1.0) for c in cells[:4]], counts[:4],
                  precision="mixed", nrhs=8)
    assert op2.ws_bytes < sizes["modhelm"]
