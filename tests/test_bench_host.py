"""Host-side arithmetic of bench.py (no GPU): the per-pair operation counts of
the roofline, the roofline fields, the SM clock it charges, and the far-field
work of a batch taken from each cell's plan."""
import math

import pytest

import bench


def test_p2p_work_counts():
    # Laplace pot + grad over 9 images: 8 FP32 per pair + 3 per (t, s), rcp + lg2/9
    f, m = bench.p2p_work("laplace", 1, True, 9)
    assert f == pytest.approx(8 + 3 / 9) and m == pytest.approx(1 + 1 / 9)
    # the singly periodic strip shares one lg2 over 3 images
    f, m = bench.p2p_work("laplace", 1, True, 3)
    assert f == pytest.approx(8 + 1) and m == pytest.approx(1 + 1 / 3)
    # tree-code leaves: one image per pair
    assert bench.p2p_work("laplace_leaf", 1, True) == (13.0, 2.0)
    assert bench.p2p_work("stokes_leaf", 1, False) == (17.0, 2.0)
    # modified Helmholtz, 8 rhs: the rhs FMAs are shared by the 9 images
    f, m = bench.p2p_work("modhelm", 8, False, 9)
    assert f == pytest.approx(16 + 8 / 9) and m == 2.5


def test_roofline_fields_and_clock():
    clocks = {"sm_mhz": 1500.0, "sm_max_mhz": 2070.0}
    r = bench.p2p_roofline("laplace_leaf", 1, True, 1.0e9, 2.0, 4.0, "leaves", 152, clocks)
    rates = bench.alu_rates()
    # the bound charges the sampled clock, not the maximum
    peak = 152 * min(rates["fp32"] / 13.0, rates["mufu"] / 2.0) * 1500.0 * 1e6 / 1e9
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(1.0e9 / 2.0e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["share_of_step"] == pytest.approx(0.5)
    assert r["bound"] == "alu" and r["unit"] == "Gpair/s"
    # without samples: the maximum clock nvidia-smi reported
    mhz, src = bench.peak_clock_mhz({"sm_max_mhz": 2070.0})
    assert mhz == 2070.0 and "maximum" in src


def test_far_units_from_plans():
    """Direct far-field work per cell: (2 Nq + 2 (M - m_lo + 1)) terms per point on the
    direct path, 2 Nq on the NUFFT path; the totals grow with the cells."""
    import workloads
    cells = workloads.batch_cells(ncell=6, seed=3, nrhs=8, scale=0.02)
    ev, fo, nnu = bench.far_units("modhelm", cells, 1.0, 8)
    assert ev == fo and ev > 0 and 0 <= nnu <= len(cells)
    ev2, _, _ = bench.far_units("modhelm", cells[:3], 1.0, 8)
    assert 0 < ev2 < ev
    # at beta = 100 the far field of these cells is dropped entirely (Eq. mpk0s bound)
    ev100, _, _ = bench.far_units("modhelm", cells, 100.0, 8)
    assert ev100 < ev
    n = sum(c["src"].shape[1] for c in cells)
    assert ev % 1 == 0 and ev >= 2 * n  # at least two terms per point
    assert math.isfinite(ev)
