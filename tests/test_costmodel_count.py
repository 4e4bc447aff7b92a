"""The ALU roofline's operation count (paper_1808_04960_gb300/costmodel.py) against the
FP64 oracle's own tally: the oracle built with -DORACLE_COUNT_OPS counts every
floating-point operation it executes for one SSP-RK3 step, and the leading term per
cell and stage must equal the closed form exactly, for R = 1, 2, 3 in 1D, 2D and 3D."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1808_04960_gb300 import costmodel
from paper_1808_04960_gb300 import workloads as W


@pytest.mark.parametrize("ndim", [1, 2, 3])
@pytest.mark.parametrize("R", [1, 2, 3])
@pytest.mark.parametrize("flux", ["lf", "hllc", "hll"])
def test_closed_form_equals_oracle_tally(R, ndim, flux):
    counted = oracle.ops_per_cell_stage(R, ndim, flux=flux)
    assert counted == costmodel.flops_per_cell_stage(R, ndim, flux=flux)


@pytest.mark.parametrize("R", [1, 2, 3])
def test_variants_equal_oracle_tally(R):
    """Non-zero-mean smoothness indicators (separate windows) and polynomial candidates
    (same work as the GP ones, other tables)."""
    assert oracle.ops_per_cell_stage(R, 2, beta_mean=True) == costmodel.flops_per_cell_stage(R, 2, beta_mean=True)
    assert oracle.ops_per_cell_stage(R, 2, candidates="poly") == costmodel.flops_per_cell_stage(R, 2)


def test_default_count_value():
    """The count the headline roofline uses: 2D, R = 2, Lax-Friedrichs."""
    assert costmodel.flops_per_cell_stage(2, 2) == 1676


def test_counting_build_computes_the_same_numbers():
    """The tally only observes: the counting build's step is bitwise the normal build's."""
    U, meta = W.smooth_field((20, 24), seed=3)
    o = oracle.Oracle(U.shape[1:], meta["dx"], meta["bc"], R=2)
    ref = o.rk3_step(U, 1e-3)
    lib = oracle._load_ops()
    V = np.ascontiguousarray(U, dtype=np.float64).copy()
    assert lib.oracle_rk3_step(ctypes.byref(o.cfg), V.ctypes.data_as(ctypes.c_void_p), 1e-3) == 0
    assert np.array_equal(V, ref)
    assert lib.oracle_ops(1) > 0
