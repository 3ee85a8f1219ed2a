"""Regression fixtures of tests/golden (written from the oracle by make_golden.py).

not gpu: the oracle still reproduces its stored output (a change of its arithmetic must come
         with regenerated fixtures and a reason).
gpu:     the FP64 path reproduces the stored residual to the parity tolerance, the FP32 and
         mixed paths to theirs.
"""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden as G  # noqa: E402


@pytest.mark.parametrize("case", sorted(G.CASES))
def test_oracle_reproduces_fixture(case):
    """To 1e-12 of the largest entry, the FP64 parity bar: numpy builds with other
    summation orders (e.g. on an Arm host) move the residual by ~2e-13 of it."""
    _, R = G.compute(case)
    stored = G.read(case).reshape(R.shape)
    np.testing.assert_allclose(R, stored, rtol=0, atol=1e-12 * np.abs(stored).max())


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-4), ("mixed", 5e-6)])
@pytest.mark.parametrize("case", sorted(G.CASES))
def test_gpu_matches_fixture(case, precision, tol):
    from gpu_helpers import gpu_residual, max_rel_err, residual_term_scale
    from paper_2209_01877_gb300 import dg
    m, P, U = G.inputs(case)
    n, jitter, p, flux, field = G.CASES[case]
    prec = {"fp64": dg.DG_FP64, "fp32": dg.DG_FP32, "mixed": dg.DG_MIXED_FP16}[precision]
    M = dg.Mesh(m.tet_vid, m.tet_xyz, None, order=p, precision=prec,
                flux=dg.DG_ROE if flux == "roe" else dg.DG_RUSANOV, renumber=dg.DG_ORDER_MORTON)
    R = gpu_residual(M, U)[: G.NKEEP]
    stored = G.read(case).reshape(R.shape)
    rows = np.arange(G.NKEEP)
    assert max_rel_err(R, stored, term_scale=residual_term_scale(P, U, rows)) < tol
