"""Pins of oracle/patchwise.py: the 1D patch matrices sum to the global 1D factors of
Eq. (9), and the patch-wise evaluation over vertex patches equals the assembled SIPG
matrix (pinned to brute-force quadrature in test_oracle_sipg.py)."""
import numpy as np
import pytest

from oracle import patchwise
from oracle.sipg import Mesh, assemble, global_1d
from tp_synth import uniform_vector


@pytest.mark.parametrize("pen", ["config", "paper"])
@pytest.mark.parametrize("nc", [2, 3, 4, 5])
@pytest.mark.parametrize("k", [1, 3, 6])
def test_patch_matrices_sum_to_the_global_1d_factors(k, nc, pen):
    M, L = patchwise.sum_1d(k, nc, 0.7, pen)
    Mg, Lg = global_1d(k, nc, 0.7, pen)
    np.testing.assert_allclose(M, Mg, rtol=0, atol=1e-14 * np.abs(Mg).max())
    np.testing.assert_allclose(L, Lg, rtol=0, atol=1e-13 * np.abs(Lg).max())


@pytest.mark.parametrize("k,dims,lengths,pen", [
    (1, (2, 2, 2), (1, 1, 1), "config"), (2, (3, 2, 4), (1, 1, 1), "config"), (3, (4, 3, 2), (1, 1, 1), "paper"),
    (2, (5, 3, 2), (0.7, 1.9, 0.45), "config"), (4, (2, 3, 2), (1, 1, 1), "config"), (7, (2, 2, 2), (1, 1, 1), "paper")])
def test_patchwise_apply_equals_the_assembled_operator(k, dims, lengths, pen):
    A = assemble(Mesh(*dims, *lengths), k, pen)
    x = uniform_vector(A.shape[0], seed=5 + k)
    y = patchwise.apply(x, k, dims, lengths, pen)
    ref = A @ x
    assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)


def test_patchwise_needs_two_cells_per_direction():
    with pytest.raises(ValueError):
        patchwise.apply(np.zeros(64 * 4), 3, (1, 2, 2))


def test_flop_count_matches_the_papers_table_at_n16():
    # Table 4 (N = 16, patch-wise): 1702..1843 flop/DoF for the non-corrected kernels; N = 2n
    assert 1690 <= patchwise.flops_per_dof(7) <= 1850
