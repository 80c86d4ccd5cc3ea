"""The approximate-inverse preconditioners of Sec. 3 as read here
(M^-1 = K^T K, first and second order, untruncated), on the oracle's Poisson
operator: symmetric positive definite for 0 < w < 2, and the ordering of
condition numbers that Sec. 7.3 reports in its tables (CG ~ Jacobi > AI1 >
AI2), with a minimum over w inside (1, 1.9)."""
import numpy as np
import pytest

import dense_ai as D


@pytest.fixture(scope="module")
def A():
    import oracle
    oracle.build()
    return D.dense_A(10, 8, 6, 30.0)


def test_ai_inverses_are_spd(A):
    for w in (0.5, 1.0, 1.65, 1.9):
        for order in (1, 2):
            M, _ = D.ai_inverse(A, w, order)
            assert np.allclose(M, M.T)
            assert np.linalg.eigvalsh(M)[0] > 0, (w, order)


def test_condition_number_ordering(A):
    k_cg, _ = D.condition(A)
    k_j, _ = D.condition(A, d=np.diag(A))
    k1, _ = D.condition(A, D.ai_inverse(A, 1.65, 1)[1])
    k2, _ = D.condition(A, D.ai_inverse(A, 1.65, 2)[1])
    assert k_cg > k_j > k1 > k2
    assert k_j / k_cg > 0.8          # Jacobi barely helps on a near-constant diagonal
    assert k1 < 0.3 * k_cg and k2 < 0.7 * k1


def test_condition_number_has_an_interior_minimum_in_w(A):
    for order in (1, 2):
        k = {w: D.condition(A, D.ai_inverse(A, w, order)[1])[0] for w in (1.0, 1.65, 1.9)}
        assert k[1.65] < k[1.0] and k[1.65] < k[1.9], (order, k)


def test_reference_pcg_iteration_ordering(A):
    b = np.random.default_rng(1).standard_normal(A.shape[0])
    its = {}
    for name, M in [("none", np.eye(A.shape[0])), ("jacobi", np.diag(1 / np.diag(A))),
                    ("ai1", D.ai_inverse(A, 1.65, 1)[0]), ("ai2", D.ai_inverse(A, 1.65, 2)[0])]:
        its[name] = D.pcg_iterations(A, M, b, 1e-10, "residual")[0]
    assert its["none"] >= its["jacobi"] > its["ai1"] > its["ai2"], its
