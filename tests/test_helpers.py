"""The Newton-count comparison rule used by the GPU parity tests."""
from tests.conftest import newton_counts_agree


def test_newton_counts_agree_rule():
    ro = {"newton_iters": 4, "hist": [1.0, 3.9e-2, 5.5e-5, 1.07e-10, 7.7e-16]}
    assert newton_counts_agree(4, ro)
    assert newton_counts_agree(3, ro)          # the oracle missed tau by 7%
    assert not newton_counts_agree(2, ro)
    assert not newton_counts_agree(5, ro)      # the oracle met tau by far at 4
    far = {"newton_iters": 4, "hist": [1.0, 3.9e-2, 5.5e-5, 3.0e-10, 7.7e-16]}
    assert not newton_counts_agree(3, far)     # 3x above tau: not a rounding decision
    just = {"newton_iters": 3, "hist": [1.0, 3.9e-2, 5.5e-5, 0.8e-10]}
    assert newton_counts_agree(4, just)        # the oracle met tau by 20%
    assert not newton_counts_agree(4, {"newton_iters": 3, "hist": [1.0, 1e-3, 1e-6, 1e-14]})
