"""The parity measure of the GPU tests: the larger of the 2-norm and the
worst-element relative differences."""
import numpy as np
import pytest

from tests.helpers import rel


def test_rel_sees_a_single_wrong_entry():
    b = np.ones(1_000_000)
    a = b.copy()
    a[7] += 1e-3                      # 2-norm ratio 1e-6, worst element 1e-3
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 2e-6
    assert rel(a, b) == pytest.approx(1e-3)
    assert rel(b, b) == 0.0


def test_rel_rejects_mismatched_shapes():
    with pytest.raises(ValueError):
        rel(np.ones(3), np.ones(4))
