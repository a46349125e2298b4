"""Canonical branch tree from outcome logs (Section IV-B), hand-built cases."""
import numpy as np

from oracle import oracle as O


def test_tree_from_outcome_logs():
    # 4 shots, random ops 0 and 1 (columns)
    out = np.array([[0, 0], [0, 1], [2, 0], [0, 1]])
    t = O.branch_tree(out, [0, 1])
    F = frozenset
    assert t == {
        (0, F({0, 1, 2, 3}), F({0, 1, 3}), 0),
        (0, F({0, 1, 2, 3}), F({2}), 2),
        (1, F({0, 1, 3}), F({0}), 0),
        (1, F({0, 1, 3}), F({1, 3}), 1),
    }


def test_tree_without_divergence_is_empty():
    out = np.zeros((5, 3), int)
    assert O.branch_tree(out, [0, 1, 2]) == set()
