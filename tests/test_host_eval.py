"""Host logic of the search measurement: recall@k with its tie and short-list rules, and
the choice of the fastest operating point at a recall target (no GPU needed)."""
import numpy as np

from paper_2511_16576_gb300 import evaluate as ev


def truth(ids, j, n_pos):
    return ev.Truth(np.asarray(ids, np.int32), np.asarray(j, np.float64), np.asarray(n_pos), 0)


def test_recall_exact_and_partial():
    t = truth([[1, 2, 3]], [[0.9, 0.5, 0.2]], [3])
    assert ev.recall_at_k(np.array([[3, 2, 1]]), np.array([[0.2, 0.5, 0.9]]), t, k=3) == 1.0
    assert ev.recall_at_k(np.array([[1, 7, -1]]), np.array([[0.9, 0.1, -1.0]]), t, k=3) == 1.0 / 3


def test_recall_counts_ties_with_the_kth_value():
    # polygon 9 is not in the exact list but ties the k-th exact J within the tolerance
    t = truth([[1, 2]], [[0.9, 0.4]], [2])
    got = ev.recall_at_k(np.array([[1, 9]]), np.array([[0.9, 0.4 - 1e-12]]), t, k=2)
    assert got == 1.0
    # a clearly smaller J does not count
    got = ev.recall_at_k(np.array([[1, 9]]), np.array([[0.9, 0.3]]), t, k=2)
    assert got == 0.5


def test_recall_short_truth_and_empty_rows():
    # only two polygons overlap the first query: the denominator is 2; the second query
    # has no overlapping polygon and is skipped
    t = truth([[4, 5, -1], [-1, -1, -1]], [[0.7, 0.1, -1.0], [-1.0, -1.0, -1.0]], [2, 0])
    ans = np.array([[5, 4, 8], [1, 2, 3]])
    js = np.array([[0.1, 0.7, 0.0], [0.0, 0.0, 0.0]])
    assert ev.recall_at_k(ans, js, t, k=3) == 1.0
    # ties at the k-th value are only honoured when the truth is a full k-list
    assert ev.recall_at_k(np.array([[4, 8, 9]]), np.array([[0.7, 0.1, 0.1]]),
                          truth([[4, 5, -1]], [[0.7, 0.1, -1.0]], [2]), k=3) == 0.5


def test_best_at_recall_picks_the_fastest_reaching_the_target():
    rows = [{"m": 8, "recall": 0.85, "qps": 900.0}, {"m": 16, "recall": 0.91, "qps": 700.0},
            {"m": 24, "recall": 0.95, "qps": 500.0}]
    assert ev.best_at_recall(rows, 0.9)["m"] == 16
    assert ev.best_at_recall(rows, 0.99) is None
