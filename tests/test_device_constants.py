"""Constants written into the device code, checked against their definitions (CPU only)."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_conserving_rounding_feedback_table():
    """The FP32 collision re-rounds its nine results in the order 1..8, 0 with the feedback
    c_k = (G + 0.01 I)^{-1} a_k, a_k = (1, e_kx, e_ky) the mass and momentum of population k, G
    the sum of a a^T over the populations not yet re-rounded.  The table in the header equals
    that definition to FP32 precision, row by row."""
    src = open(os.path.join(ROOT, "paper_2306_01525_gb300", "csrc", "d2q9_device.cuh")).read()
    order = [int(v) for v in re.search(r"kOrder\[9\] = \{([^}]*)\}", src).group(1).split(",")]
    body = re.search(r"kC\[9\]\[3\] = \{(.*?)\};", src, re.S).group(1)
    table = np.array([[float(x.strip().rstrip("f")) for x in row.split(",")]
                      for row in re.findall(r"\{([^{}]*)\}", body)])
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1.0])
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1.0])
    A = np.stack([np.ones(9), ex, ey])
    assert sorted(order) == list(range(9)) and order[-1] == 0
    for p, k in enumerate(order):
        rest = order[p:]
        G = A[:, rest] @ A[:, rest].T + 0.01 * np.eye(3)
        np.testing.assert_allclose(table[p], np.linalg.solve(G, A[:, k]), rtol=1e-7, atol=1e-9)
