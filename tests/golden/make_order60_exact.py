"""Writes tests/golden/order60_dense_exact.txt: exact rows of the order-60
single-particle right-hand side (oracle/exact.py, rational arithmetic) for
the dense state of tests/test_gpu_high_order.py at t = 0 (lambda = 1).

    python tests/golden/make_order60_exact.py

Each line: k1 k2 dM_k S_k, with dM_k the exact row rounded once to a double
and S_k the exact sum of the absolute values of its terms (the scale of the
rounding of any floating-point evaluation of the row).  Calls only oracle/.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import mmvm_inputs  # noqa: E402
from oracle.coefficients import multi_indices  # noqa: E402
from oracle.exact import self_rows_exact, to_float  # noqa: E402

ORDER = 60


def dense_state():
    """1% per moment in the weighted norm, sigma = lambda_0 = 1 (seed 61)."""
    return mmvm_inputs.random_disk(n=1, order=ORDER, radius=0.0, sigma=1.0, amp=0.01, Re=700.0,
                                   seed=61)


def rows():
    rng = np.random.default_rng(1)
    mi = multi_indices(ORDER)
    return sorted(set(rng.integers(0, len(mi), 14).tolist())
                  | {mi.index((1, 1)), mi.index((30, 30)), mi.index((59, 1)), mi.index((0, 60)),
                     mi.index((2, 0)), mi.index((12, 8)), mi.index((40, 0))})


def main():
    wl = dense_state()
    rr = rows()
    vals, sums = self_rows_exact(wl.moments[0], ORDER, rr)
    mi = multi_indices(ORDER)
    out = os.path.join(HERE, "order60_dense_exact.txt")
    with open(out, "w") as f:
        f.write("# exact rows of the order-60 single-particle right-hand side (dense state, t = 0,\n"
                "# lambda = 1): k1 k2 dM_k S_k; written by tests/golden/make_order60_exact.py\n")
        for k, v, s in zip(rr, vals, sums):
            f.write(f"{mi[k][0]} {mi[k][1]} {to_float(v)!r} {to_float(s)!r}\n")
    print(out)


if __name__ == "__main__":
    main()
