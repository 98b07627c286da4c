"""The work counts bench.py reports, against the oracle's literal sums."""
from bench import coefficient_terms
from oracle.coefficients import gamma_I_terms, gamma_II_terms, multi_indices


def test_coefficient_terms_count_the_literal_sums():
    for M in (2, 4, 6):
        mi = multi_indices(M)
        n = sum(len(gamma_I_terms(k1, k2, l1, l2, 1.0)) + len(gamma_II_terms(k1, k2, l1, l2, 1.0))
                for (k1, k2) in mi for (l1, l2) in mi)
        assert coefficient_terms(M) == n
    assert coefficient_terms(60) == 945439488
