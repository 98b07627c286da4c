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


def test_flops_split_adds_up():
    """The list form's per-kernel split of the near-pair flop count adds up
    to the count of a whole near pair at every order."""
    import bench

    for M in range(0, 9):
        assert sum(bench.flops_per_pair_parts(M)) == bench.flops_per_pair(M)
