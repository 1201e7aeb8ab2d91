"""Host helpers of the strategy study that need no GPU."""
import itertools
import math

from paper_1511_07983_gb300 import study


def test_lehmer_digits_give_the_lexicographic_position():
    # itertools.permutations enumerates in lexicographic order
    for n in (1, 2, 5, 7):
        for pos, p in enumerate(itertools.permutations(range(n))):
            d = study._lehmer_digits(p)
            assert all(0 <= d[j] <= n - 1 - j for j in range(n))
            assert sum(dj * math.factorial(n - 1 - j) for j, dj in enumerate(d)) == pos


def test_lehmer_digits_of_relabelled_kernels():
    # digits depend only on relative order, so any increasing relabelling keeps them
    assert study._lehmer_digits([30, 10, 20]) == study._lehmer_digits([2, 0, 1]) == [2, 0, 0]
