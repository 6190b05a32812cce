"""Host-side logic that needs no GPU: batch table layout and batch splitting."""
import numpy as np


def test_instance_table_layout_matches_the_header():
    from paper_1805_02755_gb300.batching import INSTANCE_DTYPE
    # ecl_binomial_instance: 7 pointers, int64 first, int64 n, float r, int32 pad
    assert INSTANCE_DTYPE.itemsize == 80
    assert INSTANCE_DTYPE.fields["first"][1] == 56 and INSTANCE_DTYPE.fields["r"][1] == 72


def test_split_uneven_sums_and_skews():
    from paper_1805_02755_gb300.batching import split_uneven
    for n, parts in [(1 << 20, 64), (1000, 7), (64, 64)]:
        s = split_uneven(n, parts, seed=1)
        assert sum(s) == n and len(s) == parts and min(s) >= 1
    s = np.array(split_uneven(1 << 20, 64, seed=1))
    assert s.max() > 8 * np.median(s)
