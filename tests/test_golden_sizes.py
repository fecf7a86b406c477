"""The system sizes printed in Sec. III (tests/golden/paper_system_sizes.txt) against the input
generator's state lists.

The paper gives N at the two ends of each l_max scan but not the basis per l. Reading: a fixed number
of radial functions per l (one-centre: hydrogenic n <= 10 plus 32 wave packets, 42 per l; two-centre:
n <= 10 plus 20 packets, 30 per l on each centre), every m = -l..l. That reproduces all four printed
sizes; counting only m >= 0 would give 2332 instead of 4257 at l_max = 10.
"""
import os

import numpy as np
import pytest

import wpccc_inputs as wi

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_system_sizes.txt")

# radial functions per l: (n_max, packets per l) for one and two centres
PER_L = {1: (10, 32), 2: (10, 20)}


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            rows.append(tuple(int(x) for x in line.split()))
    return rows


def test_golden_file_lists_both_modes():
    rows = _golden()
    assert {(c, l) for c, l, _ in rows} == {(1, 0), (1, 10), (2, 0), (2, 5)}


@pytest.mark.parametrize("centres,lmax,N", _golden())
def test_generator_reproduces_the_printed_size(centres, lmax, N):
    nmax, packets = PER_L[centres]
    g = wi.radial_grid(400)
    c = wi.make_centre(1.0, nmax, lmax, packets, 2.0, g)
    # p + H: both centres carry the same states
    assert centres * c.N == N
    # the m >= 0 count differs wherever l_max > 0
    half = c.N if lmax == 0 else int(np.count_nonzero(c.st_m >= 0))
    assert (half == c.N) == (lmax == 0)
