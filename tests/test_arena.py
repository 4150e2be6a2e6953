"""The bookkeeping of the server's field-set arena (host code, no GPU): seeded
random allocation and free sequences over regions of several sizes, with the
library's own invariant check after every step (live ranges aligned, disjoint,
inside the region; free ranges coalesced; double frees refused; no refusal
while a free range has room), and the region whole again at the end."""
import pytest

from paper_1711_05017_b300 import _binding as B


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("size", [1 << 20, 96 << 20, 120 << 30, (37 << 30) + 12345])
def test_arena_bookkeeping(seed, size):
    assert B.lib().hf_arena_selftest(seed, size, 3000) == 0


def test_arena_selftest_rejects_bad_arguments():
    assert B.lib().hf_arena_selftest(0, 0, 10) == -1
    assert B.lib().hf_arena_selftest(0, 1 << 20, 0) == -1
