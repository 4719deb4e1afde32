"""Host-side helpers of bench.py: the kernel-launch count of one pipelined
solve, against an enumeration of what the pipeline enqueues (per chunk of
links: chain + finish, the finish carrying the per-slice change at
iterations, and at iterations also the correction; one max per iteration; one fine launch per chunk that has
slices, at levels 0 .. K_max-1), and the chunking's coverage: every slice is
swept exactly once per level, by the chunk whose chain produced its start
state."""
import pytest

import bench


def _enumerate(S, chunk, kmax):
    n = -(-S // chunk)
    launches = 0
    for level in range(kmax + 1):
        for j in range(n):
            a = j * chunk
            b = min(S, a + chunk)
            launches += 2 + (1 if level >= 1 else 0)
            f0, f1 = (0 if j == 0 else a + 1), min(b + 1, S)
            if level < kmax and f1 > f0:
                launches += 1
        if level >= 1:
            launches += 1
    return launches


@pytest.mark.parametrize("S,chunk,kmax", [(256, 16, 5), (256, 32, 5), (24, 7, 4), (1, 4, 3), (5, 1, 2),
                                          (17, 4, 0), (16, 16, 5)])
def test_solve_launches(S, chunk, kmax):
    assert bench.solve_launches(S, chunk, kmax) == _enumerate(S, chunk, kmax)


@pytest.mark.parametrize("S,chunk", [(256, 16), (24, 7), (1, 4), (5, 1), (17, 4), (16, 16)])
def test_fine_chunks_cover_each_slice_once(S, chunk):
    n = -(-S // chunk)
    seen = []
    for j in range(n):
        a, b = j * chunk, min(S, j * chunk + chunk)
        f0, f1 = (0 if j == 0 else a + 1), min(b + 1, S)
        for s in range(f0, f1):
            # slice s starts from U_s, produced by link s-1 (or u0 for s = 0)
            assert s == 0 or a <= s - 1 < b
            seen.append(s)
    assert sorted(seen) == list(range(S))
