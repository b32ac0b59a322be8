"""Host-side model of the sliding-window A ring of the tensor-core kernel
(spec suffix sw=1).  The kernel's rules, restated: slab j of a CTA's run is
converted into slot j % na once slab j - na has been released; tile k of a run
of n tiles reads slabs k .. k + fh - 1 in filter-row order; slab j is released
by its last reader, tile j as its filter row 0, or the run's last tile.  The
model runs the converter and the MMA issuer as two in-order agents and checks,
for every run length, filter height and ring depth the host allows (na >= fh),
that neither waits forever, that no slab is overwritten before its last read,
and that every slab is released exactly once."""
import pytest


def run_ring(n, fh, na):
    slabs = n + fh - 1
    filled = [False] * slabs
    releases = [0] * slabs
    holder = {}
    conv = mma = 0
    while mma < n * fh or conv < slabs:
        moved = False
        if conv < slabs and (conv < na or releases[conv - na] == 1):
            holder[conv % na] = conv
            filled[conv] = True
            conv += 1
            moved = True
        if mma < n * fh:
            k, i = divmod(mma, fh)
            j = k + i
            if filled[j]:
                assert holder[j % na] == j, ("slab overwritten before its last read", n, fh, na, k, i)
                if i == 0 or k == n - 1:
                    releases[j] += 1
                mma += 1
                moved = True
        if not moved:
            return False, releases
    return True, releases


@pytest.mark.parametrize("fh", range(1, 12))
def test_window_ring_never_stalls_and_releases_each_slab_once(fh):
    for n in range(1, 20):
        for na in (fh, fh + 1, fh + 2):
            ok, releases = run_ring(n, fh, na)
            assert ok, (n, fh, na)
            assert all(r == 1 for r in releases), (n, fh, na, releases)


def test_window_ring_model_catches_a_short_ring():
    """The model is not vacuous: a ring of fh - 1 slabs still completes (slab k
    is released by tile k's first filter row, just before tile k needs slab
    k + fh - 1, so the conversion would wait on the MMAs: the host asks for
    na >= fh), and one of fh - 2 slabs stalls in the first tile."""
    for fh in range(3, 12):
        assert run_ring(6, fh, fh - 1)[0]
        assert not run_ring(6, fh, fh - 2)[0]
