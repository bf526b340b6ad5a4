"""The device-memory arena used to admit jobs by HBM footprint: host bookkeeping only
(first fit in address order, 256-byte granules, neighbours merged on free), so it is
exercised here with a fake, never dereferenced base address."""
import pytest

from paper_2303_10785_b300 import gbr

BASE = 1 << 40  # any 256-byte aligned value: the arena never touches the memory


@pytest.fixture()
def arena():
    import __graft_entry__

    __graft_entry__.build()
    a = gbr.Arena(BASE, 1 << 20)
    yield a
    a.close()


def test_first_fit_alignment_and_exhaustion(arena):
    p1 = arena.alloc(1000)          # rounds to 1024
    p2 = arena.alloc(256)
    assert p1 == BASE and p2 == BASE + 1024
    assert all(p % 256 == 0 for p in (p1, p2))
    st = arena.stats()
    assert st["used"] == 1280 and st["free"] == (1 << 20) - 1280 and st["blocks"] == 2
    assert arena.alloc(1 << 20) is None  # does not fit: the caller keeps the job queued


def test_free_merges_neighbours_and_reuses_holes(arena):
    ps = [arena.alloc(4096) for _ in range(4)]
    arena.free(ps[1])
    arena.free(ps[2])  # merges with the hole of ps[1]
    assert arena.stats()["largest_free"] == (1 << 20) - 4 * 4096
    big = arena.alloc(8192)  # first fit: the merged hole
    assert big == ps[1]
    arena.free(ps[0])
    arena.free(big)
    arena.free(ps[3])
    st = arena.stats()
    assert st["used"] == 0 and st["free"] == 1 << 20 and st["largest_free"] == 1 << 20 and st["blocks"] == 0


def test_invalid_frees_rejected(arena):
    p = arena.alloc(512)
    with pytest.raises(gbr.GbrError):
        arena.free(p + 256)   # not the start of an allocation
    with pytest.raises(gbr.GbrError):
        arena.free(BASE + (1 << 21))  # outside the arena
    arena.free(p)
    with pytest.raises(gbr.GbrError):
        arena.free(p)  # double free


def test_unaligned_base_rejected():
    import __graft_entry__

    __graft_entry__.build()
    with pytest.raises(gbr.GbrError):
        gbr.Arena(BASE + 8, 1 << 20)
