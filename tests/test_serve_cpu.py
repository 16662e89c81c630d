"""Host-side logic of the serving loop (no GPU): the pool allocator."""
from paper_1303_5057_gb300.serve import PoolAllocator, Slot


def test_first_fit_allocation_and_merge():
    a = PoolAllocator(100)
    s1 = a.alloc(30)
    s2 = a.alloc(50)
    assert (s1.first, s1.n, s2.first, s2.n) == (0, 30, 30, 50)
    assert a.alloc(30) is None  # only 20 left
    a.release(s1)
    s3 = a.alloc(25)
    assert s3.first == 0
    a.release(s2)
    a.release(s3)
    assert a.free == [Slot(0, 100)] and a.free_rays() == 100


def test_fragmentation_reuses_holes():
    a = PoolAllocator(64)
    slots = [a.alloc(8) for _ in range(8)]
    for s in slots[::2]:
        a.release(s)
    assert a.free_rays() == 32
    assert a.alloc(16) is None  # no hole of 16
    assert a.alloc(8).first == 0
