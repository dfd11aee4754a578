"""Host logic of the server's device arenas (CudaExecutor._arena), run on CPU tensors:
pieces are 256-byte aligned and sized as asked, an arena kept under a key is reused
while large enough and replaced by one of the next power-of-two size otherwise, and a
zero-filled arena is cleared over the requested range on every reuse."""
import types

import torch

from paper_2302_07992_gb300.serve import CudaExecutor


def _ex():
    return types.SimpleNamespace(_arenas={})


def _arena(ex, sizes, zero, key=None):
    return CudaExecutor._arena(ex, sizes, zero, "cpu", key)


def test_pieces_are_aligned_and_sized():
    buf, views = _arena(_ex(), [10, None, 300, 1], False)
    assert views[1] is None
    assert [v.numel() for v in (views[0], views[2], views[3])] == [10, 300, 1]
    base = buf.data_ptr()
    offs = [v.data_ptr() - base for v in (views[0], views[2], views[3])]
    assert offs == [0, 256, 768] and all(o % 256 == 0 for o in offs)


def test_keyed_arena_is_reused_and_grows_by_powers_of_two():
    ex = _ex()
    a, _ = _arena(ex, [1000], False, key=("s", "img"))
    assert a.numel() == 1024                      # next power of two of 1024 (rounded pieces)
    b, _ = _arena(ex, [500], False, key=("s", "img"))
    assert b.data_ptr() == a.data_ptr()           # large enough: the same memory
    c, _ = _arena(ex, [3000], False, key=("s", "img"))
    assert c.numel() == 4096 and ex._arenas[("s", "img")] is c
    d, _ = _arena(ex, [10], False, key=("t", "img"))
    assert d.data_ptr() != c.data_ptr()           # another stream: its own arena


def test_zero_arena_is_cleared_on_reuse():
    ex = _ex()
    buf, views = _arena(ex, [300, 20], True, key=("s", "bits"))
    buf.fill_(0xA5)                               # the previous batch's contents
    buf2, views2 = _arena(ex, [300, 20], True, key=("s", "bits"))
    assert buf2.data_ptr() == buf.data_ptr()
    assert not views2[0].any() and not views2[1].any()
    assert not buf2[:512].any()                   # the whole requested range


def test_unkeyed_arena_is_fresh_each_time():
    ex = _ex()
    a, _ = _arena(ex, [100], True)
    b, _ = _arena(ex, [100], True)
    assert a.data_ptr() != b.data_ptr() and not ex._arenas
