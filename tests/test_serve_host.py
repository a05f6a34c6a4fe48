"""Serving loop, host side: the first-fit memory arena that admission uses, and
the request memory layout (no GPU)."""
import random

from paper_2504_09820_gb300 import serve as SV


def test_arena_first_fit_and_coalescing():
    a = SV.Arena(10 * 256)
    b1 = a.alloc(300)          # rounds up to 512
    b2 = a.alloc(256)
    b3 = a.alloc(1024)
    assert b1 == (0, 512) and b2 == (512, 256) and b3 == (768, 1024)
    assert a.alloc(2048) is None                 # only 768 bytes left
    a.free(*b2)
    assert a.alloc(512) == (1792, 512)            # the freed 256 is too small: first fit further on
    a.free(*b1)
    a.free(*b3)                                   # 0..1792 coalesces into one range
    assert a.free_list[0] == (0, 1792)
    assert a.alloc(1792) == (0, 1792)


def test_arena_random_never_overlaps():
    rng = random.Random(1)
    a = SV.Arena(1 << 20)
    live = []
    for _ in range(2000):
        if live and rng.random() < 0.45:
            a.free(*live.pop(rng.randrange(len(live))))
        else:
            blk = a.alloc(rng.randrange(1, 40000))
            if blk:
                live.append(blk)
        spans = sorted(live)
        for (o1, n1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + n1 <= o2
        assert a.used == sum(n for _, n in live)
        assert sum(n for _, n in a.free_list) + a.used == a.size
    for blk in live:
        a.free(*blk)
    assert a.free_list == [(0, a.size)] and a.used == 0


def test_request_bytes_cover_buffers():
    n_rb, n_re, N, K = 5, 14 * 50, 256, 64
    total = SV.request_bytes(n_rb, n_re, N, K)
    raw = n_rb * K * N * 8 + n_re * N * 8 + n_re * 4 + (n_rb + 1) * 8 + n_rb * 8 + n_re * 4 + n_re * K \
        + n_rb * K * K * 8 + n_rb * K * 8 + n_re * K * 8 + n_re * K + n_re * 8 + n_re * 4 + 8
    assert raw <= total <= raw + 14 * 256
