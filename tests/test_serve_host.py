"""Host logic of the serving loop that needs no GPU: the arena allocator."""
import numpy as np

import paper_1609_05530_gb300 as cg


def test_arena_first_fit_and_coalescing():
    a = cg.Arena(1 << 20)
    offs = [a.alloc(1000) for _ in range(8)]
    assert offs == [i * 1024 for i in range(8)]          # 256-byte granules, first fit
    assert a.stats()["used"] == 8 * 1024
    assert a.free(offs[1]) and a.free(offs[2])           # neighbours coalesce
    assert a.alloc(2048) == offs[1]
    assert a.free(offs[5]) and a.free(offs[4]) and a.free(offs[6])
    assert a.alloc(3 * 1024) == offs[4]
    assert not a.free(12345)                             # unknown offset
    assert a.alloc(2 << 20) is None                      # larger than the arena


def test_arena_random_workload_keeps_invariants():
    g = np.random.default_rng(0)
    a = cg.Arena(64 << 20)
    live = {}
    for step in range(4000):
        if live and (g.random() < 0.45 or len(live) > 200):
            off = list(live)[int(g.integers(0, len(live)))]
            assert a.free(off)
            del live[off]
        else:
            n = int(g.integers(1, 1 << 18))
            off = a.alloc(n)
            if off is None:
                continue
            need = (n + 255) // 256 * 256
            for o, m in live.items():                    # no overlap with live blocks
                assert off + need <= o or o + m <= off
            live[off] = need
        assert a.stats()["used"] == sum(live.values())
    for off in list(live):
        a.free(off)
    st = a.stats()
    assert st["used"] == 0 and st["largest_free"] == 64 << 20   # fully coalesced again
