"""Host logic of the serving loop (no GPU): the range allocator behind the
memory-gated admission, the byte layout of a request's resident tensors, and
the seeded request stream."""
import random

import numpy as np

from paper_2311_04406_gb300.serve import RangeAllocator, _carve, make_requests, request_bytes


def test_range_allocator_invariants():
    size = 1 << 20
    a = RangeAllocator(size)
    rng = random.Random(1)
    live = []
    for _ in range(4000):
        if live and rng.random() < 0.5:
            o, n = live.pop(rng.randrange(len(live)))
            a.release(o, n)
        else:
            n = rng.randint(1, 30000)
            o = a.alloc(n)
            if o is not None:
                assert o % 256 == 0 and o + n <= size
                live.append((o, n))
        free = a.free
        assert all(free[i][0] + free[i][1] < free[i + 1][0] for i in range(len(free) - 1)), "sorted, coalesced"
        spans = sorted([(o, -(-n // 256) * 256) for o, n in live] + free)
        assert all(spans[i][0] + spans[i][1] <= spans[i + 1][0] for i in range(len(spans) - 1)), "disjoint"
        assert sum(sz for _, sz in free) + a.used == size
    for o, n in live:
        a.release(o, n)
    assert a.free == [(0, size)] and a.used == 0


def test_allocator_refuses_what_does_not_fit():
    a = RangeAllocator(4096)
    x = a.alloc(3000)
    assert x == 0 and a.alloc(2000) is None
    a.release(x, 3000)
    assert a.alloc(4096) == 0


def test_request_layout():
    for r in make_requests(8, 5.0, seed=3):
        for words in (1, 2):
            plan, inputs_end, keys_end, total = _carve(r.layers, words)
            assert total == request_bytes(r.layers, words)
            spans = []
            for li, L in enumerate(r.layers):
                assert set(plan[li]) == {"E", "A", "mA", "F", "B", "mB", "C", "mC", "R", "mR", "Drest", "alpha",
                                         "chi", "chi_hat", "Z", "mZ", "Dt", "mDc", "Dc", "cs"}
                for k, (shape, off, words_k) in plan[li].items():
                    assert words_k == int(np.prod(shape))
                    n = 8 * words_k
                    assert off % 16 == 0 and off + n <= total
                    assert shape[-1] == 2 if words == 2 else True
                    spans.append((off, n))
                    if k in ("alpha", "chi", "chi_hat"):
                        assert inputs_end <= off and off + n <= keys_end
                    elif k in ("Z", "mZ", "Dt", "mDc", "Dc", "cs"):
                        assert keys_end <= off and off % 256 == 0
                    else:
                        assert off + n <= inputs_end and off % 256 == 0
            spans.sort()
            assert all(spans[i][0] + spans[i][1] <= spans[i + 1][0] for i in range(len(spans) - 1))


def test_request_stream_is_seeded_and_poisson():
    a = make_requests(200, 10.0, seed=5)
    b = make_requests(200, 10.0, seed=5)
    assert [(r.model, r.batch, r.arrival, r.seed) for r in a] == [(r.model, r.batch, r.arrival, r.seed) for r in b]
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert 0.07 < gaps.mean() < 0.13                  # exponential, mean 1 / rate
    assert {r.model for r in a} == {"resnet18", "vgg16"}
    assert min(r.batch for r in a) >= 1 and max(r.batch for r in a) <= 32
    c = make_requests(10, 1.0, seed=5, all_at_once=True)
    assert all(r.arrival == 0.0 for r in c)
