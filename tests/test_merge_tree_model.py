"""A CPU model of the pair kernels' merge tree (hk_internal.h, merge_tree) under random
interleavings of the CTAs' steps: for item spans 1, 2 and 4 and every leaf count up to 80,
exactly one CTA completes the root, every counter index stays below 2 K, every slot read was
published before it is read, and the root's sums (float32 additions, so order would show) do
not depend on the order in which items finish. Both arrival protocols are modelled: every
arriver stores then counts, and the first arriver publishes with a ready mark (arrivals add
1, the mark adds 4) while the second waits for it."""
import random

import numpy as np
import pytest

ARRIVED, READY = 1, 4


def _run(K, span, seed, publish_first):
    rng = random.Random(seed)
    n_items = (K + span - 1) // span
    vals = [np.float32(1.0 + 0.37 * i + 1e-3 * i * i) for i in range(n_items)]
    slots, cnt, results = {}, {}, []

    def item(i):
        own = vals[i]
        width, off = span, 0
        w = 1
        while w < span:
            off += (K + 2 * w - 1) // (2 * w)
            w *= 2
        node = i
        while width < K:
            parent, sib = node >> 1, node ^ 1
            if sib * width < K:
                key = off + parent
                assert key < 2 * K
                my_slot, sib_slot = node * width // span, sib * width // span
                if not publish_first:
                    slots[my_slot] = own
                    yield
                    old = cnt.get(key, 0)
                    cnt[key] = old + ARRIVED
                    if old == 0:
                        return
                    yield
                else:
                    old = cnt.get(key, 0)
                    cnt[key] = old + ARRIVED
                    yield
                    if old == 0:
                        slots[my_slot] = own
                        yield
                        cnt[key] += READY
                        return
                    while not (cnt[key] & READY):
                        yield
                assert sib_slot in slots  # published before it is read
                own = np.float32(own + slots[sib_slot])
                yield
            off += (K + 2 * width - 1) // (2 * width)
            node >>= 1
            width *= 2
        results.append(own)

    gens = [item(i) for i in range(n_items)]
    live = list(range(n_items))
    while live:
        i = rng.choice(live)
        try:
            next(gens[i])
        except StopIteration:
            live.remove(i)
    assert len(results) == 1, (K, span, len(results))
    return results[0]


@pytest.mark.parametrize("publish_first", [False, True], ids=["store_then_count", "publish_first"])
@pytest.mark.parametrize("span", [1, 2, 4])
def test_merge_tree_one_root_and_order_independent_sums(span, publish_first):
    for K in range(1, 81):
        ref = _run(K, span, 0, publish_first)
        for seed in range(1, 6):
            assert _run(K, span, seed, publish_first) == ref, (K, span, seed)
