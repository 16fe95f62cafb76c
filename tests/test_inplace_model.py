"""A host model of the in-place digit permutation (no GPU).

It restates, in plain Python, the protocol of the in-place mode for one big
bucket -- classification of each stripe into one-digit blocks and partial
buffers, the carry of blocks to their digit's slots under concurrently
running carrier groups, and the cleanup -- and runs the carriers as
interleaved coroutines in random orders.  Every atomic step of a group is one
scheduling point.  Checks: no slot is overwritten while its block has not
been read out, every block lands exactly once, no group waits forever, and
the result is the bucket partitioned by digit with the same multiset.
"""
import random

import pytest

FULL, TAKEN, HOLE = 0, 1, 3


def classify(keys, digit_of, stripe_keys, B, ndig):
    """Phase A for every stripe: the stripe front gets its full one-digit
    blocks (in the order they fill), the rest of each digit goes to the
    stripe's partial buffer.  Returns the buffer after classification, the
    state words (state, digit, rank) per slot, per-stripe full counts and
    partial buffers."""
    n = len(keys)
    buf = list(keys)
    nslots = (n + B - 1) // B
    state = [(HOLE, 0, 0)] * nslots
    nfull, parts = [], []
    for s0 in range(0, n, stripe_keys):
        stripe = keys[s0:s0 + stripe_keys]
        fill = [[] for _ in range(ndig)]
        wp, counts = 0, [0] * ndig
        for k in stripe:  # one key per "tile": the order of block emission is what matters
            d = digit_of(k)
            fill[d].append(k)
            if len(fill[d]) == B:
                for e in range(B):
                    buf[s0 + wp * B + e] = fill[d][e]
                state[s0 // B + wp] = (FULL, d, counts[d])
                counts[d] += 1
                wp += 1
                fill[d] = []
        nfull.append(counts)
        parts.append(fill)
    return buf, state, nfull, parts


def carrier(gid, seeds, shared, log):
    """One carrier group as a coroutine; every yield is a scheduling point."""
    buf, state, B, dend = shared["buf"], shared["state"], shared["B"], shared["dend"]
    for seed in seeds:
        st, d, dst0 = state[seed]  # atomic OR of TAKEN: read and set in one step
        if shared.get("split_seed_or"):  # planted mistake: read, then set later
            yield
        if st == FULL:
            state[seed] = (TAKEN, d, dst0)
        yield
        if st != FULL:  # it was taken or a hole
            continue
        x = buf[seed * B:(seed + 1) * B]
        log["read"].add(seed)
        yield
        state[seed] = (HOLE, d, dst0)
        xw = (d, dst0)  # the carried block's digit (from its keys) and destination (from its word)
        while True:
            yield
            dst = xw[1]
            y = buf[dst * B:(dst + 1) * B]  # speculative read, same round trip as the OR
            dst_state = state[dst]
            if dst_state[0] == FULL:
                state[dst] = (TAKEN,) + dst_state[1:]
            yield
            if dst_state[0] == FULL:
                log["read"].add(dst)
                put(buf, dst, x, B, xw[0], dend, shared, log)
                x, xw = y, dst_state[1:]
                continue
            spins = 0
            while state[dst][0] != HOLE:  # a seeder is reading dst out
                spins += 1
                assert spins < 10 ** 6, "wait never ended"
                yield
            put(buf, dst, x, B, xw[0], dend, shared, log)
            break


def put(buf, slot, x, B, d, dend, shared, log):
    assert slot in log["read"] or shared["state0"][slot][0] == HOLE, "slot %d overwritten before read" % slot
    assert slot not in log["written"], "slot %d written twice" % slot
    log["written"].add(slot)
    for e, v in enumerate(x):
        pos = slot * B + e
        if pos < dend[d + 1]:
            buf[pos] = v
        else:
            shared["ovf"][d].append((pos - dend[d + 1], v))


def run_model(n, B, stripe_blocks, ndig, groups, seed, split_seed_or=False):
    rng = random.Random(seed)
    keys = [rng.randrange(ndig * 7) for _ in range(n)]
    digit_of = lambda k: k % ndig  # noqa: E731
    stripe_keys = stripe_blocks * B
    counts = [sum(1 for k in keys if digit_of(k) == d) for d in range(ndig)]
    D = [0]
    for c in counts:
        D.append(D[-1] + c)
    buf, state, nfull, parts = classify(keys, digit_of, stripe_keys, B, ndig)
    nstripes = len(nfull)
    # each stripe claims its share of each digit's slots, in a random stripe order
    N = [0] * ndig
    prefix = [[0] * ndig for _ in range(nstripes)]
    for s in rng.sample(range(nstripes), nstripes):
        for d in range(ndig):
            prefix[s][d] = N[d]
            N[d] += nfull[s][d]
    A = [(D[d] + B - 1) // B for d in range(ndig)]
    # each full slot's word then names its block's destination: digit slot
    # base + the stripe's share + the block's rank
    for slot, (st, d, r) in enumerate(state):
        if st == FULL:
            state[slot] = (FULL, d, A[d] + prefix[slot // stripe_blocks][d] + r)

    shared = {"buf": buf, "state": state, "state0": list(state), "B": B, "dend": D,
              "ovf": [[] for _ in range(ndig)], "split_seed_or": split_seed_or}
    log = {"read": set(), "written": set()}
    # groups seed the full slots of the stripes, interleaved
    seeds_of = [[] for _ in range(groups)]
    full_slots = [s * stripe_blocks + j for s in range(nstripes) for j in range(sum(nfull[s]))]
    for i, slot in enumerate(full_slots):
        seeds_of[i % groups].append(slot)
    live = [carrier(g, seeds_of[g], shared, log) for g in range(groups)]
    while live:
        g = rng.randrange(len(live))
        try:
            next(live[g])
        except StopIteration:
            live.pop(g)
    assert len(log["written"]) == sum(N), "every block lands exactly once"
    # cleanup: partial blocks of every stripe, then the overflow, fill the
    # digit's range outside its full slots
    for d in range(ndig):
        h1 = A[d] * B if N[d] else D[d + 1]
        t0 = min((A[d] + N[d]) * B, D[d + 1]) if N[d] else D[d + 1]
        pos = list(range(D[d], h1)) + list(range(t0, D[d + 1]))
        pool = [k for s in range(nstripes) for k in parts[s][d]] + [v for _, v in sorted(shared["ovf"][d])]
        assert len(pool) == len(pos)
        for p, v in zip(pos, pool):
            buf[p] = v
    return keys, buf, D, digit_of


@pytest.mark.parametrize("seed", range(40))
def test_permutation_protocol_random_interleavings(seed):
    rng = random.Random(1000 + seed)
    n = rng.randrange(50, 600)
    B = rng.choice([2, 3, 4])
    ndig = rng.choice([2, 3, 5, 8])
    keys, out, D, digit_of = run_model(n, B, stripe_blocks=rng.choice([4, 7, 16]), ndig=ndig,
                                       groups=rng.choice([1, 2, 5, 9]), seed=seed)
    assert sorted(out) == sorted(keys), "not a permutation of the bucket"
    for d in range(ndig):
        assert all(digit_of(k) == d for k in out[D[d]:D[d + 1]]), "digit %d range holds other digits" % d


def test_model_catches_a_non_atomic_take():
    """Planted mistake: the seeder reads the slot state and sets it in two
    steps.  Some interleaving then lets two groups take one block."""
    caught = 0
    for seed in range(40):
        try:
            run_model(400, 3, 7, 5, 9, seed, split_seed_or=True)
        except AssertionError:
            caught += 1
    assert caught > 0
