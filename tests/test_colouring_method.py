"""The colouring method of the GPU path, modelled on the CPU: incidence lists
sorted by priority, per-body fronts and colour masks, and rounds that colour
every contact at the front of all its bodies' lists (the fronts as they were
when the round began).  It must give first-fit greedy colouring in
decreasing priority -- the rule the oracle implements -- and each round must
colour exactly the contacts whose predecessors were all coloured before it
(the Jones-Plassmann rounds).  Random contact graphs, walls and bodies of
infinite mass (no incidence list) included."""
import numpy as np


def first_fit(n_contacts, ends, prio):
    """The definition: contacts in decreasing priority (ties: lower index
    first), each taking the smallest colour none of its incident contacts
    already coloured has."""
    order = sorted(range(n_contacts), key=lambda c: (-prio[c], c))
    col = [-1] * n_contacts
    by_body = {}
    for c in range(n_contacts):
        for x in ends[c]:
            by_body.setdefault(x, []).append(c)
    for c in order:
        used = {col[d] for x in ends[c] for d in by_body[x] if d != c and col[d] >= 0}
        k = 0
        while k in used:
            k += 1
        col[c] = k
    return col


def frontier_rounds(n_contacts, ends, prio):
    beats = lambda d, c: (prio[d], -d) > (prio[c], -c)
    lists = {}
    for c in range(n_contacts):
        for x in ends[c]:
            lists.setdefault(x, []).append(c)
    for x in lists:
        lists[x].sort(key=lambda c: (-prio[c], c))
    pos = {(c, x): lists[x].index(c) for x in lists for c in lists[x]}
    front = {x: 0 for x in lists}
    mask = {x: set() for x in lists}
    col = [-1] * n_contacts
    ready = [c for c in range(n_contacts) if all(pos[(c, x)] == 0 for x in ends[c])]
    rounds = []
    while ready:
        start = dict(front)   # every check in a round reads the fronts as the round began
        now = [c for c in dict.fromkeys(ready)
               if col[c] < 0 and all(start[x] == pos[(c, x)] for x in ends[c])]
        exposed = []
        for c in now:
            used = set().union(*[mask[x] for x in ends[c]]) if ends[c] else set()
            k = 0
            while k in used:
                k += 1
            col[c] = k
            for x in ends[c]:
                mask[x].add(k)
                front[x] += 1
                if front[x] < len(lists[x]):
                    exposed.append(lists[x][front[x]])
        rounds.append(now)
        ready = exposed
    return col, rounds, beats


def random_graph(rng, n_bodies, n_contacts, infinite_frac=0.1):
    finite = rng.random(n_bodies) >= infinite_frac
    ends = []
    for _ in range(n_contacts):
        a = int(rng.integers(n_bodies))
        if rng.random() < 0.1:   # a wall: one end only
            ends.append([a] if finite[a] else [])
            continue
        b = int(rng.integers(n_bodies - 1))
        b += b >= a
        ends.append([x for x in (a, b) if finite[x]])
    prio = rng.integers(0, 2 ** 63, n_contacts, dtype=np.uint64).tolist()
    if n_contacts > 4:
        prio[3] = prio[1]   # a tie: broken by the lower index
    return ends, prio


def test_frontier_rounds_give_first_fit_colours():
    rng = np.random.default_rng(12)
    for trial in range(40):
        nb = int(rng.integers(5, 60))
        nc = int(rng.integers(1, 4 * nb))
        ends, prio = random_graph(rng, nb, nc)
        col, rounds, beats = frontier_rounds(nc, ends, prio)
        assert col == first_fit(nc, ends, prio), trial
        # each round: exactly the contacts whose predecessors were all coloured before it
        done = set()
        incident = lambda c: {d for x in ends[c] for d in range(nc) if d != c and x in ends[d]}
        for r in rounds:
            expect = {c for c in range(nc) if c not in done and all(d in done for d in incident(c) if beats(d, c))}
            assert set(r) == expect, trial
            done |= set(r)
        assert len(done) == nc
