"""Every interleaving of the visited-set insert protocol, explored on tiny
tables (a model check of the lock-free insert, on the CPU).

The exploration kernel inserts the keys of level L + 1 into a table that
still holds keys of earlier levels (a slot holding one is free) and is never
cleared between levels.  This file restates the protocol's atomic steps --
the CAS-first insert (a compare-and-swap from empty on the key's first slot;
from a key of an earlier level, a second compare-and-swap from that key; the
general insert otherwise), the split insert (a compare-and-swap on the first
free slot of the fetched bucket, the general insert when it fails or the
bucket holds no free slot), the general insert (read a bucket slot by slot,
then compare-and-swap the first free slot, up to three tries a slot), and
the clearing scheme's compare-and-swap of an expanded state's own first slot
back to empty -- as explicit state machines, and explores every order of
their atomic steps.  In every final state each inserted key must sit in
exactly one slot and exactly one of the threads inserting it must report the
win, the others a duplicate: the exactness the counts rely on.
"""
import pytest

L = 5  # the level being expanded; the inserts are of level L + 1


def lvl(v):
    return v[1]


def cas(table, i, expect, new):
    old = table[i]
    if old == expect:
        table = table[:i] + (new,) + table[i + 1:]
    return table, old


class Model:
    def __init__(self, B, S, first_retry=True):
        self.B, self.S, self.first_retry = B, S, first_retry

    # thread state: (kind, key, home, pc, bucket, probe, s, cur, tries, v, result)
    def start(self, kind, key, home):
        pc = {"cas_first": "first", "split": "sread", "general": "gread", "clear": "clear"}[kind]
        return (kind, key, home, pc, home, 0, 0, 0, 0, (), None)

    def _general_from(self, th, bucket, probe):
        kind, key, home = th[:3]
        if probe == self.B:
            return (kind, key, home, "done", bucket, probe, 0, 0, 0, (), -1)
        return (kind, key, home, "gread", bucket, probe, 0, 0, 0, (), None)

    def _scan(self, th):
        """Local steps of the general insert after its bucket read, up to its
        next compare-and-swap or its end."""
        kind, key, home, pc, bucket, probe, s, cur, tries, v, res = th
        while True:
            if s == self.S:  # next bucket
                return self._general_from(th, (bucket + 1) % self.B, probe + 1)
            if tries == 3 or (cur != 0 and cur != key and lvl(cur) >= L + 1):
                s += 1  # taken this level (or the defensive bound): next slot
                cur, tries = (v[s] if s < self.S else 0), 0
                th = (kind, key, home, "gscan", bucket, probe, s, cur, tries, v, None)
                continue
            if cur == key:
                return (kind, key, home, "done", bucket, probe, s, cur, tries, v, 0)
            return (kind, key, home, "gcas", bucket, probe, s, cur, tries, v, None)

    def step(self, table, th):
        kind, key, home, pc, bucket, probe, s, cur, tries, v, res = th
        S = self.S
        if pc == "clear":  # an expanded state empties its own first slot
            table, _ = cas(table, home * S, key, 0)
            return table, (kind, key, home, "done", bucket, probe, s, cur, tries, v, "cleared")
        if pc == "first":
            table, old = cas(table, home * S, 0, key)
            if old == 0:
                return table, (kind, key, home, "done", bucket, probe, s, cur, tries, v, 1)
            if old == key:
                return table, (kind, key, home, "done", bucket, probe, s, cur, tries, v, 0)
            if self.first_retry and lvl(old) <= L:
                return table, (kind, key, home, "retry", bucket, probe, s, old, tries, v, None)
            return table, self._general_from(th, home, 0)
        if pc == "retry":
            table, old = cas(table, home * S, cur, key)
            if old == cur:
                return table, (kind, key, home, "done", bucket, probe, s, cur, tries, v, 1)
            if old == key:
                return table, (kind, key, home, "done", bucket, probe, s, cur, tries, v, 0)
            return table, self._general_from(th, home, 0)
        if pc == "sread":  # split: the first bucket is fetched, a free slot picked from it
            v = v + (table[home * S + s],)
            if len(v) < S:
                return table, (kind, key, home, "sread", bucket, probe, s + 1, cur, tries, v, None)
            if key in v:
                return table, (kind, key, home, "done", bucket, probe, s, cur, tries, v, 0)
            free = [i for i, x in enumerate(v) if x == 0 or lvl(x) <= L]
            if not free:  # the bucket holds this level's keys: the general insert, rereading it
                return table, self._general_from(th, home, 0)
            return table, (kind, key, home, "spick", bucket, probe, free[0], v[free[0]], tries, v, None)
        if pc == "spick":
            table, old = cas(table, home * S + s, cur, key)
            if old == cur:
                return table, (kind, key, home, "done", bucket, probe, s, cur, tries, v, 1)
            if old == key:
                return table, (kind, key, home, "done", bucket, probe, s, cur, tries, v, 0)
            return table, self._general_from(th, home, 0)
        if pc == "gread":  # one slot of the bucket per step (the loads are not one atomic read)
            v = v + (table[bucket * S + s],)
            if len(v) < S:
                return table, (kind, key, home, "gread", bucket, probe, s + 1, cur, tries, v, None)
            if key in v:
                return table, (kind, key, home, "done", bucket, probe, s, cur, tries, v, 0)
            return table, self._scan((kind, key, home, "gscan", bucket, probe, 0, v[0], 0, v, None))
        if pc == "gcas":
            table, old = cas(table, bucket * S + s, cur, key)
            if old == cur:
                return table, (kind, key, home, "done", bucket, probe, s, cur, tries, v, 1)
            return table, self._scan((kind, key, home, "gscan", bucket, probe, s, old, tries + 1, v, None))
        raise AssertionError(pc)

    def explore(self, table, threads):
        """Every interleaving; returns the number of distinct states and the
        final states reached."""
        start = (tuple(table), tuple(self.start(*t) for t in threads))
        seen, stack, finals = {start}, [start], set()
        while stack:
            tab, ths = stack.pop()
            live = [i for i, t in enumerate(ths) if t[3] != "done"]
            if not live:
                finals.add((tab, ths))
                continue
            for i in live:
                tab2, th2 = self.step(tab, ths[i])
                nxt = (tab2, ths[:i] + (th2,) + ths[i + 1:])
                if nxt not in seen:
                    seen.add(nxt)
                    stack.append(nxt)
        return len(seen), finals


def check_finals(finals, threads, present):
    """Each key inserted by some thread: one slot holds it, one inserter won
    (none when the key was already in the table), none hit the probe limit."""
    assert finals
    for tab, ths in finals:
        keys = {t[1] for t in threads if t[0] != "clear"}
        for k in keys:
            assert sum(1 for x in tab if x == k) == 1, (k, tab, ths)
            results = [t[10] for t in ths if t[1] == k and t[0] != "clear"]
            assert -1 not in results
            assert results.count(1) == (0 if k in present else 1), (k, results, tab)
            assert results.count(0) == len(results) - results.count(1)


K1, K2, K3 = ("k1", L + 1), ("k2", L + 1), ("k3", L + 1)
X, Y, Z, W = ("x", L), ("y", L - 1), ("z", L + 1), ("w", L)

SCENARIOS = [
    # a stale first slot, raced by two inserts of one key, another key and the clearing of the stale key
    ("stale_first_slot", (X, 0, Y, 0),
     [("cas_first", K1, 0), ("cas_first", K1, 0), ("cas_first", K2, 0), ("clear", X, 0)], set()),
    # the first slot holds a key of this level; a duplicate of that key is also inserted
    ("current_first_slot", (Z, X, 0, W),
     [("cas_first", K1, 0), ("cas_first", K1, 0), ("cas_first", Z, 0), ("clear", X, 0)], {Z}),
    # every slot stale: inserts spill over buckets
    ("all_stale", (X, W, Y, X),
     [("cas_first", K1, 0), ("cas_first", K1, 0), ("cas_first", K2, 0), ("cas_first", K3, 1)], set()),
    # the CAS-first insert racing the general insert (the fallback) for the same key
    ("mixed_paths", (X, 0, 0, W),
     [("cas_first", K1, 0), ("general", K1, 0), ("general", K2, 0), ("clear", X, 0)], set()),
    # a full first bucket of this level's keys, one free slot in the next
    ("spill", (Z, ("v", L + 1), W, 0),
     [("cas_first", K1, 0), ("cas_first", K1, 0), ("general", K2, 0)], set()),
]
# the same checks with four slots a bucket (64-bit keys) and with three buckets and six threads
BIG = [
    ("split_four_slots", 2, 4, (X, Z, 0, W, Y, 0, X, 0),
     [("split", K1, 0), ("split", K1, 0), ("split", K2, 0), ("cas_first", K2, 0), ("general", K1, 0)], set()),
    ("four_slots", 2, 4, (X, 0, Z, W, Y, 0, 0, X),
     [("cas_first", K1, 0), ("cas_first", K1, 0), ("general", K2, 0), ("clear", X, 0)], set()),
    ("three_buckets", 3, 2, (X, Z, W, 0, Y, X),
     [("cas_first", K1, 0), ("cas_first", K1, 0), ("cas_first", K2, 0), ("general", K1, 0),
      ("clear", X, 0), ("clear", W, 1)], set()),
]


@pytest.mark.parametrize("first_retry", [True, False], ids=["second_cas", "reread"])
@pytest.mark.parametrize("name,table,threads,present", SCENARIOS, ids=[s[0] for s in SCENARIOS])
def test_every_interleaving_inserts_each_key_once(name, table, threads, present, first_retry):
    states, finals = Model(B=2, S=2, first_retry=first_retry).explore(table, threads)
    assert states > 50  # the scenario does interleave
    check_finals(finals, threads, present)


@pytest.mark.parametrize("name,B,S,table,threads,present", BIG, ids=[s[0] for s in BIG])
def test_every_interleaving_on_larger_tables(name, B, S, table, threads, present):
    states, finals = Model(B=B, S=S).explore(table, threads)
    assert states > 1000
    check_finals(finals, threads, present)


def test_the_check_catches_a_broken_protocol():
    """A protocol that takes a stale first slot without the compare-and-swap
    (a plain store) loses a duplicate race: the exploration must find it."""
    class Broken(Model):
        def step(self, table, th):
            if th[3] == "retry":  # store without comparing
                kind, key, home = th[:3]
                table = table[:home * self.S] + (key,) + table[home * self.S + 1:]
                return table, (kind, key, home, "done") + th[4:10] + (1,)
            return super().step(table, th)
    table, threads = (X, 0, Y, 0), [("cas_first", K1, 0), ("cas_first", K1, 0)]
    _, finals = Broken(B=2, S=2).explore(table, threads)
    with pytest.raises(AssertionError):
        check_finals(finals, threads, set())
