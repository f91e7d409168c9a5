"""Acquisition-function selection of Sec. III-G: 'multi' and 'advanced multi'.

Test infrastructure only (see the package docstring).  Parity unpinned
against the paper, which prints no trace of either procedure; the readings
below are pinned by scripted scenarios in tests/test_oracle_selection.py.

Readings of Sec. III-G and Table I taken here:
  * One prediction pass per round; every active AF contributes one pick from
    those shared predictions, in the order (ei, poi, lcb) of Table I.
  * dos (discounted observation score) of an AF: dos <- gamma * dos + o for
    each observation o of a candidate that AF picked, i.e.
    dos_t = sum_i o_i gamma^(t-i) over that AF's own observations, raw units.
    An invalid observation enters as the median of all valid observations so
    far (the paper states this for advanced multi; multi uses it too, which
    keeps the score finite).  gamma = 0.65 (multi) / 0.75 (advanced multi).
  * multi: for every pair of AFs whose picks coincide in a round, both
    AFs' duplicate counts grow by one and they become partners; the shared
    candidate is evaluated once and credited to each of them.  At the start
    of a round, if some active AF's count exceeds the skip threshold (5),
    that AF and its partners are pitted against each other: the lowest dos
    (ties: earlier AF) stays, the others are skipped for good, and all
    counts and partners are reset.
  * advanced multi: an AF's pick is the best candidate not already picked by
    an earlier AF in the round.  At the start of every round after the
    first, with two or more AFs active and m the mean dos over them, an AF
    with dos > m (1 + rif) gains an 'over' count and one with dos < m (1 - rif)
    an 'under' count (cumulative; rif = 0.1).  The first AF (in order) whose
    under count reaches the skip threshold becomes the only AF; otherwise the
    first whose over count reaches it is skipped and the counts of the rest
    are reset.
"""
from __future__ import annotations

__all__ = ["SingleSelector", "MultiSelector", "AdvancedMultiSelector", "make_selector"]


class SingleSelector:
    def __init__(self, af):
        self.active = [af]
        self.dos = {af: 0.0}

    def begin_round(self):
        pass

    def assign(self, topk):
        a = self.active[0]
        return [(topk[a][0][0], [a])] if topk[a] else []

    def credit(self, afs, value):
        pass


class MultiSelector:
    def __init__(self, afs=("ei", "poi", "lcb"), skip_threshold=5, discount=0.65):
        self.active = list(afs)
        self.order = list(afs)
        self.threshold = skip_threshold
        self.gamma = discount
        self.dos = {a: 0.0 for a in afs}
        self.dup = {a: 0 for a in afs}
        self.partners = {a: set() for a in afs}
        self.rounds = 0

    def begin_round(self):
        if self.rounds > 0:
            exceeded = [a for a in self.active if self.dup[a] > self.threshold]
            if exceeded:
                group = set(exceeded)
                for a in exceeded:
                    group |= self.partners[a]
                group &= set(self.active)
                keep = min(group, key=lambda a: (self.dos[a], self.order.index(a)))
                self.active = [a for a in self.active if a not in group or a == keep]
                for a in self.order:
                    self.dup[a] = 0
                    self.partners[a] = set()
        self.rounds += 1

    def assign(self, topk):
        picks = []                       # [idx, [afs]] in AF order
        for a in self.active:
            if not topk[a]:
                continue
            i = topk[a][0][0]
            for p in picks:
                if p[0] == i:
                    for b in p[1]:
                        self.dup[a] += 1
                        self.dup[b] += 1
                        self.partners[a].add(b)
                        self.partners[b].add(a)
                    p[1].append(a)
                    break
            else:
                picks.append([i, [a]])
        return [(i, afs) for i, afs in picks]

    def credit(self, afs, value):
        for a in afs:
            self.dos[a] = self.gamma * self.dos[a] + value


class AdvancedMultiSelector:
    def __init__(self, afs=("ei", "poi", "lcb"), skip_threshold=5, discount=0.75, rif=0.1):
        self.active = list(afs)
        self.order = list(afs)
        self.threshold = skip_threshold
        self.gamma = discount
        self.rif = rif
        self.dos = {a: 0.0 for a in afs}
        self.over = {a: 0 for a in afs}
        self.under = {a: 0 for a in afs}
        self.rounds = 0

    def begin_round(self):
        if self.rounds > 0 and len(self.active) >= 2:
            m = sum(self.dos[a] for a in self.active) / len(self.active)
            for a in self.active:
                if self.dos[a] > m * (1.0 + self.rif):
                    self.over[a] += 1
                elif self.dos[a] < m * (1.0 - self.rif):
                    self.under[a] += 1
            promoted = [a for a in self.active if self.under[a] >= self.threshold]
            if promoted:
                self.active = [promoted[0]]
            else:
                skipped = [a for a in self.active if self.over[a] >= self.threshold]
                if skipped:
                    self.active.remove(skipped[0])
                    for a in self.active:
                        self.over[a] = 0
                        self.under[a] = 0
        self.rounds += 1

    def assign(self, topk):
        taken = set()
        picks = []
        for a in self.active:
            for i, _ in topk[a]:
                if i not in taken:
                    taken.add(i)
                    picks.append((i, [a]))
                    break
        return picks

    def credit(self, afs, value):
        for a in afs:
            self.dos[a] = self.gamma * self.dos[a] + value


def make_selector(af, skip_threshold=5, discount=None, rif=0.1):
    if af in ("ei", "poi", "lcb"):
        return SingleSelector(af)
    if af == "multi":
        return MultiSelector(skip_threshold=skip_threshold,
                             discount=0.65 if discount is None else discount)
    if af == "advanced_multi":
        return AdvancedMultiSelector(skip_threshold=skip_threshold, rif=rif,
                                     discount=0.75 if discount is None else discount)
    raise ValueError(af)
