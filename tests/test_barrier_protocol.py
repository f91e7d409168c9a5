"""A model of the tensor-core prediction kernel's mbarrier protocol (single
space, the roles of csrc/bo_predict_tc.cu: K* producers, one or two MMA
issuers, the accumulator epilogue, the bulk-copy loaders), run under random
interleavings.  mbarriers are modelled exactly as the hardware defines them
(arrival count, phase parity, try_wait on a parity); MMA completion and copy
landing are immediate.  Every pipeline shape the autotuner tries must finish
without a deadlock.  (A shared B ring for two issuers deadlocks here, as it
timed out on the GPU: an issuer that skips the other's pieces can run a full
ring ahead of the loader and take an older phase of the same parity.)"""
import random

import pytest


class Bar:
    def __init__(self, count):
        self.count, self.pending, self.phase = count, count, 0

    def arrive(self):
        self.pending -= 1
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count

    def done(self, parity):          # try_wait.parity: the phase of that parity has completed
        return (self.phase & 1) != parity


def pieces(c, cw, n_pad):
    """The L^-1 pieces of chunk c: region r's rows [max(c cw, 256 r), min(256 (r+1), n_pad))."""
    out = []
    for r in (0, 1):
        lo, hi = max(c * cw, 256 * r), min(256 * (r + 1), n_pad)
        if lo < hi:
            out.append(r)
    return out


def run(SA, b_slots, n_pad, shared_ring=False, tiles=4, cw=32, seed=0, max_steps=400_000, split_loaders=True):
    rnd = random.Random(seed)
    chunks = n_pad // cw
    issuers = 2 if n_pad > 256 else 1
    stages = 2 if n_pad <= 256 else 1        # accumulator buffers (2 x n_pad columns fit in TMEM)
    if issuers == 1 or shared_ring:
        ring = [b_slots, 0] if not shared_ring else [b_slots, b_slots]
    else:
        ring = [b_slots - b_slots // 2, b_slots // 2]
    a_full = [Bar(1) for _ in range(SA)]
    a_empty = [Bar(issuers) for _ in range(SA)]
    nb = b_slots if shared_ring or issuers == 1 else b_slots
    b_full = [Bar(1) for _ in range(nb)]
    b_empty = [Bar(1) for _ in range(nb)]
    base = [0, 0 if shared_ring else ring[0]]
    acc_full = [Bar(1) for _ in range(32)]
    acc_empty = [Bar(4) for _ in range(2)]
    mu_full, mu_empty = [Bar(1) for _ in range(2)], [Bar(1) for _ in range(2)]

    def slot_seq(rme):                # the slots issuer rme (or, None, the loader) uses, in order
        pos = [0, 0]
        ph = [0, 0]
        for _ in range(tiles):
            for c in range(chunks):
                for r in pieces(c, cw, n_pad):
                    k = 0 if shared_ring else r
                    if rme is None or r == rme:
                        yield c, r, base[k] + pos[k], ph[k]
                    if rme is None or r == rme or shared_ring:
                        pos[k] += 1
                        if pos[k] == ring[k]:
                            pos[k] = 0
                            ph[k] ^= 1

    def producer():
        s = ph = 0
        for t in range(tiles):
            for _ in range(chunks):
                while not a_empty[s].done(ph ^ 1):
                    yield
                a_full[s].arrive()
                s = (s + 1) % SA
                ph ^= s == 0
            while not mu_empty[t & 1].done(((t >> 1) & 1) ^ 1):
                yield
            mu_full[t & 1].arrive()

    def issuer(rme):
        mine = slot_seq(rme)
        sa = pha = 0
        fill = [0, 0]                 # tiles started per accumulator buffer
        for t in range(tiles):
            buf = t % stages
            for c in range(chunks):
                s = sa
                while not a_full[s].done(pha):
                    yield
                if rme in pieces(c, cw, n_pad):
                    _, _, slot, ph = next(mine)
                    if c == 0:
                        while not acc_empty[buf + rme].done((fill[buf] & 1) ^ 1):
                            yield
                        fill[buf] += 1
                    while not b_full[slot].done(ph):
                        yield
                    b_empty[slot].arrive()
                a_empty[s].arrive()
                if issuers == 1 or (c * cw) >> 8 == rme:
                    acc_full[buf * 16 + c].arrive()      # column block c is final
                sa = (sa + 1) % SA
                pha ^= sa == 0

    def epilogue():
        par = [0, 0]
        for t in range(tiles):
            buf = t % stages
            for c in range(chunks):
                while not acc_full[buf * 16 + c].done((par[buf] >> c) & 1):
                    yield
                par[buf] ^= 1 << c
                kend = c * cw + cw
                if kend == n_pad or kend % 256 == 0:
                    for _ in range(4):
                        acc_empty[buf + ((kend - 1) >> 8)].arrive()
            while not mu_full[t & 1].done((t >> 1) & 1):
                yield
            mu_empty[t & 1].arrive()

    def loader(region):               # region None: every piece, in chunk order
        for _, _, slot, ph in slot_seq(region):
            while not b_empty[slot].done(ph ^ 1):
                yield
            b_full[slot].arrive()

    live = {"producers": producer(), "epilogue": epilogue(), "issuer0": issuer(0)}
    if issuers == 2:
        live["issuer1"] = issuer(1)
    if issuers == 2 and split_loaders and not shared_ring:
        live["loader0"], live["loader1"] = loader(0), loader(1)   # one loader per region's ring
    else:
        live["loader"] = loader(None)
    stalled = 0
    for _ in range(max_steps):
        if not live:
            return "ok"
        name = rnd.choice(sorted(live))
        try:
            next(live[name])
            stalled += 1
        except StopIteration:
            del live[name]
            stalled = 0
        if stalled > 20_000:
            return "deadlock"
    return "unfinished"


SHAPES = [(sa, bs) for sa in (2, 3, 4, 6, 8) for bs in (2, 3, 4, 6)]


@pytest.mark.parametrize("n_pad", [224, 288, 512])
@pytest.mark.parametrize("split_loaders", [True, False])
def test_every_shape_completes(n_pad, split_loaders):
    for sa, bs in SHAPES:
        for seed in range(3):
            assert run(sa, bs, n_pad, seed=seed, split_loaders=split_loaders) == "ok", (n_pad, sa, bs, seed)


def test_model_finds_the_shared_ring_deadlock():
    """The model is sharp enough to see the bug the per-region rings fix."""
    outcomes = {run(8, 2, 512, shared_ring=True, seed=s) for s in range(6)}
    assert "deadlock" in outcomes
