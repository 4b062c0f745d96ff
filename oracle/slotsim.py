"""Cleartext slot simulator (O2): the layer backend on FP64 slot vectors.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Rot(v, r) is ``np.roll(v, -r)`` (paper Sec. II-B: slot j+r moves to slot j),
Mul (P) is the elementwise product with the mask, square is v*v.  Each vector
carries the number of levels it has consumed: rescale adds one, and Add (C)
refuses operands of different levels, as a CKKS library would.  Running
``layers`` on this backend checks the paper's slot algorithms against the FP64
CNN without encryption, and its level accounting against the #Mult tables.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class SV:
    v: np.ndarray
    used: int = 0        # levels consumed so far
    pending_rescale: bool = False


class SlotSim:
    def __init__(self):
        self.count = {"rot": 0, "pmul": 0, "rescale": 0, "square": 0}

    @staticmethod
    def wrap(v):
        return SV(np.asarray(v, dtype=np.float64))

    @staticmethod
    def levels_left(x):
        return None        # cleartext: no level budget, Drop-Level never applies

    def rot(self, x, r):
        self.count["rot"] += 1
        return SV(np.roll(x.v, -r), x.used, x.pending_rescale)

    def rot_many(self, x, steps):
        self.count["rot"] += len({s for s in steps if s % len(x.v)})
        return {s: SV(np.roll(x.v, -s), x.used, x.pending_rescale) for s in steps}

    def lincomb_diag(self, xs, steps):
        m = len(xs[0].v)
        self.count["rot"] += len([s for s in steps if s % m])
        for x in xs[1:]:
            assert x.used == xs[0].used and not x.pending_rescale
        return SV(sum(np.roll(x.v, -s) for x, s in zip(xs, steps)), xs[0].used, False)

    def lincomb_chan_rescale(self, xs, steps, weights):
        m = len(xs[0].v)
        self.count["rot"] += sum(len({s % m for s in st if s % m}) for st in steps)
        self.count["pmul"] += sum(len(w) for w in weights)
        self.count["rescale"] += 1
        for x in xs[1:]:
            assert x.used == xs[0].used and not x.pending_rescale
        v = sum(np.roll(x.v, -s) * w for x, st, ws in zip(xs, steps, weights) for s, w in zip(st, ws))
        return SV(v, xs[0].used + 1, False)

    def lincomb(self, xs, steps, weights):
        m = len(xs[0].v)
        self.count["rot"] += len(xs) * len({s % m for s in steps if s % m})
        for x in xs[1:]:
            assert x.used == xs[0].used and not x.pending_rescale
        if weights is None:
            v = sum(np.roll(x.v, -s) for x in xs for s in steps)
            return [SV(v, xs[0].used, False)]
        outs = []
        for wo in weights:
            v = np.zeros(m)
            for i, x in enumerate(xs):
                for s, w in zip(steps, wo[i]):
                    self.count["pmul"] += 1
                    v = v + np.roll(x.v, -s) * w
            outs.append(SV(v, xs[0].used, True))
        return outs

    def lincomb_rescale(self, xs, steps, weights):
        return [self.rescale(y) for y in self.lincomb(xs, steps, weights)]

    def mul_rescale_to(self, x, v, target):
        assert not x.pending_rescale and not target.pending_rescale and x.used < target.used
        self.count["pmul"] += 1
        self.count["rescale"] += 1
        return SV(x.v * v, target.used, False)

    def add(self, x, y):
        assert x.used == y.used and x.pending_rescale == y.pending_rescale, "level mismatch"
        return SV(x.v + y.v, x.used, x.pending_rescale)

    def mul_mask(self, x, v):
        assert not x.pending_rescale
        self.count["pmul"] += 1
        return SV(x.v * v, x.used, True)

    def add_mask(self, x, v):
        return SV(x.v + v, x.used, x.pending_rescale)

    def rescale(self, x):
        assert x.pending_rescale
        self.count["rescale"] += 1
        return SV(x.v, x.used + 1, False)

    def square(self, x):
        assert not x.pending_rescale
        self.count["square"] += 1
        return SV(x.v * x.v, x.used + 1, False)
