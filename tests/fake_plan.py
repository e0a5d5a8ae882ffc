"""A CPU stand-in for ``binding.Plan`` built on the FP64 oracle (test infrastructure only).

It keeps the same raw per-level statistics as the C library (N, the sum of D, the sum of
||D||_F^2), evaluates samples with ``oracle.sample`` and applies the same allocation rule
(Remark 3.6 with C_0 = c_0, C_l = c_l + c_{l-1}), so the host-side drivers can be run on CPU
processes.  It records every sample id it evaluates.
"""
import math

import numpy as np
import torch

import oracle


class FakePlan:
    def __init__(self, pps, *, c0, L, ratio=2, pilot_n=8, nl_scale=1.0, fkind=0):
        self.problems = list(pps)
        self.levels = [L] * len(self.problems)
        self.c0, self.ratio, self.L = c0, ratio, L
        self.pilot_n = pilot_n
        self.nl_scale = nl_scale
        self.fkind = fkind
        self.device = torch.device("cpu")
        self._orc = [oracle.Problem(*pp.f64(), seed_A=pp.seed_A, seed_B=pp.seed_B, seed_idx=pp.seed_idx,
                                    problem_id=pp.problem_id) for pp in self.problems]
        self._lv = oracle.Levels(c0, ratio, L)
        self.state = {}
        self.evaluated = {}
        for q, pp in enumerate(self.problems):
            m, _, p = pp.shape
            for l in range(L + 1):
                self.state[(q, l)] = [0, torch.zeros(m, p, dtype=torch.float64), 0.0]
                self.evaluated[(q, l)] = []

    def level_stats(self, q, l, begin, count):
        st = self.state[(q, l)]
        for s in range(begin, begin + count):
            D = oracle.sample(self._orc[q], self._lv, l, s, fkind=self.fkind)[0]
            st[1] += torch.from_numpy(D)
            st[2] += float((D * D).sum())
            self.evaluated[(q, l)].append(s)
        st[0] += count

    def level_stats_batch(self, ranges):
        for q, l, b, c in ranges:
            self.level_stats(q, l, b, c)

    def get_level_state(self, q, l):
        N, s, sq = self.state[(q, l)]
        return N, s.clone(), sq

    def set_level_state(self, q, l, N, s, sq):
        self.state[(q, l)] = [int(N), s.clone().to(torch.float64), float(sq)]

    def reset(self, q, l=-1):
        levels = range(self.L + 1) if l < 0 else [l]
        for ll in levels:
            m, _, p = self.problems[q].shape
            self.state[(q, ll)] = [0, torch.zeros(m, p, dtype=torch.float64), 0.0]

    def cl(self, l):
        return self.c0 * self.ratio ** l

    def allocate(self, eps_abs):
        out = []
        for q in range(len(self.problems)):
            V, C = [], []
            for l in range(self.L + 1):
                N, s, sq = self.state[(q, l)]
                M2 = sq - float((s * s).sum()) / N
                V.append(max(0.0, M2 / (N - 1)))
                C.append(self.cl(0) if l == 0 else self.cl(l) + self.cl(l - 1))
            root = sum(math.sqrt(v * c) for v, c in zip(V, C))
            out.append([max(self.pilot_n, int(math.ceil(self.nl_scale * 2.0 / eps_abs[q]**2 * math.sqrt(v / c) * root)))
                        for v, c in zip(V, C)])
        return out

    def telescoping_sum(self):
        out = []
        for q in range(len(self.problems)):
            Y = None
            for l in range(self.L + 1):
                N, s, _ = self.state[(q, l)]
                if N == 0:   # levels never run add nothing (as in the C library)
                    continue
                Y = s / N if Y is None else Y + s / N
            out.append(Y)
        return out
