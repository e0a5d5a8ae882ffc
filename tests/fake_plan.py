"""A CPU stand-in for ``binding.Plan`` built on the FP64 oracle (test infrastructure only).

It keeps the same per-level statistics as the C library (N, the sum of D, and
M2 = sum_s ||D_s - mean||_F^2 grown by Welford's update sample by sample, states merged by
Chan's pairwise update), evaluates samples with ``oracle.sample`` and applies the same allocation
rule (Remark 3.6 with C_0 = c_0, C_l = c_l + c_{l-1}) and stopping test (Remark 3.5), so the
host-side drivers can be run on CPU processes.  It records every sample id it evaluates.
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
            D = torch.from_numpy(oracle.sample(self._orc[q], self._lv, l, s, fkind=self.fkind)[0])
            k = st[0]
            if k > 0:
                st[2] += float(((k * D - st[1]) ** 2).sum()) / (k * (k + 1))
            st[1] += D
            st[0] += 1
            self.evaluated[(q, l)].append(s)

    def level_stats_batch(self, ranges):
        for q, l, b, c in ranges:
            self.level_stats(q, l, b, c)

    def get_level_state(self, q, l):
        N, s, sq = self.state[(q, l)]
        return N, s.clone(), sq

    def set_level_state(self, q, l, N, s, M2):
        self.state[(q, l)] = [int(N), s.clone().to(torch.float64), float(M2)]

    def merge_level_state(self, q, l, N, s, M2):
        st = self.state[(q, l)]
        N = int(N)
        if N == 0:
            return
        s = s.to(torch.float64)
        if st[0] > 0:
            d = s / N - st[1] / st[0]
            st[2] += float(M2) + st[0] * N / (st[0] + N) * float((d * d).sum())
        else:
            st[2] = float(M2)
        st[1] = st[1] + s
        st[0] += N

    def reset(self, q, l=-1):
        levels = range(self.L + 1) if l < 0 else [l]
        for ll in levels:
            m, _, p = self.problems[q].shape
            self.state[(q, ll)] = [0, torch.zeros(m, p, dtype=torch.float64), 0.0]

    def cl(self, l):
        return self.c0 * self.ratio ** l

    def allocate_levels(self, q, L, eps):
        V, C = [], []
        for l in range(L + 1):
            N, _, M2 = self.state[(q, l)]
            V.append(max(0.0, M2 / (N - 1)))
            C.append(self.cl(0) if l == 0 else self.cl(l) + self.cl(l - 1))
        root = sum(math.sqrt(v * c) for v, c in zip(V, C))
        return [max(self.pilot_n, int(math.ceil(self.nl_scale * 2.0 / eps**2 * math.sqrt(v / c) * root)))
                for v, c in zip(V, C)]

    def allocate(self, eps_abs):
        return [self.allocate_levels(q, self.L, eps_abs[q]) for q in range(len(self.problems))]

    def bias_test(self, q, L, eps):
        N, s, _ = self.state[(q, L)]
        nrm = float(torch.linalg.norm(s)) / N if N > 0 else 0.0
        return L >= 2 and nrm < (math.sqrt(self.ratio) + 1.0) * eps / math.sqrt(2.0), nrm

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
