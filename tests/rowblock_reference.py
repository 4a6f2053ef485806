"""Test helpers for the row-block condensation (Sec. 2.1, Fig. 6).

`oracle_rowblock` runs the same schedule with the oracle's single-step
condensation (natural column order, pivot column removed), so its pivot values
and labels are what any correct implementation of the schedule must produce;
`HostSteps` is a CPU stand-in for the device steps (torch FP64, not fused), for
multi-rank tests without a GPU.
"""
import math

import numpy as np
import torch

from oracle import core as oracle


def paper_schedule(counts):
    """(rank, local row) per step: the loops of Fig. 6, each rank keeping its last row."""
    out = []
    for i in range(max(counts) - 1):
        for p, c in enumerate(counts):
            if i < c - 1:
                out.append((p, i))
    return out


def oracle_rowblock(A, counts):
    """(sign, log|det|, pivot labels, pivot values) of the row-block schedule, each
    step one oracle condense_once around (k, l) with l = argmax |a_kj| (ties to
    the smallest original column: the remaining labels stay in increasing order,
    so the first maximum), the last rows finished by the oracle sweep."""
    A = np.array(A, dtype=np.float64)
    rows = [(p, i) for p, c in enumerate(counts) for i in range(c)]
    labels = list(range(A.shape[0]))
    sign, logs, lab, piv = 1.0, [], [], []
    for (p, i) in paper_schedule(counts):
        k = rows.index((p, i))
        l = int(np.argmax(np.abs(A[k])))
        lab.append(labels[l])
        piv.append(float(A[k, l]))
        A, f = oracle.condense_once(A, k, l)
        sign *= -1.0 if f < 0 else 1.0
        logs.append(math.log(abs(f)))
        del labels[l]
        del rows[k]
    fin = oracle.logdet(A)
    return sign * fin.sign, math.fsum(logs + [fin.logabs]), lab, piv


class HostSteps:
    """CPU stand-in for the device steps on FP64 torch tensors."""

    def factor(self, row, labels, m, step):
        a = row[:m].clone()
        mx = a.abs().max()
        cand = torch.nonzero(a.abs() == mx).flatten()
        l = int(cand[torch.argmin(labels[cand])])
        p = float(a[l])
        a[l] = a[m - 1]
        row[:m - 1] = a[:m - 1] / p
        row[m - 1] = p
        step.copy_(torch.tensor([l, p, 0.0 if p != 0 else 1.0, float(labels[l])],
                                dtype=torch.float64))

    def update(self, F, rows, m, r, labels, step):
        if step[2] != 0:
            return
        l = int(step[0])
        if rows > 0:
            c = F[:, l].clone()
            F[:, l] = F[:, m - 1]
            F[:, :m - 1] -= c[:, None] * r[None, :m - 1]
            F[:, m - 1] = c
        t = int(labels[l])
        labels[l] = labels[m - 1]
        labels[m - 1] = t

    def small(self, M):
        res = oracle.logdet(M.numpy())
        return res.sign, res.logabs
